"""Velocity-space requirement of one cell (oracle; test infrastructure only).  Sec. 3.2.

Per-point contributions (Eq. M2): M1 = w g / sum w g, M2 = w (h + |xi|^2 g) / sum w (h + |xi|^2 g);
block indicator I_B = max(sum_B M1, sum_B M2) (Eq. block-contribution-indicator); three-regime
rule with hysteresis (Eq. block-hysteresis-rule); optional transport-error test
(Eq. merge-transport-error, Eq. combined-merge-condition); hierarchical scan of 8x8, then 4x4,
then 2x2 candidate blocks, a merged parent skipping its children.

Readings used:
 * Candidate blocks at level L (1, 2, 3) are products of the level-L axis groups of the base
   grid (vspace.axis_groups); the "2x2 blocks" that kappa indexes are the level-1 products.
 * The criterion is evaluated on the base grid after projecting the cell's stored (g~, h~)
   from its current space (refinement by inheritance, Sec. 3.3.2).
 * "Previous status": a candidate block in the band [C_merge, C_split] stays merged iff all
   of its level-1 blocks had kappa_prev >= L.  The initial kappa_prev is 0 (fine).
 * S_r = max_d sum_i w_i |xi_{i,d}| |m_r(xi_i)| over the whole base grid.
 * The merged-block flux F~ uses the merged cell of the block: weight sum, weight-averaged
   coordinate, aggregated g and H = h + |xi|^2 g (Sec. 3.3.2 coarsening).
"""
from __future__ import annotations

import numpy as np

from . import vspace


def _contrib(g, h, base):
    """M1, M2 on the base grid, shaped [ny, nx] (2-D) or [n] (1-D)."""
    xi = base.x
    if base.D == 1:
        w = base.w
        x2 = xi ** 2
    else:
        w = np.outer(base.w, base.w)
        X, Y = np.meshgrid(xi, xi)     # [iy, ix]
        x2 = X ** 2 + Y ** 2
    wg = w * g
    we = w * (h + x2 * g)
    return wg / wg.sum(), we / we.sum()


def _m_vectors(g, h, xs):
    """m(xi) = (g, xi_x g, xi_y g, (h + |xi|^2 g)/2) for points with coordinates xs (..., 2)."""
    x2 = np.sum(xs * xs, axis=-1)
    return np.stack([g, xs[..., 0] * g, xs[..., 1] * g, 0.5 * (h + x2 * g)], axis=-1)


def criterion_2d(g, h, base, kappa_prev, C_split, C_merge, eps_merge=None, max_level=3):
    """kappa (per level-1 block, [N1, N1] = [by, bx]) for one cell from base-grid (g, h) [ny, nx].
    Sec. 3.2, Eqs. block-contribution-indicator, block-hysteresis-rule, merge-transport-error,
    combined-merge-condition."""
    n = base.n
    M1, M2 = _contrib(g, h, base)
    groups = {L: vspace.axis_groups(n, L) for L in range(1, max_level + 1)}
    maps = vspace.level1_parent_maps(n, max_level)
    g1 = groups[1]
    N1 = len(g1)
    kappa = np.zeros((N1, N1), dtype=np.int64)
    done = np.zeros((N1, N1), dtype=bool)
    X, Y = np.meshgrid(base.x, base.x)
    W = np.outer(base.w, base.w)
    if eps_merge is not None:
        m_all = _m_vectors(g, h, np.stack([X, Y], axis=-1))            # [ny, nx, 4]
        S = np.max(np.stack([np.sum(W[..., None] * np.abs(X)[..., None] * np.abs(m_all), axis=(0, 1)),
                             np.sum(W[..., None] * np.abs(Y)[..., None] * np.abs(m_all), axis=(0, 1))]),
                   axis=0)                                              # S_r, r = 0..3

    def members(L, px, py):
        """level-1 block indices (by, bx) inside the level-L parent (px, py)."""
        bx = np.nonzero(maps[L] == px)[0]
        by = np.nonzero(maps[L] == py)[0]
        return bx, by

    def transport_ok(ix, iy):
        if eps_merge is None:
            return True
        sl = (slice(iy[0], iy[-1] + 1), slice(ix[0], ix[-1] + 1))
        w = W[sl]
        gg, hh = g[sl], h[sl]
        xs = np.stack([X[sl], Y[sl]], axis=-1)
        m = _m_vectors(gg, hh, xs)
        wsum = w.sum()
        xb = np.array([np.sum(w * X[sl]), np.sum(w * Y[sl])]) / wsum
        gb = np.sum(w * gg) / wsum
        Hb = np.sum(w * (hh + (X[sl] ** 2 + Y[sl] ** 2) * gg)) / wsum
        hb = Hb - np.sum(xb ** 2) * gb
        mb = _m_vectors(np.array(gb), np.array(hb), xb)
        err = 0.0
        for d in range(2):
            xd = xs[..., d]
            for s in (+1.0, -1.0):
                sel = (s * xd >= 0)
                F = np.sum((w * xd * sel)[..., None] * m, axis=(0, 1))
                Ft = (wsum * xb[d] * mb) if s * xb[d] >= 0 else np.zeros(4)
                err = max(err, float(np.max(np.abs(F - Ft) / S)))
        return err <= eps_merge

    def decide(L, px, py):
        bx, by = members(L, px, py)
        ix = [i for b in bx for i in g1[b]]
        iy = [i for b in by for i in g1[b]]
        sl = (slice(min(iy), max(iy) + 1), slice(min(ix), max(ix) + 1))
        IB = max(M1[sl].sum(), M2[sl].sum())
        if IB < C_merge:
            return transport_ok(sorted(ix), sorted(iy))
        if IB <= C_split:
            return bool(np.all(kappa_prev[np.ix_(by, bx)] >= L))
        return False

    def scan(L, px, py):
        if decide(L, px, py):
            bx, by = members(L, px, py)
            kappa[np.ix_(by, bx)] = L
            return
        if L == 1:
            return
        # children at level L-1 inside this parent
        bx, by = members(L, px, py)
        cx = sorted(set(maps[L - 1][bx])) if L - 1 > 1 else sorted(set(bx))
        cy = sorted(set(maps[L - 1][by])) if L - 1 > 1 else sorted(set(by))
        for qy in cy:
            for qx in cx:
                scan(L - 1, qx, qy)

    nL = len(groups[max_level])
    for py in range(nL):
        for px in range(nL):
            scan(max_level, px, py)
    return kappa


def kappa_min(kappa):
    """min over blocks: the coarsest uniform level that encloses the requirement.  Sec. 3.2."""
    return int(np.min(kappa))
