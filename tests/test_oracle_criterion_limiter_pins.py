"""Pins of the oracle's velocity-space criterion and unstructured limiter against values
computed here from the paper's definitions, independently of the oracle's code:

* the transport error of a merged block (Sec. 3.2, Eq. merge-transport-error with the S_r
  reading of the oracle's header) on a 5 x 5 base grid carrying two occupied corner blocks,
  evaluated in exact rational arithmetic node by node; the oracle's merge decision switches
  exactly at that value of eps_merge;
* the hierarchical scan of Sec. 3.2 (8x8, 4x4, then 2x2 candidate blocks, a merged parent
  skipping its children) by brute force: every candidate block's decision recomputed from
  Eq. block-contribution-indicator, Eq. block-hysteresis-rule and Eq. combined-merge-condition,
  and each level-1 block's expected index taken as the first level, from the coarsest down,
  whose block containing it merges;
* Venkatakrishnan's limiter (Sec. 2.2, Eq. reconstruction; the oracle's reading of eps^2) on a
  three-cell strip where it is active and the two one-sided increments differ, so that using
  the minimum where the maximum belongs (or the reverse) changes the result.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import criterion, kinetic, unstructured as un, vspace


# ------------------------------------------------------------------ transport error, by hand

def _boole5(h):
    """Composite Boole weights of 5 nodes with spacing h: 2h/45 [7, 32, 12, 32, 7]."""
    return [Fr(2, 45) * h * c for c in (7, 32, 12, 32, 7)]


def _exact_transport_error(g, x, w, block):
    """eps_B of Eq. merge-transport-error for block (list of (ix, iy)) with h = 0, in exact
    arithmetic: m = (g, xi_x g, xi_y g, |xi|^2 g / 2); F^s_{r,d} over the block's nodes with
    s xi_d >= 0; F~ from the merged point (weight sum, weighted mean coordinate, mean g and
    H = |xi|^2 g); S_r = max_d sum over all nodes of w |xi_d| |m_r|."""
    n = len(x)

    def m(gg, xx, yy, H):
        return [gg, xx * gg, yy * gg, H / 2]

    S = []
    for r in range(4):
        best = Fr(0)
        for d in range(2):
            tot = Fr(0)
            for iy in range(n):
                for ix in range(n):
                    xs = (x[ix], x[iy])
                    mr = m(g[iy][ix], xs[0], xs[1], (xs[0] ** 2 + xs[1] ** 2) * g[iy][ix])[r]
                    tot += w[ix] * w[iy] * abs(xs[d]) * abs(mr)
            best = max(best, tot)
        S.append(best)
    W = sum(w[ix] * w[iy] for ix, iy in block)
    xb = sum(w[ix] * w[iy] * x[ix] for ix, iy in block) / W
    yb = sum(w[ix] * w[iy] * x[iy] for ix, iy in block) / W
    gb = sum(w[ix] * w[iy] * g[iy][ix] for ix, iy in block) / W
    Hb = sum(w[ix] * w[iy] * (x[ix] ** 2 + x[iy] ** 2) * g[iy][ix] for ix, iy in block) / W
    mt = m(gb, xb, yb, Hb)
    err = Fr(0)
    for d in range(2):
        cb = (xb, yb)[d]
        for s in (1, -1):
            for r in range(4):
                F = Fr(0)
                for ix, iy in block:
                    xd = (x[ix], x[iy])[d]
                    if s * xd >= 0:
                        F += w[ix] * w[iy] * xd * m(g[iy][ix], x[ix], x[iy], (x[ix] ** 2 + x[iy] ** 2) * g[iy][ix])[r]
                Ft = W * cb * mt[r] if s * cb >= 0 else Fr(0)
                err = max(err, abs(F - Ft) / S[r])
    return err


def test_transport_error_of_a_corner_block_matches_the_hand_value():
    """5 x 5 Boole grid on [-2, 2]^2 (nodes -2..2, level-1 groups {0,1}, {2}, {3,4} per axis).
    g is nonzero on two corner blocks only: B = {x, y in {1, 2}} with (g(1,1), g(2,1), g(1,2),
    g(2,2)) = (3, 1, 2, 5) and B' = {x, y in {-2, -1}} with 4, 1, 1, 2; h = 0.  The merge of B
    is decided by the transport test alone (C_merge above any indicator): it merges exactly when
    eps_merge reaches eps_B."""
    x = [Fr(i) for i in (-2, -1, 0, 1, 2)]
    w = _boole5(Fr(1))
    g = [[Fr(0)] * 5 for _ in range(5)]                 # g[iy][ix]
    g[3][3], g[3][4], g[4][3], g[4][4] = Fr(3), Fr(1), Fr(2), Fr(5)
    g[0][0], g[0][1], g[1][0], g[1][1] = Fr(4), Fr(1), Fr(1), Fr(2)
    B = [(3, 3), (4, 3), (3, 4), (4, 4)]
    eps = _exact_transport_error(g, x, w, B)
    assert 1e-3 < float(eps) < 1.0                      # a merge that distorts the fluxes
    base = vspace.make_base(5, -2.0, 2.0, D=2)
    np.testing.assert_allclose(base.w, [float(v) for v in w], rtol=1e-15)
    G = np.array([[float(v) for v in row] for row in g])
    H = np.zeros_like(G)
    N1 = len(vspace.axis_groups(5, 1))
    z = np.zeros((N1, N1), int)
    k_hi = criterion.criterion_2d(G, H, base, z, 3.0, 2.0, eps_merge=float(eps) * (1 + 1e-9), max_level=1)
    k_lo = criterion.criterion_2d(G, H, base, z, 3.0, 2.0, eps_merge=float(eps) * (1 - 1e-9), max_level=1)
    assert k_hi[2, 2] == 1 and k_lo[2, 2] == 0          # block B is (by, bx) = (2, 2)


# ------------------------------------------------------------------ hierarchical scan, brute force

def _indicator(M1, M2, ix, iy):
    return max(sum(M1[j, i] for j in iy for i in ix), sum(M2[j, i] for j in iy for i in ix))


def _transport_error(g, h, X, Y, W, ix, iy):
    """Eq. merge-transport-error node by node (float), the oracle's S_r reading."""
    def m(gg, hh, xx, yy):
        return np.array([gg, xx * gg, yy * gg, 0.5 * (hh + (xx * xx + yy * yy) * gg)])
    ny, nx = g.shape
    S = np.zeros(4)
    for d, C in enumerate((X, Y)):
        tot = np.zeros(4)
        for j in range(ny):
            for i in range(nx):
                tot += W[j, i] * abs(C[j, i]) * np.abs(m(g[j, i], h[j, i], X[j, i], Y[j, i]))
        S = np.maximum(S, tot)
    nodes = [(j, i) for j in iy for i in ix]
    Wb = sum(W[j, i] for j, i in nodes)
    xb = sum(W[j, i] * X[j, i] for j, i in nodes) / Wb
    yb = sum(W[j, i] * Y[j, i] for j, i in nodes) / Wb
    gb = sum(W[j, i] * g[j, i] for j, i in nodes) / Wb
    Hb = sum(W[j, i] * (h[j, i] + (X[j, i] ** 2 + Y[j, i] ** 2) * g[j, i]) for j, i in nodes) / Wb
    mt = m(gb, Hb - (xb * xb + yb * yb) * gb, xb, yb)
    err = 0.0
    for d in range(2):
        cb = (xb, yb)[d]
        for s in (1.0, -1.0):
            F = np.zeros(4)
            for j, i in nodes:
                xd = (X[j, i], Y[j, i])[d]
                if s * xd >= 0:
                    F += W[j, i] * xd * m(g[j, i], h[j, i], X[j, i], Y[j, i])
            Ft = Wb * cb * mt if s * cb >= 0 else np.zeros(4)
            err = max(err, float(np.max(np.abs(F - Ft) / S)))
    return err


def _brute_kappa(g, h, base, kprev, C_split, C_merge, eps, max_level):
    n = base.n
    wg = np.outer(base.w, base.w) * g
    X, Y = np.meshgrid(base.x, base.x)
    W = np.outer(base.w, base.w)
    we = W * (h + (X ** 2 + Y ** 2) * g)
    M1, M2 = wg / wg.sum(), we / we.sum()
    g1 = vspace.axis_groups(n, 1)
    N1 = len(g1)
    # every candidate block at every level: its level-1 members and its decision
    decision = {}
    for L in range(1, max_level + 1):
        gL = vspace.axis_groups(n, L)
        for py, Gy in enumerate(gL):
            for px, Gx in enumerate(gL):
                bx = [b for b in range(N1) if g1[b][0] in Gx]
                by = [b for b in range(N1) if g1[b][0] in Gy]
                IB = _indicator(M1, M2, Gx, Gy)
                if IB < C_merge:
                    ok = eps is None or _transport_error(g, h, X, Y, W, Gx, Gy) <= eps
                elif IB <= C_split:
                    ok = all(kprev[j, i] >= L for j in by for i in bx)
                else:
                    ok = False
                for j in by:
                    for i in bx:
                        decision[(L, j, i)] = ok
    kap = np.zeros((N1, N1), int)
    for j in range(N1):
        for i in range(N1):
            for L in range(max_level, 0, -1):
                if decision[(L, j, i)]:
                    kap[j, i] = L
                    break
    return kap


def _state(n, umax, seed):
    """A drifted hot Maxwellian plus a cold beam: blocks of every kind of decision."""
    base = vspace.make_base(n, -umax, umax, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2)
    g1, h1 = kinetic.maxwell_gh(np.array(1.0), np.array([0.4, -0.2]), np.array(1.3), sp.xi, gas)
    g2, h2 = kinetic.maxwell_gh(np.array(0.15), np.array([-2.0, 1.0]), np.array(0.3), sp.xi, gas)
    return base, (g1 + g2).reshape(n, n), (h1 + h2).reshape(n, n)


@pytest.mark.parametrize("eps", [None, 2e-4], ids=["contribution", "with_transport_test"])
def test_hierarchical_scan_matches_brute_force(eps):
    n = 33
    base, g, h = _state(n, 6.0, 0)
    N1 = len(vspace.axis_groups(n, 1))
    rng = np.random.default_rng(20261202)
    for C_split, C_merge, kprev in [(5e-3, 2.5e-3, np.zeros((N1, N1), int)),
                                    (2e-2, 1e-3, rng.integers(0, 4, (N1, N1))),
                                    (1e-2, 2e-3, np.full((N1, N1), 3))]:
        got = criterion.criterion_2d(g, h, base, kprev, C_split, C_merge, eps_merge=eps, max_level=3)
        want = _brute_kappa(g, h, base, kprev, C_split, C_merge, eps, 3)
        np.testing.assert_array_equal(got, want)
        assert len(np.unique(got)) >= 3                  # the case exercises several levels


# ------------------------------------------------------------------ Venkatakrishnan limiter

def test_venkatakrishnan_limiter_on_an_active_three_cell_strip():
    """Three square cells of side 0.1 in a row with values 0, 1, 1.2 (one velocity).  The middle
    cell's least-squares gradient is (p2 - p0) / (2 dx) = 6 (its top and bottom faces are
    boundary faces whose reflected ghosts only enter the normal matrix).  Face increments
    d2 = 6 * (+-0.05) = +-0.3 against the neighbour extrema d1 = 0.2 (right, max - p1) and
    d1 = -1 (left, min - p1); eps^2 = (sqrt(area))^3 p1^2 = 1e-3.  Venkatakrishnan's function
    ((d1^2 + eps^2) d2 + 2 d2^2 d1) / (d1^2 + 2 d2^2 + d1 d2 + eps^2) / d2 gives
    0.0483 / 0.281 / 0.3 on the right face and 0.4803 / 1.481 / 0.3 on the left, so the limiter
    is the right face's 0.57295...; a swap of the extrema gives a different value."""
    dx = 0.1
    nodes = np.array([[i * dx, j * dx] for j in range(2) for i in range(4)])
    cells = [(0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6)]
    mesh = un.UMesh(nodes, cells)
    P = np.array([[0.0], [1.0], [1.2]])
    grad = un._gradients(P, mesh, "venkat")
    right = (0.0483 / 0.281) / 0.3
    left = (0.4803 / 1.481) / 0.3
    phi = min(1.0, right, left)
    assert phi == pytest.approx(0.572953736654804, rel=1e-12)
    np.testing.assert_allclose(grad[1, 0], [6.0 * phi, 0.0], rtol=1e-12, atol=1e-12)
    swapped = ((1 + 1e-3) * 0.3 + 2 * 0.09 * (-1.0)) / (1 + 0.18 - 0.3 + 1e-3) / 0.3
    assert abs(swapped - phi) > 0.1
    # unlimited: the plain least-squares gradient
    np.testing.assert_allclose(un._gradients(P, mesh, "none")[1, 0], [6.0, 0.0], rtol=1e-12, atol=1e-12)
