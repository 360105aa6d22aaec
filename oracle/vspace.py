"""Velocity quadrature and quadtree level spaces (oracle; test infrastructure only).

Sec. 2.3 (discrete velocity formulation): the velocity set is a uniform Cartesian grid with
Newton--Cotes weights.  The paper does not name the Newton--Cotes order; every grid size it
uses is 4k+1, so the default here is the composite Boole (5-point closed) rule, with Simpson
and trapezoid kept as options.

Sec. 3.1-3.2: coarser velocity cells are formed by merging adjacent base cells of a
quadtree-structured reference grid.  A merged cell carries the summed weight and the
weight-averaged coordinate (Eq. hierarchical_projection_operator and the two relations
under it).  Reading used for odd base sizes: per axis the centre node stays single and the
(n-1)/2 nodes on each side are grouped outward from the centre in runs of 2^L, the
remainder folded into the outermost group (101 -> 51 -> 25 -> 13, 201 -> 101 -> 51 -> 25).
A "2x2 block" of the coarsening index kappa is a product of two level-1 groups.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def newton_cotes_1d(n: int, umin: float, umax: float, rule: str = "boole"):
    """Nodes and weights of a closed composite Newton--Cotes rule on [umin, umax] (Sec. 2.3).

    boole:   panels of 4 intervals, weights 2h/45 * [7, 32, 12, 32, 7]
    simpson: panels of 2 intervals, weights h/3 * [1, 4, 1]
    trapz:   weights h * [1/2, 1, ..., 1, 1/2]
    """
    if n < 2:
        raise ValueError("need at least 2 nodes")
    x = np.linspace(umin, umax, n)
    h = (umax - umin) / (n - 1)
    w = np.zeros(n)
    if rule == "boole":
        if (n - 1) % 4:
            raise ValueError("Boole rule needs n = 4k+1 nodes")
        panel = np.array([7.0, 32.0, 12.0, 32.0, 7.0]) * (2.0 * h / 45.0)
        for p in range((n - 1) // 4):
            w[4 * p: 4 * p + 5] += panel
    elif rule == "simpson":
        if (n - 1) % 2:
            raise ValueError("Simpson rule needs an odd node count")
        panel = np.array([1.0, 4.0, 1.0]) * (h / 3.0)
        for p in range((n - 1) // 2):
            w[2 * p: 2 * p + 3] += panel
    elif rule == "trapz":
        w[:] = h
        w[0] = w[-1] = 0.5 * h
    else:
        raise ValueError(rule)
    return x, w


def axis_groups(n: int, L: int):
    """Index groups of one axis at coarsening level L (reading of Sec. 3.2 for odd n).

    Returns a list of index lists in ascending order.  Level 0 is every node on its own.
    """
    if n % 2 != 1:
        raise ValueError("the level rule needs an odd base size")
    if L == 0:
        return [[i] for i in range(n)]
    c = (n - 1) // 2
    m = c
    size = 2 ** L
    ng = max(1, m // size)
    right = []
    for g in range(ng):
        lo = c + 1 + g * size
        hi = c + (g + 1) * size if g < ng - 1 else n - 1
        right.append(list(range(lo, hi + 1)))
    left = [[2 * c - i for i in reversed(grp)] for grp in reversed(right)]
    return left + [[c]] + right


@dataclass
class Base:
    """Reference grid V_base: tensor product of one 1-D rule per axis (Sec. 3.1)."""
    x: np.ndarray          # 1-D nodes
    w: np.ndarray          # 1-D weights
    D: int                 # velocity dimension (1 or 2)

    @property
    def n(self):
        return len(self.x)


@dataclass
class Space:
    """A discrete velocity space described on V_base.

    xi   (Nv, D)   velocity coordinates (weighted means of the covered base nodes)
    w    (Nv,)     quadrature weights (sums of the covered base weights)
    rect (Nv, 2D)  covered base index ranges [x0, x1) (and [y0, y1))
    owner          base-shaped array: index of the cell covering each base node
    Secs. 3.1-3.2.
    """
    xi: np.ndarray
    w: np.ndarray
    rect: np.ndarray
    owner: np.ndarray
    base: Base

    @property
    def nv(self):
        return len(self.w)


def _merge_1d(base: Base, groups):
    X = np.array([np.sum(base.w[g] * base.x[g]) / np.sum(base.w[g]) for g in groups])
    W = np.array([np.sum(base.w[g]) for g in groups])
    return X, W


def uniform_space(base: Base, L: int) -> Space:
    """Tensor-product space with every axis grouped at level L (Sec. 3.2 merging rules)."""
    groups = axis_groups(base.n, L)
    X, W = _merge_1d(base, groups)
    if base.D == 1:
        rect = np.array([[g[0], g[-1] + 1] for g in groups])
        owner = np.empty(base.n, dtype=np.int64)
        for k, g in enumerate(groups):
            owner[g] = k
        return Space(X[:, None].copy(), W.copy(), rect, owner, base)
    ng = len(groups)
    xi = np.zeros((ng * ng, 2))
    w = np.zeros(ng * ng)
    rect = np.zeros((ng * ng, 4), dtype=np.int64)
    owner = np.empty((base.n, base.n), dtype=np.int64)   # [iy, ix]
    for gy in range(ng):
        for gx in range(ng):
            k = gy * ng + gx
            xi[k] = (X[gx], X[gy])
            w[k] = W[gx] * W[gy]
            rect[k] = (groups[gx][0], groups[gx][-1] + 1, groups[gy][0], groups[gy][-1] + 1)
            owner[groups[gy][0]:groups[gy][-1] + 1, groups[gx][0]:groups[gx][-1] + 1] = k
    return Space(xi, w, rect, owner, base)


def aniso_space(base: Base, Lx: int, Ly: int) -> Space:
    """Tensor-product space with the x axis grouped at level Lx and the y axis at Ly (2-D).
    (the projection sequence of Sec. 4.1.2)."""
    gx, gy = axis_groups(base.n, Lx), axis_groups(base.n, Ly)
    rect = np.array([(a[0], a[-1] + 1, b[0], b[-1] + 1) for b in gy for a in gx], dtype=np.int64)
    return space_from_rects(base, rect)


def level1_parent_maps(n: int, max_level: int = 3):
    """For each level L (1..max_level) the level-L group index of every level-1 group.
    (the quadtree of Sec. 3.2)."""
    g1 = axis_groups(n, 1)
    maps = {1: np.arange(len(g1))}
    for L in range(2, max_level + 1):
        gL = axis_groups(n, L)
        first = {}
        for k, g in enumerate(gL):
            for i in g:
                first[i] = k
        maps[L] = np.array([first[g[0]] for g in g1])
    return maps


def enforce_consistency(kappa: np.ndarray, n: int, max_level: int = 3) -> np.ndarray:
    """Parent-child consistency of a block coarsening index (Sec. 3.2, last paragraph).

    Reading: kappa_eff(b) is the largest L <= kappa(b) such that every level-1 block inside
    b's level-L parent has kappa >= L.  kappa has shape (N1, N1) = [by, bx] (2-D) or (N1,).
    """
    maps = level1_parent_maps(n, max_level)
    out = np.zeros_like(kappa)
    if kappa.ndim == 1:
        for b in range(kappa.shape[0]):
            best = 0
            for L in range(1, int(kappa[b]) + 1):
                members = maps[L] == maps[L][b]
                if np.all(kappa[members] >= L):
                    best = L
            out[b] = best
        return out
    N1 = kappa.shape[0]
    for by in range(N1):
        for bx in range(N1):
            best = 0
            for L in range(1, int(kappa[by, bx]) + 1):
                my = maps[L] == maps[L][by]
                mx = maps[L] == maps[L][bx]
                if np.all(kappa[np.ix_(my, mx)] >= L):
                    best = L
            out[by, bx] = best
    return out


def kappa_space(base: Base, kappa: np.ndarray, max_level: int = 3) -> Space:
    """Convert a block coarsening-index array to (xi, w) (Sec. 3.2, enclosing-mask paragraph).

    kappa is indexed by level-1 blocks; consistency is enforced first.  Cells are emitted in
    row-major order of their lower-left base index (y major, x minor).
    """
    n = base.n
    k_eff = enforce_consistency(np.asarray(kappa), n, max_level)
    gl = {L: axis_groups(n, L) for L in range(0, max_level + 1)}
    maps = level1_parent_maps(n, max_level)
    g1 = gl[1]
    cells = []  # (y0, x0, rect)
    if base.D == 1:
        seen = set()
        for b in range(len(g1)):
            L = int(k_eff[b])
            if L == 0:
                for i in g1[b]:
                    cells.append((0, i, (i, i + 1)))
            else:
                p = int(maps[L][b])
                if (L, p) in seen:
                    continue
                seen.add((L, p))
                g = gl[L][p]
                cells.append((0, g[0], (g[0], g[-1] + 1)))
    else:
        seen = set()
        for by in range(len(g1)):
            for bx in range(len(g1)):
                L = int(k_eff[by, bx])
                if L == 0:
                    for iy in g1[by]:
                        for ix in g1[bx]:
                            cells.append((iy, ix, (ix, ix + 1, iy, iy + 1)))
                else:
                    px, py = int(maps[L][bx]), int(maps[L][by])
                    if (L, px, py) in seen:
                        continue
                    seen.add((L, px, py))
                    gx, gy = gl[L][px], gl[L][py]
                    cells.append((gy[0], gx[0], (gx[0], gx[-1] + 1, gy[0], gy[-1] + 1)))
    cells.sort(key=lambda c: (c[0], c[1]))
    rect = np.array([c[2] for c in cells], dtype=np.int64)
    return space_from_rects(base, rect)


def space_from_rects(base: Base, rect: np.ndarray) -> Space:
    """Build (xi, w) for a partition of V_base into rectangles (Sec. 3.3.2 coarsening rules)."""
    nv = rect.shape[0]
    if base.D == 1:
        xi = np.zeros((nv, 1))
        w = np.zeros(nv)
        owner = -np.ones(base.n, dtype=np.int64)
        for k in range(nv):
            x0, x1 = rect[k]
            ww = base.w[x0:x1]
            w[k] = ww.sum()
            xi[k, 0] = np.sum(ww * base.x[x0:x1]) / w[k]
            owner[x0:x1] = k
    else:
        xi = np.zeros((nv, 2))
        w = np.zeros(nv)
        owner = -np.ones((base.n, base.n), dtype=np.int64)
        for k in range(nv):
            x0, x1, y0, y1 = rect[k]
            wx = base.w[x0:x1]
            wy = base.w[y0:y1]
            w[k] = wx.sum() * wy.sum()
            xi[k, 0] = np.sum(wx * base.x[x0:x1]) / wx.sum()
            xi[k, 1] = np.sum(wy * base.x[y0:y1]) / wy.sum()
            owner[y0:y1, x0:x1] = k
    if np.any(owner < 0):
        raise ValueError("rectangles do not cover the base grid")
    return Space(xi, w, rect, owner, base)


def make_base(n: int, umin: float, umax: float, D: int = 2, rule: str = "boole") -> Base:
    """Base grid of Sec. 2.3: Newton-Cotes nodes and weights per axis, their tensor product in 2-D."""
    x, w = newton_cotes_1d(n, umin, umax, rule)
    return Base(x, w, D)
