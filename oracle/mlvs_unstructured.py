"""Multi-level DUGKS step on an unstructured mesh of polygonal cells (oracle; test
infrastructure only).

Sec. 3.4 on the unstructured step of `unstructured` (the two-cavity expansion of Sec. 4 is an
MLVS run on unstructured cells).  Every cell carries (g~, h~) on its own representative space.
A face is evaluated on V_f, the common refinement of its two cells' spaces; the two cells and
the cells across their faces (the stencil of their least-squares gradients) are represented on
V_f by projection plus the moment-constrained correction with their own moments as targets
(Eq. interface_state_moment_matching), as in `mlvs.step`.  On V_f the face follows the
unstructured step (gradient, limiter, upwind reconstruction at the midpoint, face model and
recovery, diffuse walls); the microflux (xi.n) phi returns to each cell's space with the flux
correction (Eq. native_flux_moment_matching) and updates it by dt |S| / |V|.

Per face and per cell with plain loops (small cases only).
"""
from __future__ import annotations

import numpy as np

from . import dugks, kinetic, mapping
from .kinetic import maxwell_gh
from .mlvs import MLVSState
from .unstructured import geometry


def _gradient(c, vals, mesh, G, limiter):
    """Least-squares gradient (Nv, 2) of cell c from vals: cell id -> values on one space."""
    cen = G["cen"]
    P = vals(c)
    nv = P.shape[0]
    M = np.zeros((2, 2))
    rhs = np.zeros((nv, 2))
    nb = []
    for f, sgn in G["cell_faces"][c]:
        o = G["fR"][f] if sgn > 0 else G["fL"][f]
        if o >= 0:
            d = cen[o] - cen[c]
            Po = vals(o)
            du = Po - P
            nb.append(Po)
        else:
            d = 2.0 * (G["fb"][f] - cen[c])
            du = np.zeros(nv)
        M += np.outer(d, d)
        rhs += du[:, None] * d[None, :]
    g = np.linalg.solve(M, rhs.T).T
    if limiter == "venkat":
        umax = np.max(np.stack(nb + [P]), axis=0) - P
        umin = np.min(np.stack(nb + [P]), axis=0) - P
        eps2 = np.sqrt(G["area"][c]) ** 3 * P * P
        phi = np.ones(nv)
        for f, _ in G["cell_faces"][c]:
            d2 = g @ (G["fb"][f] - cen[c])
            d1 = np.where(d2 > 0, umax, umin)
            with np.errstate(divide="ignore", invalid="ignore"):
                v = ((d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2) / d2
            phi = np.minimum(phi, np.where(d2 == 0.0, 1.0, v))
        g = g * phi[:, None]
    return g


def step(st: MLVSState, limiter: str = "venkat"):
    """Advance every cell of st (whose mesh is an `unstructured.UMesh`) by one time step.
    Sec. 3.4 on the unstructured step."""
    mesh, gas, book, dt, opt = st.mesh, st.gas, st.book, st.dt, st.opt
    s = 0.5 * dt
    G = geometry(mesh)
    cen = G["cen"]
    nc = mesh.ncell
    state, gbp, hbp, gtp, htp = [], [], [], [], []
    for c in range(nc):
        S = book.space(st.sp[c])
        cs = dugks.cell_state(st.g[c], st.h[c], S.xi, S.w, gas, dt)
        gS, hS = dugks.model_at(cs, S.xi, S.w, gas, dt, opt.compat_cell, opt.compat_moments)
        a = dugks.bar_plus(st.g[c], gS, cs["tau"], dt)
        b = dugks.bar_plus(st.h[c], hS, cs["tau"], dt)
        state.append(cs)
        gbp.append(a)
        hbp.append(b)
        gtp.append(dugks.tilde_plus(a, st.g[c]))
        htp.append(dugks.tilde_plus(b, st.h[c]))

    cache = {}

    def on(c, key):
        if st.sp[c] == key:
            return gbp[c], hbp[c]
        if (c, key) not in cache:
            cache[(c, key)] = mapping.map_state(gbp[c], hbp[c], book.space(st.sp[c]), book.space(key), gas,
                                                opt.map_moments, opt.positive_mapping)
        return cache[(c, key)]

    def to_native(c, Fg, Fh, key, Tb):
        if st.sp[c] == key:
            return Fg, Fh
        src, dst = book.space(key), book.space(st.sp[c])
        gp, hp = mapping.project(Fg, Fh, src, dst)
        if opt.map_moments == 9:
            return mapping.correct9(gp, hp, mapping.raw9(Fg, Fh, src), dst)
        tar = kinetic.conserved(Fg, Fh, src.xi, src.w)
        return mapping.correct4(gp, hp, tar, Tb, dst, gas)

    new_g = [x.copy() for x in gtp]
    new_h = [x.copy() for x in htp]
    for f in range(len(G["fL"])):
        L, R = G["fL"][f], G["fR"][f]
        key = st.sp[L] if R < 0 else book.refine(st.sp[L], st.sp[R])
        S = book.space(key)
        xi = S.xi
        nrm, xb = G["fn"][f], G["fb"][f]
        xn = nrm[0] * xi[:, 0] + nrm[1] * xi[:, 1]
        bars = []
        for k in range(2):
            vals = lambda c: on(c, key)[k]
            gL = _gradient(L, vals, mesh, G, limiter)
            vL = vals(L) + (xb[0] - cen[L][0] - xi[:, 0] * s) * gL[:, 0] + (xb[1] - cen[L][1] - xi[:, 1] * s) * gL[:, 1]
            if R >= 0:
                gR = _gradient(R, vals, mesh, G, limiter)
                vR = (vals(R) + (xb[0] - cen[R][0] - xi[:, 0] * s) * gR[:, 0]
                      + (xb[1] - cen[R][1] - xi[:, 1] * s) * gR[:, 1])
            else:
                off = cen[L] - xb                             # from the reflected ghost centroid
                vR = vals(L) + (off[0] - xi[:, 0] * s) * gL[:, 0] + (off[1] - xi[:, 1] * s) * gL[:, 1]
            bars.append(np.where(xn > 0, vL, np.where(xn < 0, vR, 0.5 * (vL + vR))))
        if R >= 0:
            gf, hf = dugks._face_model_phi(bars[0], bars[1], xi, S.w, gas, s, opt.compat_face, opt.compat_moments)
            Tb = kinetic.moments(bars[0], bars[1], xi, S.w, gas)["T"]
        else:
            uw, vw, Tw = mesh.wall[G["fw"][f]]
            gw, hw = maxwell_gh(np.array(1.0), np.array([uw, vw]), np.array(Tw), xi, gas)
            xin = -xn
            num = -np.sum(S.w * xin * np.where(xin <= 0.0, bars[0], 0.0))
            den = np.sum(S.w * xin * np.where(xin > 0.0, gw, 0.0))
            rw = num / den
            gf = np.where(xin > 0.0, rw * gw, bars[0])
            hf = np.where(xin > 0.0, rw * hw, bars[1])
            Tb = Tw
        Fg, Fh = xn * gf, xn * hf
        lam = dt * G["fl"][f]
        g_, h_ = to_native(L, Fg, Fh, key, Tb)
        new_g[L] -= lam / G["area"][L] * g_
        new_h[L] -= lam / G["area"][L] * h_
        if R >= 0:
            g_, h_ = to_native(R, Fg, Fh, key, Tb)
            new_g[R] += lam / G["area"][R] * g_
            new_h[R] += lam / G["area"][R] * h_
    st.g, st.h = new_g, new_h
    return state
