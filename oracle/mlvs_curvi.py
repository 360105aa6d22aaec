"""Multi-level DUGKS step on a structured curvilinear mesh (oracle; test infrastructure only).

Sec. 3.4 on the curvilinear step of `curvi` (the cylinder configuration of Sec. 4 runs on an
O-grid).  Every cell carries (g~, h~) on its own representative space.  A face is evaluated
on V_f, the common refinement of its two cells' spaces; every stencil cell on another space is
represented on V_f by the hierarchical projection plus the four-moment correction with its own
moments as targets (Eq. interface_state_moment_matching), exactly as in `mlvs.step`.  On V_f
the face value follows the curvilinear step: van Leer differences along the index directions
(unit spacing) turned into the physical gradient with the cell's J^{-T}, reconstruction at the
face midpoint with the (ghost) centroid offsets, xi.n with the face normal, the face model and
recovery (Eqs. reconstruction ... recover_phi), walls and freestream sides as in `curvi`.  The
microflux (xi.n) phi is returned to each cell's space with the flux correction
(Eq. native_flux_moment_matching) and updates the cell by dt |S| / |V| (Eq. explicit_update).

The readings of `curvi` apply (node order, normals, J^{-T}, ghost centroids, dt); those of
`mlvs` apply to the level coupling.  Per face and per cell with plain loops (small cases).
"""
from __future__ import annotations

import numpy as np

from . import curvi, dugks, kinetic, mapping
from .dugks import FREE, PERIODIC, WALL
from .mlvs import MLVSState, _cell_index


def step(st: MLVSState):
    """Advance every cell of st (whose mesh is a `curvi.CurviMesh`) by one time step.
    Sec. 3.4 on the curvilinear step."""
    mesh, gas, book, dt, opt = st.mesh, st.gas, st.book, st.dt, st.opt
    s = 0.5 * dt
    nx, ny = mesh.nx, mesh.ny
    G = curvi.geometry(mesh)
    cenP = curvi._ghost_centroids(G, mesh)          # padded by two on every side
    JtP = curvi._pad_cells(G["Jt"], mesh)
    area = G["area"].ravel()
    # 1. cell-local part (Sec. 2.2 steps 1-3) on the native spaces
    state, gbp, hbp, gtp, htp = [], [], [], [], []
    for c in range(nx * ny):
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
        """phi-bar-plus of cell c on space key (Eq. interface_state_moment_matching)."""
        if st.sp[c] == key:
            return gbp[c], hbp[c]
        if (c, key) not in cache:
            cache[(c, key)] = mapping.map_state(gbp[c], hbp[c], book.space(st.sp[c]), book.space(key), gas,
                                                opt.map_moments, opt.positive_mapping)
        return cache[(c, key)]

    def recon(j, i, key, xb, xi, k):
        """phi-bar of stencil position (j, i) (a cell, a periodic image or a ghost) at the face
        midpoint xb, on space key: Eq. reconstruction with the physical slope."""
        val = lambda jj, ii: on(_cell_index(mesh, jj, ii), key)[k]
        P0 = val(j, i)
        di = dugks._limited(val(j, i + 1) - P0, P0 - val(j, i - 1), 1.0, opt.limiter)
        dj = dugks._limited(val(j + 1, i) - P0, P0 - val(j - 1, i), 1.0, opt.limiter)
        Jt = JtP[j + 2, i + 2]
        sx = Jt[0] * di + Jt[1] * dj
        sy = Jt[2] * di + Jt[3] * dj
        off = xb - cenP[j + 2, i + 2]
        return P0 + (off[0] - xi[:, 0] * s) * sx + (off[1] - xi[:, 1] * s) * sy

    def face(jL, iL, jR, iR, nrm, xb, bnd):
        """Microflux (xi.n phi^g, xi.n phi^h) on V_f of the face between stencil positions L and
        R, its normal nrm pointing from L to R; bnd = (side, inward sign) on a wall or
        freestream side."""
        cL = _cell_index(mesh, jL, iL)
        cR = _cell_index(mesh, jR, iR)
        key = book.refine(st.sp[cL], st.sp[cR])
        S = book.space(key)
        xi = S.xi
        xn = nrm[0] * xi[:, 0] + nrm[1] * xi[:, 1]
        bars = []
        for k in range(2):
            vL = recon(jL, iL, key, xb, xi, k)
            vR = recon(jR, iR, key, xb, xi, k)
            bars.append(np.where(xn > 0, vL, np.where(xn < 0, vR, 0.5 * (vL + vR))))
        if bnd is None:
            gf, hf = dugks._face_model_phi(bars[0], bars[1], xi, S.w, gas, s, opt.compat_face, opt.compat_moments)
            Tb = kinetic.moments(bars[0], bars[1], xi, S.w, gas)["T"]
        elif mesh.bc[bnd[0]] == FREE:
            side, inward = bnd
            rho_f, ux_f, uy_f, T_f = mesh.far
            vel = np.array([ux_f, uy_f])
            gw, hw = kinetic.maxwell_gh(np.array(rho_f), vel, np.array(T_f), xi, gas)
            if opt.compat_face:
                gw, hw = kinetic.compat_correct4(gw, hw, np.array(rho_f), vel, np.array(T_f), xi, S.w, gas)
            xin = inward * xn
            gf = np.where(xin > 0, gw, bars[0])
            hf = np.where(xin > 0, hw, bars[1])
            Tb = T_f
        else:
            side, inward = bnd
            uw, vw, Tw = mesh.wall[side]
            gw, hw = kinetic.maxwell_gh(np.array(1.0), np.array([uw, vw]), np.array(Tw), xi, gas)
            xin = inward * xn
            num = -np.sum(S.w * xin * np.where(xin <= 0, bars[0], 0.0))
            den = np.sum(S.w * xin * np.where(xin > 0, gw, 0.0))
            rw = num / den
            gf = np.where(xin > 0, rw * gw, bars[0])
            hf = np.where(xin > 0, rw * hw, bars[1])
            Tb = Tw
        return xn * gf, xn * hf, key, Tb

    def to_native(c, Fg, Fh, key, Tb):
        if st.sp[c] == key:
            return Fg, Fh
        src, dst = book.space(key), book.space(st.sp[c])
        gp, hp = mapping.project(Fg, Fh, src, dst)
        if opt.map_moments == 9:
            return mapping.correct9(gp, hp, mapping.raw9(Fg, Fh, src), dst)
        tar = kinetic.conserved(Fg, Fh, src.xi, src.w)
        return mapping.correct4(gp, hp, tar, Tb, dst, gas)

    def bside(side, inward):
        return (side, inward) if mesh.bc[side] in (WALL, FREE) else None

    new_g = [x.copy() for x in gtp]
    new_h = [x.copy() for x in htp]
    perx, pery = mesh.bc[0] == PERIODIC, mesh.bc[2] == PERIODIC
    # i-faces: between (j, i-1) and (j, i), normal towards (j, i)
    for j in range(ny):
        for i in range(nx if perx else nx + 1):
            bnd = None
            if not perx and i == 0:
                bnd = bside(0, +1.0)
            if not perx and i == nx:
                bnd = bside(1, -1.0)
            Fg, Fh, key, Tb = face(j, i - 1, j, i, G["ni"][j, i], G["bi"][j, i], bnd)
            L = G["li"][j, i]
            if perx or i >= 1:
                c = _cell_index(mesh, j, i - 1)
                g_, h_ = to_native(c, Fg, Fh, key, Tb)
                new_g[c] -= dt * L / area[c] * g_
                new_h[c] -= dt * L / area[c] * h_
            if perx or i <= nx - 1:
                c = _cell_index(mesh, j, i)
                g_, h_ = to_native(c, Fg, Fh, key, Tb)
                new_g[c] += dt * L / area[c] * g_
                new_h[c] += dt * L / area[c] * h_
    # j-faces: between (j-1, i) and (j, i), normal towards (j, i)
    for j in range(ny if pery else ny + 1):
        for i in range(nx):
            bnd = None
            if not pery and j == 0:
                bnd = bside(2, +1.0)
            if not pery and j == ny:
                bnd = bside(3, -1.0)
            Fg, Fh, key, Tb = face(j - 1, i, j, i, G["nj"][j, i], G["bj"][j, i], bnd)
            L = G["lj"][j, i]
            if pery or j >= 1:
                c = _cell_index(mesh, j - 1, i)
                g_, h_ = to_native(c, Fg, Fh, key, Tb)
                new_g[c] -= dt * L / area[c] * g_
                new_h[c] -= dt * L / area[c] * h_
            if pery or j <= ny - 1:
                c = _cell_index(mesh, j, i)
                g_, h_ = to_native(c, Fg, Fh, key, Tb)
                new_g[c] += dt * L / area[c] * g_
                new_h[c] += dt * L / area[c] * h_
    st.g, st.h = new_g, new_h
    return state
