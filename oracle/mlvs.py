"""Multi-level DUGKS step with cross-level coupling (oracle; test infrastructure only).

Sec. 3.4 on top of Sec. 2.2.  Every cell carries (g~, h~) on its own representative space.
For every face, the face is evaluated on V_f, the common refinement of the two adjacent
cells' spaces (for a same-level face, their space).  Every stencil cell whose space differs
from V_f is represented on V_f by the hierarchical projection plus the four-moment mapping
correction with its own moments as targets (Eq. interface_state_moment_matching; the
reading of "represented consistently" covers the tangential neighbours of the cross term).
The face value is then the ordinary DUGKS face (Eqs. reconstruction ... recover_phi) and the
microflux F = (xi.n) (g, h) (Eq. interface_reduced_fluxes).  A cell whose space differs from
V_f receives the flux projected to its space and corrected so that its mass, momentum and
energy fluxes equal those of F on V_f (Eq. native_flux_moment_matching), with the face
temperature in the delta h coupling.

This module is written per face and per cell with plain loops (small cases only).
"""
from __future__ import annotations

import numpy as np

from . import dugks, kinetic, mapping, vspace
from .dugks import FREE, PERIODIC, WALL


class SpaceBook:
    """Spaces keyed by their kappa array (uniform level L == kappa identically L).
    The representative spaces of Sec. 3.2 and the common refinement of Sec. 3.4."""

    def __init__(self, base):
        self.base = base
        self.N1 = len(vspace.axis_groups(base.n, 1))
        self._by_key = {}

    def key(self, kappa):
        k = vspace.enforce_consistency(np.asarray(kappa, dtype=np.int64), self.base.n)
        return k.tobytes(), k

    def get(self, kappa):
        key, k = self.key(kappa)
        if key not in self._by_key:
            self._by_key[key] = (k, vspace.kappa_space(self.base, k))
        return key

    def space(self, key):
        return self._by_key[key][1]

    def kappa(self, key):
        return self._by_key[key][0]

    def uniform(self, L):
        shape = (self.N1,) if self.base.D == 1 else (self.N1, self.N1)
        return self.get(np.full(shape, L, dtype=np.int64))

    def refine(self, ka, kb):
        """Common refinement: blockwise minimum of the two coarsening indices (Sec. 3.4)."""
        if ka == kb:
            return ka
        return self.get(np.minimum(self.kappa(ka), self.kappa(kb)))


class MLVSState:
    """Cells [ny][nx] (flat index j*nx+i), each with a space key and (g~, h~) on it.  Sec. 3.4."""

    def __init__(self, mesh, gas, book, space_of_cell, g, h, dt, opt):
        self.mesh, self.gas, self.book = mesh, gas, book
        self.sp = list(space_of_cell)
        self.g, self.h = list(g), list(h)
        self.dt, self.opt = dt, opt

    @classmethod
    def from_primitives(cls, mesh, gas, book, space_of_cell, rho, u, T, dt, opt):
        g, h = [], []
        for c, key in enumerate(space_of_cell):
            S = book.space(key)
            gc, hc = dugks.initial_tilde(rho.ravel()[c], u.reshape(-1, gas.D)[c], T.ravel()[c],
                                         S.xi, S.w, gas, compat=opt.compat_cell)
            g.append(gc)
            h.append(hc)
        return cls(mesh, gas, book, space_of_cell, g, h, dt, opt)

    def moments(self):
        out = []
        for c in range(len(self.g)):
            S = self.book.space(self.sp[c])
            out.append(kinetic.moments(self.g[c], self.h[c], S.xi, S.w, self.gas))
        return out

    def totals(self):
        """Sum over cells of (rho, rho u, rho v, rho E) (cell volumes equal)."""
        tot = 0.0
        for c in range(len(self.g)):
            S = self.book.space(self.sp[c])
            tot = tot + kinetic.conserved(self.g[c], self.h[c], S.xi, S.w)
        return tot


def _cell_index(mesh, j, i):
    """Source cell of a possibly out-of-range index: wrap (periodic) or clamp (ghost copy)."""
    if mesh.bc[0] == PERIODIC:
        i %= mesh.nx
    else:
        i = min(max(i, 0), mesh.nx - 1)
    if mesh.ny > 1 or mesh.bc[2] != PERIODIC:
        if mesh.bc[2] == PERIODIC:
            j %= mesh.ny
        else:
            j = min(max(j, 0), mesh.ny - 1)
    else:
        j = 0
    return j * mesh.nx + i


def step(st: MLVSState):
    """One multi-level step: Sec. 3.4 on the step of Sec. 2.2."""
    mesh, gas, book, dt, opt = st.mesh, st.gas, st.book, st.dt, st.opt
    D = gas.D
    s = 0.5 * dt
    nx, ny = mesh.nx, mesh.ny
    ncell = nx * ny
    # 1. cell-local part (Sec. 2.2 steps 1-3) on the native spaces
    state, gbp, hbp, gtp, htp = [], [], [], [], []
    for c in range(ncell):
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

    def vl(a, b, hh):
        return dugks._limited(a, b, hh, opt.limiter)

    def face(dir_, jL, iL, jR, iR, wall_side=None):
        """Flux (F^g, F^h) on V_f and V_f for the face between cells L and R (normal +x or +y).
        wall_side = (side, inward normal sign) on a boundary face: a diffuse wall, or a freestream
        side (the freestream Maxwellian, corrected like the face models, for velocities entering
        the domain; the reconstructed phi-bar for those leaving), as in the uniform step."""
        cL = _cell_index(mesh, jL, iL)
        cR = _cell_index(mesh, jR, iR)
        key = book.refine(st.sp[cL], st.sp[cR])
        S = book.space(key)
        xi = S.xi
        if dir_ == 0:
            hn, ht = mesh.dx, mesh.dy
            nrm = xi[:, 0]
            tang = xi[:, 1] if D == 2 else None
            offs = [(jL, iL - 1), (jL, iL), (jR, iR), (jR, iR + 1)]
            tL = [(jL - 1, iL), (jL + 1, iL)]
            tR = [(jR - 1, iR), (jR + 1, iR)]
        else:
            hn, ht = mesh.dy, mesh.dx
            nrm = xi[:, 1]
            tang = xi[:, 0]
            offs = [(jL - 1, iL), (jL, iL), (jR, iR), (jR + 1, iR)]
            tL = [(jL, iL - 1), (jL, iL + 1)]
            tR = [(jR, iR - 1), (jR, iR + 1)]
        vals = [on(_cell_index(mesh, j, i), key) for (j, i) in offs]
        tv = [[on(_cell_index(mesh, j, i), key) for (j, i) in tt] for tt in (tL, tR)] if D == 2 else None
        bars = []
        for k in range(2):
            P = [v[k] for v in vals]
            sn_L = vl(P[2] - P[1], P[1] - P[0], hn)
            sn_R = vl(P[3] - P[2], P[2] - P[1], hn)
            recL = P[1] + (0.5 * hn - nrm * s) * sn_L
            recR = P[2] + (-0.5 * hn - nrm * s) * sn_R
            if D == 2:
                stL = vl(tv[0][1][k] - P[1], P[1] - tv[0][0][k], ht)
                stR = vl(tv[1][1][k] - P[2], P[2] - tv[1][0][k], ht)
                recL = recL - tang * s * stL
                recR = recR - tang * s * stR
            bars.append(np.where(nrm > 0, recL, np.where(nrm < 0, recR, 0.5 * (recL + recR))))
        if wall_side is None:
            gf, hf = dugks._face_model_phi(bars[0], bars[1], xi, S.w, gas, s, opt.compat_face, opt.compat_moments)
            m = kinetic.moments(bars[0], bars[1], xi, S.w, gas)
            Tb = m["T"]
        elif mesh.bc[wall_side[0]] == FREE:
            side, inward = wall_side
            rho_f, ux_f, uy_f, T_f = mesh.far
            vel = np.array([ux_f, uy_f])[:D]
            gw, hw = kinetic.maxwell_gh(np.array(rho_f), vel, np.array(T_f), xi, gas)
            if opt.compat_face:
                gw, hw = kinetic.compat_correct4(gw, hw, np.array(rho_f), vel, np.array(T_f), xi, S.w, gas)
            xn = inward * nrm
            gf = np.where(xn > 0, gw, bars[0])
            hf = np.where(xn > 0, hw, bars[1])
            Tb = T_f
        else:
            side, inward = wall_side
            uw, vw, Tw = mesh.wall[side]
            vel = np.array([uw, vw])[:D]
            gw, hw = kinetic.maxwell_gh(np.array(1.0), vel, np.array(Tw), xi, gas)
            xn = inward * nrm
            num = -np.sum(S.w * xn * np.where(xn <= 0, bars[0], 0.0))
            den = np.sum(S.w * xn * np.where(xn > 0, gw, 0.0))
            rw = num / den
            gf = np.where(xn > 0, rw * gw, bars[0])
            hf = np.where(xn > 0, rw * hw, bars[1])
            Tb = Tw
        return nrm * gf, nrm * hf, key, Tb

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
    # x-faces
    nfx = nx if mesh.bc[0] == PERIODIC else nx + 1
    for j in range(ny):
        for i in range(nfx):
            wall = None
            if mesh.bc[0] in (WALL, FREE) and i == 0:
                wall = (0, +1.0)
            if mesh.bc[1] in (WALL, FREE) and i == nx:
                wall = (1, -1.0)
            Fg, Fh, key, Tb = face(0, j, i - 1, j, i, wall)
            per = mesh.bc[0] == PERIODIC
            if per or i >= 1:                  # the cell on the low side exists
                cL = _cell_index(mesh, j, i - 1)
                g_, h_ = to_native(cL, Fg, Fh, key, Tb)
                new_g[cL] -= dt / mesh.dx * g_
                new_h[cL] -= dt / mesh.dx * h_
            if per or i <= nx - 1:
                cR = _cell_index(mesh, j, i)
                g_, h_ = to_native(cR, Fg, Fh, key, Tb)
                new_g[cR] += dt / mesh.dx * g_
                new_h[cR] += dt / mesh.dx * h_
    if D == 2:
        nfy = ny if mesh.bc[2] == PERIODIC else ny + 1
        for j in range(nfy):
            for i in range(nx):
                wall = None
                if mesh.bc[2] in (WALL, FREE) and j == 0:
                    wall = (2, +1.0)
                if mesh.bc[3] in (WALL, FREE) and j == ny:
                    wall = (3, -1.0)
                Fg, Fh, key, Tb = face(1, j - 1, i, j, i, wall)
                per = mesh.bc[2] == PERIODIC
                if per or j >= 1:
                    cS = _cell_index(mesh, j - 1, i)
                    g_, h_ = to_native(cS, Fg, Fh, key, Tb)
                    new_g[cS] -= dt / mesh.dy * g_
                    new_h[cS] -= dt / mesh.dy * h_
                if per or j <= ny - 1:
                    cN = _cell_index(mesh, j, i)
                    g_, h_ = to_native(cN, Fg, Fh, key, Tb)
                    new_g[cN] += dt / mesh.dy * g_
                    new_h[cN] += dt / mesh.dy * h_
    st.g, st.h = new_g, new_h
    return state


def remap(st: MLVSState, c, new_key):
    """Level switch of cell c (Eq. level_switch_conservation; four-moment form, or the
    nine-moment form when st.opt.map_moments is 9, with the exponential fallback when
    st.opt.positive_mapping is set)."""
    if st.sp[c] == new_key:
        return
    src, dst = st.book.space(st.sp[c]), st.book.space(new_key)
    st.g[c], st.h[c] = mapping.map_state(st.g[c], st.h[c], src, dst, st.gas, st.opt.map_moments,
                                         st.opt.positive_mapping)
    st.sp[c] = new_key
