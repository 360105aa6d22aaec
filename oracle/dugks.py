"""One DUGKS time step on a uniform structured Cartesian mesh (oracle; test infrastructure).

Follows Sec. 2.2 in the paper's order, in FP64 numpy, arrays shaped [ny, nx, Nv] (D = 2)
or [1, nx, Nv] (D = 1):

 1. cell conservative variables from the tilde distributions (Eq. W_from_tilde,
    Eq. discrete_W) and the heat flux q = 2 tau / (2 tau + dt Pr) q~ (Eq. discrete_q);
 2. the Shakhov model distribution at the cell (Eq. g_h_eq_Pr), with the four-moment
    compatibility correction (Sec. 3.3.1) when enabled;
 3. phi-bar-plus and phi-tilde-plus at the cell.  The paper defines the four transformed
    distributions but prints no conversion; substituting phi = (2 tau phi~ + dt phi^S) /
    (2 tau + dt) (from phi~ = phi - dt/2 Omega, Omega = (phi^S - phi)/tau) into the
    definitions of phi-bar-plus and phi~+ gives
        phi-bar-plus = (2 tau - s)/(2 tau + dt) phi~ + 3 s/(2 tau + dt) phi^S,   s = dt/2
        phi~+        = 4/3 phi-bar-plus - 1/3 phi~ ;
 4. limited slopes of phi-bar-plus (Eq. reconstruction; reading: van Leer per direction);
 5. face phi-bar by the characteristic (Eq. bar_phi_transport, Eq. reconstruction);
 6. face moments, q = 2 tau/(2 tau + s Pr) q-bar (Eq. W_from_bar), face model distribution
    and face phi by Eq. recover_phi;
 7. the update phi~^{n+1} = phi~+ - dt/|V| F (Eq. explicit_update).

Readings of points the paper leaves open (the same ones the CUDA library uses):
 * dt = CFL * min(dx, dy) / max_i |xi_i|_inf.
 * Upwind side by the sign of xi.n; a velocity with xi.n = 0 takes the mean of both sides.
 * van Leer: sigma = 2ab/(a+b)/dx when a and b have the same strict sign, else 0.
 * Ghost cells outside non-periodic sides are copies of the boundary cell (slopes there
   vanish in the normal direction).
 * Diffuse isothermal wall: the face distribution for the flux is the reconstructed
   phi-bar for velocities leaving the domain and the wall Maxwellian (rho_w, u_w, T_w) for
   velocities entering it; rho_w makes the net normal mass flux zero.
 * Zero-gradient sides: the ghost copy acts as an ordinary neighbour and the face is an
   ordinary face.
 * Freestream sides: the face distribution is the reconstructed phi-bar for velocities
   leaving the domain and the freestream Maxwellian W_inf (with the four-moment
   compatibility correction when it is on at faces) for velocities entering it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .kinetic import Gas, compat_correct4, compat_correct8, moments, shakhov_gh, maxwell_gh, viscosity

PERIODIC, ZEROGRAD, WALL, FREE = "periodic", "zerograd", "wall", "freestream"


@dataclass
class Mesh:
    """Structured Cartesian mesh of Sec. 2.2 with the boundary kinds and wall / freestream states
    of the readings above."""
    nx: int
    ny: int
    dx: float
    dy: float
    # boundary kinds for the sides x-low, x-high, y-low, y-high
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    # wall data (u_w, v_w, T_w) per side
    wall: tuple = ((0.0, 0.0, 1.0),) * 4
    # freestream state (rho, u, v, T) of the freestream sides
    far: tuple = (1.0, 0.0, 0.0, 1.0)


@dataclass
class Options:
    """Switches of the step: compatibility correction (Sec. 3.3.1), inter-level mapping (Sec.
    3.3.2), limiter (Sec. 2.2)."""
    cfl: float = 0.5
    compat_cell: bool = True
    compat_face: bool = True
    limiter: str = "vanleer"      # or "none" (central slope) for smooth tests
    compat_moments: int = 4       # 4: collision invariants; 8: also heat flux and deviatoric stress (D = 2)
    map_moments: int = 4          # cross-level mapping: 4 (conserved moments) or 9 (raw second moments and
                                  # energy fluxes too, D = 2), for stencil states, fluxes and level switches
    positive_mapping: bool = False  # exponential fallback where the 4-moment state mapping makes g negative


def time_step(mesh: Mesh, xi: np.ndarray, cfl: float, D: int) -> float:
    """Global time step (reading of 'CFL = 0.5', Sec. 4)."""
    h = mesh.dx if D == 1 else min(mesh.dx, mesh.dy)
    return cfl * h / np.max(np.abs(xi))


def bar_plus(phit, phiS, tau, dt):
    """phi-bar-plus from phi~ and phi^S (derived from the definitions in Sec. 2.2, s = dt/2)."""
    s = 0.5 * dt
    return (2.0 * tau - s) / (2.0 * tau + dt) * phit + 3.0 * s / (2.0 * tau + dt) * phiS


def tilde_plus(phibp, phit):
    """phi~+ = 4/3 phi-bar-plus - 1/3 phi~ (derived from the definitions in Sec. 2.2)."""
    return 4.0 / 3.0 * phibp - 1.0 / 3.0 * phit


def recover(phib, phiS, tau, s):
    """Eq. recover_phi: phi = 2 tau/(2 tau + s) phi-bar + s/(2 tau + s) phi^S."""
    return 2.0 * tau / (2.0 * tau + s) * phib + s / (2.0 * tau + s) * phiS


def model_at(W, xi, w, gas: Gas, dt_or_s: float, compat: bool, nmom: int = 4):
    """Model distribution at points with state W = dict(rho, u, T, q) (Eq. g_h_eq_Pr + Sec. 3.3.1).
    nmom = 8: the eight-moment correction, whose heat-flux target is the Shakhov model's own
    heat flux (1 - Pr) q (Eq. g_h_eq_Pr)."""
    gS, hS = shakhov_gh(W["rho"], W["u"], W["T"], W["q"], xi, gas)
    if compat and nmom == 8:
        q_tar = (1.0 - gas.Pr) * np.asarray(W["q"])
        gS, hS = compat_correct8(gS, hS, W["rho"], W["u"], W["T"], q_tar, xi, w, gas)
    elif compat:
        gS, hS = compat_correct4(gS, hS, W["rho"], W["u"], W["T"], xi, w, gas)
    return gS, hS


def cell_state(gt, ht, xi, w, gas: Gas, dt: float):
    """Step 1: W, T, tau and q from the tilde distributions (Eqs. discrete_W, discrete_q)."""
    m = moments(gt, ht, xi, w, gas)
    tau = viscosity(m["T"], gas) / m["p"]
    q = (2.0 * tau / (2.0 * tau + dt * gas.Pr))[..., None] * m["q"]
    return {"rho": m["rho"], "u": m["u"], "T": m["T"], "p": m["p"], "tau": tau, "q": q,
            "qt": m["q"]}


def initial_tilde(rho, u, T, xi, w, gas: Gas, compat: bool = True):
    """phi~ at t = 0 for a gas at rest in local equilibrium: phi~ = phi^eq (Omega = 0).

    With compat the Maxwellian is corrected so its discrete moments equal (rho, u, T).
    Sec. 2.2 with Omega = 0 at t = 0; Sec. 3.3.1.
    """
    geq, heq = maxwell_gh(rho, u, T, xi, gas)
    if compat:
        geq, heq = compat_correct4(geq, heq, rho, u, T, xi, w, gas)
    return geq, heq


def _pad(a, mesh: Mesh, D: int):
    """Two ghost layers per side: wrap for periodic axes, edge copies otherwise."""
    xm = "wrap" if mesh.bc[0] == PERIODIC else "edge"
    a = np.pad(a, ((0, 0), (2, 2), (0, 0)), mode=xm)
    if D == 2:
        ym = "wrap" if mesh.bc[2] == PERIODIC else "edge"
        a = np.pad(a, ((2, 2), (0, 0), (0, 0)), mode=ym)
    return a


def _limited(a, b, h, limiter):
    if limiter == "none":
        return 0.5 * (a + b) / h
    same = ((a > 0) & (b > 0)) | ((a < 0) & (b < 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(same, 2.0 * a * b / (a + b), 0.0)
    return s / h


def _face_model_phi(gb, hb, xi, w, gas: Gas, s: float, compat: bool, nmom: int = 4):
    """Step 6 at a set of faces: face W, q, model distribution and Eq. recover_phi."""
    m = moments(gb, hb, xi, w, gas)
    tau = viscosity(m["T"], gas) / m["p"]
    q = (2.0 * tau / (2.0 * tau + s * gas.Pr))[..., None] * m["q"]
    W = {"rho": m["rho"], "u": m["u"], "T": m["T"], "q": q}
    gS, hS = model_at(W, xi, w, gas, s, compat, nmom)
    t = tau[..., None]
    return recover(gb, gS, t, s), recover(hb, hS, t, s)


def step(gt, ht, mesh: Mesh, xi, w, gas: Gas, dt: float, opt: Options = Options()):
    """Advance (g~, h~) by one time step.  Returns (g~^{n+1}, h~^{n+1}, cell state at t_n).
    Sec. 2.2, Eqs. phi_update ... recover_phi."""
    D = gas.D
    s = 0.5 * dt
    ny, nx, nv = gt.shape
    st = cell_state(gt, ht, xi, w, gas, dt)
    gS, hS = model_at(st, xi, w, gas, dt, opt.compat_cell, opt.compat_moments)
    tau = st["tau"][..., None]
    gbp = bar_plus(gt, gS, tau, dt)
    hbp = bar_plus(ht, hS, tau, dt)
    gtp = tilde_plus(gbp, gt)
    htp = tilde_plus(hbp, ht)

    P = [_pad(gbp, mesh, D), _pad(hbp, mesh, D)]     # padded phi-bar-plus
    oy = 2 if D == 2 else 0
    # slopes on the padded arrays (valid away from the outermost padding ring)
    sx, sy = [], []
    for a in P:
        c = a[:, 1:-1, :]
        sxa = np.zeros_like(a)
        sxa[:, 1:-1, :] = _limited(a[:, 2:, :] - c, c - a[:, :-2, :], mesh.dx, opt.limiter)
        sx.append(sxa)
        if D == 2:
            c = a[1:-1, :, :]
            sya = np.zeros_like(a)
            sya[1:-1, :, :] = _limited(a[2:, :, :] - c, c - a[:-2, :, :], mesh.dy, opt.limiter)
            sy.append(sya)

    def recon(k, jj, ii, dxb, dyb):
        """phi-bar at a face from padded cell (jj, ii): Eq. reconstruction."""
        val = P[k][jj, ii, :] + (dxb - xi[:, 0] * s) * sx[k][jj, ii, :]
        if D == 2:
            val = val + (dyb - xi[:, 1] * s) * sy[k][jj, ii, :]
        return val

    def far_phi(n):
        """The freestream distribution on n faces (corrected like the face models)."""
        rho, ux, uy, T = mesh.far
        vel = np.array([ux, uy]) if D == 2 else np.array([ux])
        r, u, t = np.full(n, rho), np.repeat(vel[None, :], n, 0), np.full(n, T)
        gf, hf = maxwell_gh(r, u, t, xi, gas)
        if opt.compat_face:
            gf, hf = compat_correct4(gf, hf, r, u, t, xi, w, gas)
        return gf, hf

    def face_phi_x():
        """phi at the x-faces i = 0..nx (non-periodic) or 0..nx-1 (periodic); shape [ny, nfx, Nv]."""
        nfx = nx if mesh.bc[0] == PERIODIC else nx + 1
        rows = np.arange(ny) + oy
        J = np.repeat(rows[:, None], nfx, axis=1)
        iL = np.arange(nfx)[None, :] - 1 + 2
        iR = np.arange(nfx)[None, :] + 2
        iL = np.repeat(iL, ny, axis=0)
        iR = np.repeat(iR, ny, axis=0)
        bars = []
        for k in range(2):
            vL = recon(k, J, iL, 0.5 * mesh.dx, 0.0)
            vR = recon(k, J, iR, -0.5 * mesh.dx, 0.0)
            pos = xi[:, 0] > 0
            neg = xi[:, 0] < 0
            bar = np.where(pos, vL, np.where(neg, vR, 0.5 * (vL + vR)))
            bars.append(bar)
        phig, phih = _face_model_phi(bars[0], bars[1], xi, w, gas, s, opt.compat_face, opt.compat_moments)
        out = [phig, phih]
        # freestream and walls on the x sides
        for side, idx, inward in ((0, 0, +1.0), (1, nfx - 1, -1.0)):
            if mesh.bc[side] == FREE:
                gf, hf = far_phi(ny)
                in_m = inward * xi[:, 0] > 0.0
                out[0][:, idx, :] = np.where(in_m, gf, bars[0][:, idx, :])
                out[1][:, idx, :] = np.where(in_m, hf, bars[1][:, idx, :])
                continue
            if mesh.bc[side] != WALL:
                continue
            uw, vw, Tw = mesh.wall[side]
            vel = np.array([uw, vw]) if D == 2 else np.array([uw])
            gw, hw = maxwell_gh(np.ones(ny), np.repeat(vel[None, :], ny, 0), np.full(ny, Tw), xi, gas)
            xn = inward * xi[:, 0]                         # xi . n_in
            out_m = xn <= 0.0                              # leaving the domain (towards the wall)
            in_m = xn > 0.0
            gbar = bars[0][:, idx, :]
            num = -np.sum(w * xn * np.where(out_m, gbar, 0.0), axis=-1)
            den = np.sum(w * xn * np.where(in_m, gw, 0.0), axis=-1)
            rw = (num / den)[:, None]
            out[0][:, idx, :] = np.where(in_m, rw * gw, gbar)
            out[1][:, idx, :] = np.where(in_m, rw * hw, bars[1][:, idx, :])
        return out

    def face_phi_y():
        nfy = ny if mesh.bc[2] == PERIODIC else ny + 1
        cols = np.arange(nx) + 2
        I = np.repeat(cols[None, :], nfy, axis=0)
        jS = np.repeat((np.arange(nfy) - 1 + 2)[:, None], nx, axis=1)
        jN = np.repeat((np.arange(nfy) + 2)[:, None], nx, axis=1)
        bars = []
        for k in range(2):
            vS = recon(k, jS, I, 0.0, 0.5 * mesh.dy)
            vN = recon(k, jN, I, 0.0, -0.5 * mesh.dy)
            pos = xi[:, 1] > 0
            neg = xi[:, 1] < 0
            bars.append(np.where(pos, vS, np.where(neg, vN, 0.5 * (vS + vN))))
        phig, phih = _face_model_phi(bars[0], bars[1], xi, w, gas, s, opt.compat_face, opt.compat_moments)
        out = [phig, phih]
        for side, idx, inward in ((2, 0, +1.0), (3, nfy - 1, -1.0)):
            if mesh.bc[side] == FREE:
                gf, hf = far_phi(nx)
                in_m = inward * xi[:, 1] > 0.0
                out[0][idx, :, :] = np.where(in_m, gf, bars[0][idx, :, :])
                out[1][idx, :, :] = np.where(in_m, hf, bars[1][idx, :, :])
                continue
            if mesh.bc[side] != WALL:
                continue
            uw, vw, Tw = mesh.wall[side]
            vel = np.array([uw, vw])
            gw, hw = maxwell_gh(np.ones(nx), np.repeat(vel[None, :], nx, 0), np.full(nx, Tw), xi, gas)
            yn = inward * xi[:, 1]
            out_m = yn <= 0.0
            in_m = yn > 0.0
            gbar = bars[0][idx, :, :]
            num = -np.sum(w * yn * np.where(out_m, gbar, 0.0), axis=-1)
            den = np.sum(w * yn * np.where(in_m, gw, 0.0), axis=-1)
            rw = (num / den)[:, None]
            out[0][idx, :, :] = np.where(in_m, rw * gw, gbar)
            out[1][idx, :, :] = np.where(in_m, rw * hw, bars[1][idx, :, :])
        return out

    fx = face_phi_x()
    new = []
    for k, (tp) in enumerate((gtp, htp)):
        F = fx[k]
        if mesh.bc[0] == PERIODIC:
            Fw, Fe = F, np.roll(F, -1, axis=1)
        else:
            Fw, Fe = F[:, :-1, :], F[:, 1:, :]
        div = xi[:, 0] * (Fe - Fw) / mesh.dx
        new.append(tp - dt * div)
    if D == 2:
        fy = face_phi_y()
        for k in range(2):
            F = fy[k]
            if mesh.bc[2] == PERIODIC:
                Fs, Fn = F, np.roll(F, -1, axis=0)
            else:
                Fs, Fn = F[:-1, :, :], F[1:, :, :]
            new[k] = new[k] - dt * xi[:, 1] * (Fn - Fs) / mesh.dy
    return new[0], new[1], st


def run(gt, ht, mesh: Mesh, xi, w, gas: Gas, dt: float, nsteps: int, opt: Options = Options()):
    """N steps of `step` (Sec. 2.2)."""
    for _ in range(nsteps):
        gt, ht, _ = step(gt, ht, mesh, xi, w, gas, dt, opt)
    return gt, ht
