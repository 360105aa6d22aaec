"""Moment-consistent mapping between velocity spaces (oracle; test infrastructure only).

Sec. 3.3.2:
 * hierarchical projection P_{s->t} (Eq. hierarchical_projection_operator): coarsening by
   weighted aggregation of g (Eq. mapping_g_projection) and of H = h + |xi|^2 g
   (Eq. mapping_energy_projection), h recovered with the target coordinate
   (Eq. mapping_h_projection); refinement by inheritance of g and H;
 * forced-conservation correction (Eq. forced_conservation_mapping), kept as a comparator;
 * four-moment linear correction: chi = 1, raw basis [1, xi_x, xi_y, xi^2]
   (Eq. raw_four_g_basis), delta h = (3 - D + K) R T_tar delta g (Eq. raw_four_gh_coupling),
   targets (rho, rho u, rho v, rho E) (Eq. mapping_four_targets);
 * nine-moment block-triangular correction: g-block with basis Eq. raw_six_g_basis and
   targets (rho, rho u, rho v, G_xx, G_yy, G_xy) (Eq. source_second_raw_moments), then the
   h-block with basis Eq. raw_three_h_basis solving Eq. mapping_h_residual_correction for
   (rho E, J_x, J_y) (Eq. source_energy_flux_moments);
 * the exponential correction proposed as a positivity-preserving fallback
   (Eq. exponential_moment_correction), four constraints, by Newton iteration.

Both spaces are partitions of the same base grid (vspace.Space), so every target cell either
lies inside one source cell (refinement) or is a union of source cells (coarsening).
Distributions have shape (..., Nv).
"""
from __future__ import annotations

import numpy as np

from .kinetic import Gas, maxwell_gh, moments


def projection_matrix(src, dst) -> np.ndarray:
    """Dense (Nt x Ns) matrix of P_{s->t}: rows average (coarsen) or pick (refine).
    Eq. hierarchical_projection_operator."""
    P = np.zeros((dst.nv, src.nv))
    for i in range(dst.nv):
        r = dst.rect[i]
        if src.base.D == 1:
            cover = src.owner[r[0]:r[1]]
        else:
            cover = src.owner[r[2]:r[3], r[0]:r[1]]
        owners = np.unique(cover)
        if len(owners) == 1:
            o = owners[0]
            P[i, o] = 1.0                       # refinement: inherit from the parent
        else:
            # coarsening: the target cell must be exactly the union of its source cells
            area = np.sum(src.w[owners])
            if abs(area - dst.w[i]) > 1e-12 * dst.w[i]:
                raise ValueError("spaces are not nested")
            P[i, owners] = src.w[owners] / area
    return P


def project(g, h, src, dst):
    """Hierarchical projection of (g, h) from src to dst (Sec. 3.3.2, projection equations)."""
    P = projection_matrix(src, dst)
    xs2 = np.sum(src.xi ** 2, axis=-1)
    xt2 = np.sum(dst.xi ** 2, axis=-1)
    gt = g @ P.T
    Ht = (h + xs2 * g) @ P.T
    return gt, Ht - xt2 * gt


def _conserved_targets(rho, u, T, gas: Gas):
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    rhoE = rho * (0.5 * np.sum(u * u, axis=-1) + gas.cv * T)
    return np.concatenate([rho[..., None], rho[..., None] * u, rhoE[..., None]], axis=-1)


def correct4(gp, hp, M_tar, T_tar, space, gas: Gas):
    """Four-moment mapping correction (Eqs. raw_four_g_basis, raw_four_gh_coupling).

    M_tar (..., D+2) = (rho, rho u, rho E) targets, T_tar the temperature of the coupling.
    """
    xi, w = space.xi, space.w
    D = gas.D
    xi2 = np.sum(xi * xi, axis=-1)
    nm = D + 2
    phi = np.empty((nm, len(w)))
    phi[0] = 1.0
    phi[1:1 + D] = xi.T
    phi[D + 1] = xi2
    T_tar = np.asarray(T_tar, dtype=np.float64)
    cK = gas.c_extra * gas.R * T_tar                  # delta h = cK delta g
    # rows psi_k: 1, xi, 1/2 (xi^2 + cK)  (energy row includes delta h)
    base = np.einsum("kv,mv->km", phi[:D + 1] * w, phi)          # rows 0..D
    e_a = 0.5 * np.einsum("v,mv->m", w * xi2, phi)                # 1/2 sum w xi^2 phi_m
    e_b = 0.5 * np.einsum("v,mv->m", w, phi)                      # 1/2 sum w phi_m
    A = np.zeros(T_tar.shape + (nm, nm))
    A[..., :D + 1, :] = base
    A[..., D + 1, :] = e_a + cK[..., None] * e_b
    cur = np.concatenate([
        np.sum(w * gp, axis=-1)[..., None],
        np.einsum("...v,vd->...d", w * gp, xi),
        (0.5 * np.sum(w * (xi2 * gp + hp), axis=-1))[..., None]], axis=-1)
    dM = M_tar - cur
    a = np.linalg.solve(A, dM[..., None])[..., 0]
    dg = np.einsum("...m,mv->...v", a, phi)
    return gp + dg, hp + cK[..., None] * dg


def map4(g, h, src, dst, gas: Gas, M_tar=None, T_tar=None):
    """Projection + four-moment correction with the source moments as targets (Eq. level_switch_conservation)."""
    gp, hp = project(g, h, src, dst)
    if M_tar is None:
        m = moments(g, h, src.xi, src.w, gas)
        M_tar = _conserved_targets(m["rho"], m["u"], m["T"], gas)
        T_tar = m["T"]
    return correct4(gp, hp, M_tar, T_tar, dst, gas)


def map_state(g, h, src, dst, gas: Gas, nmom=4, positive=False):
    """A cell state carried to another space with its own moments as targets: the projection
    plus the four-moment correction (Eqs. interface_state_moment_matching and
    level_switch_conservation), or the nine-moment correction (nmom = 9).  With `positive`, a
    four-moment result with a negative g where the projection had none is replaced by the
    exponential correction of the same targets (the fallback Sec. 3.3.2 proposes)."""
    if nmom == 9:
        return map9(g, h, src, dst)
    m = moments(g, h, src.xi, src.w, gas)
    tar = np.concatenate([[m["rho"]], m["rho"] * m["u"], [m["rhoE"]]])
    gp, hp = project(g, h, src, dst)
    gl, hl = correct4(gp, hp, tar, m["T"], dst, gas)
    if positive and gl.min() < 0.0 <= gp.min():
        return correct_exp4(gp, hp, tar, dst)
    return gl, hl


def correct_exp4(gp, hp, M_tar, space, tol=1e-14, maxit=60):
    """Exponential moment-constrained correction (Eq. exponential_moment_correction), the
    positivity-preserving alternative to the additive correction that Sec. 3.3.2 proposes:
    phi* = phi^p exp(a . psi) with one factor for g and h, psi = [1, xi_x, xi_y, xi^2 / 2]
    (2-D), and a solving the four constraints (rho, rho u, rho v, rho E) of Eq.
    mapping_four_targets.  Damped Newton iteration from a = 0 (halving the step until the
    residual norm decreases).  gp, hp of shape (Nv,); raises if it does not converge.
    """
    xi = space.xi
    w = space.w
    x, y = xi[:, 0], xi[:, 1]
    xi2 = x * x + y * y
    basis = np.stack([np.ones_like(x), x, y, 0.5 * xi2])                 # 4 x Nv
    kern = np.stack([gp, x * gp, y * gp, 0.5 * (xi2 * gp + hp)])         # 4 x Nv, before the factor
    M_tar = np.asarray(M_tar, dtype=np.float64)
    scale = np.maximum(np.abs(M_tar), np.max(np.abs(M_tar)) * 1e-3)

    def residual(a):
        e = np.exp(a @ basis)
        return (kern * e) @ w - M_tar, e

    a = np.zeros(4)
    r, e = residual(a)
    for _ in range(maxit):
        if np.max(np.abs(r) / scale) < tol:
            return gp * e, hp * e
        J = (kern * e * w) @ basis.T
        da = np.linalg.solve(J, -r)
        t = 1.0
        while True:
            r1, e1 = residual(a + t * da)
            if np.linalg.norm(r1 / scale) < np.linalg.norm(r / scale) or t < 1e-8:
                break
            t *= 0.5
        a, r, e = a + t * da, r1, e1
    if np.max(np.abs(r) / scale) < tol:
        return gp * e, hp * e
    raise RuntimeError("exponential correction did not converge")


def forced_conservation(gp, hp, g_src, h_src, src, dst, gas: Gas):
    """Phi^FC = Phi^p + Phi^eq(W^s) - Phi^eq(W^p) (Eq. forced_conservation_mapping)."""
    ms = moments(g_src, h_src, src.xi, src.w, gas)
    mp = moments(gp, hp, dst.xi, dst.w, gas)
    gs_eq, hs_eq = maxwell_gh(ms["rho"], ms["u"], ms["T"], dst.xi, gas)
    gp_eq, hp_eq = maxwell_gh(mp["rho"], mp["u"], mp["T"], dst.xi, gas)
    return gp + gs_eq - gp_eq, hp + hs_eq - hp_eq


def raw9(g, h, space):
    """The nine raw target moments (rho, rho u, rho v, rho E, Gxx, Gyy, Gxy, Jx, Jy) (2-D).
    Eqs. source_second_raw_moments, source_energy_flux_moments."""
    xi, w = space.xi, space.w
    x, y = xi[:, 0], xi[:, 1]
    xi2 = x * x + y * y
    e = h + xi2 * g
    return np.stack([np.sum(w * g, -1), np.sum(w * x * g, -1), np.sum(w * y * g, -1),
                     0.5 * np.sum(w * e, -1), np.sum(w * x * x * g, -1), np.sum(w * y * y * g, -1),
                     np.sum(w * x * y * g, -1), 0.5 * np.sum(w * x * e, -1), 0.5 * np.sum(w * y * e, -1)],
                    axis=-1)


def correct9(gp, hp, M_tar, space):
    """Nine-moment block-triangular correction (Sec. 3.3.2, Eqs. raw_six_g_basis ... mapping_h_residual_correction).

    M_tar (..., 9) ordered as raw9.  2-D only.
    """
    xi, w = space.xi, space.w
    x, y = xi[:, 0], xi[:, 1]
    xi2 = x * x + y * y
    phig = np.stack([np.ones_like(x), x, y, x * x, y * y, x * y])       # 6 x Nv
    psig = phig                                                          # rho, rho u, rho v, Gxx, Gyy, Gxy
    Ag = np.einsum("kv,mv->km", psig * w, phig)
    cur = raw9(gp, hp, space)
    dg_t = M_tar[..., [0, 1, 2, 4, 5, 6]] - cur[..., [0, 1, 2, 4, 5, 6]]
    a = np.linalg.solve(Ag, dg_t[..., None])[..., 0]
    dg = np.einsum("...m,mv->...v", a, phig)
    phih = np.stack([np.ones_like(x), x, y])                             # 3 x Nv
    Ah = 0.5 * np.einsum("kv,mv->km", phih * w, phih)
    # remaining defects in (rho E, Jx, Jy) after the g-block
    rhs = (M_tar[..., [3, 7, 8]] - cur[..., [3, 7, 8]]) - 0.5 * np.einsum(
        "kv,...v->...k", np.stack([xi2, x * xi2, y * xi2]) * w, dg)
    b = np.linalg.solve(Ah, rhs[..., None])[..., 0]
    dh = np.einsum("...m,mv->...v", b, phih)
    return gp + dg, hp + dh


def map9(g, h, src, dst):
    """Projection plus the nine-moment correction with the source's raw moments as targets (Sec.
    3.3.2)."""
    gp, hp = project(g, h, src, dst)
    return correct9(gp, hp, raw9(g, h, src), dst)
