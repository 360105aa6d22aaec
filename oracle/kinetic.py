"""Reduced BGK/Shakhov model, discrete moments and the compatibility correction (oracle).

Test infrastructure only.  FP64 numpy; sums over velocity run in ascending index order
(numpy reductions over the last axis).

Conventions: distributions have shape (..., Nv); rho (...,), u (..., D), T (...,), q (..., D);
xi (Nv, D), w (Nv,).
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np


@dataclass
class Gas:
    """Gas model of Sec. 2.1 and the viscosity law of Sec. 4 (power law)."""
    D: int = 2           # velocity dimension
    K: float = 0.0       # internal degrees of freedom (monatomic: 0)
    R: float = 1.0
    Pr: float = 2.0 / 3.0
    omega: float = 0.81
    mu_ref: float = 1e-3
    T_ref: float = 1.0

    @property
    def c_extra(self):
        """3 - D + K: the degrees of freedom folded into h (Eq. g_h_eq_Pr, h^eq line)."""
        return 3.0 - self.D + self.K

    @property
    def cv(self):
        """c_V = (3+K) R / 2 (text under Eq. moments)."""
        return 0.5 * (3.0 + self.K) * self.R


def mu_ref_from_kn(Kn: float, omega: float = 0.81, alpha: float = 1.0, rho_ref: float = 1.0,
                   R: float = 1.0, T_ref: float = 1.0, L_ref: float = 1.0) -> float:
    """Reference viscosity from a Knudsen number.

    The paper gives only the temperature law mu = mu_ref (T/T_ref)^omega (Sec. 4).  Reading:
    the standard VHS/VSS mean-free-path relation,
        mu_ref = 5 (alpha+1)(alpha+2) sqrt(pi) / (4 alpha (5-2 omega)(7-2 omega))
                 * Kn * rho_ref * sqrt(2 R T_ref) * L_ref .
    """
    c = 5.0 * (alpha + 1.0) * (alpha + 2.0) * math.sqrt(math.pi) / (
        4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega))
    return c * Kn * rho_ref * math.sqrt(2.0 * R * T_ref) * L_ref


def viscosity(T, gas: Gas):
    """mu = mu_ref (T/T_ref)^omega (Sec. 4, power-law relation)."""
    return gas.mu_ref * (np.asarray(T) / gas.T_ref) ** gas.omega


def maxwell_gh(rho, u, T, xi, gas: Gas):
    """Reduced Maxwellians g^eq, h^eq (Eq. g_h_eq_Pr, first two lines)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    RT = gas.R * T
    c = xi - u[..., None, :]                      # (..., Nv, D)
    c2 = np.sum(c * c, axis=-1)
    geq = (rho / (2.0 * np.pi * RT) ** (gas.D / 2.0))[..., None] * np.exp(-c2 / (2.0 * RT[..., None]))
    heq = gas.c_extra * RT[..., None] * geq
    return geq, heq


def shakhov_gh(rho, u, T, q, xi, gas: Gas):
    """Reduced Shakhov distributions g^S = g^eq + g^Pr, h^S = h^eq + h^Pr (Eq. g_h_eq_Pr).

    With Pr = 1 (BGK) the Pr terms vanish.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    geq, heq = maxwell_gh(rho, u, T, xi, gas)
    if gas.Pr == 1.0:
        return geq, heq
    RT = (gas.R * T)[..., None]
    p = (rho * gas.R * T)[..., None]
    c = xi - u[..., None, :]
    c2 = np.sum(c * c, axis=-1)
    cq = np.sum(c * q[..., None, :], axis=-1)
    fac = (1.0 - gas.Pr) * cq / (5.0 * p * RT)
    D, K = gas.D, gas.K
    gpr = fac * (c2 / RT - D - 2.0) * geq
    hpr = fac * ((c2 / RT - D) * (K + 3.0 - D) - 2.0 * K) * RT * geq
    return geq + gpr, heq + hpr


def moments(g, h, xi, w, gas: Gas):
    """Conservative variables, temperature, heat flux and stress of (g, h).

    Eq. discrete_W / Eq. reduced_moments:  rho = sum w g,  rho u = sum w xi g,
    rho E = 1/2 sum w (xi^2 g + h),  q = 1/2 sum w c (c^2 g + h),  c = xi - u.
    T from rho E = 1/2 rho u^2 + rho c_V T (text under Eq. moments).
    Stress P_ab = sum w c_a c_b g (central second moment of g).
    """
    rho = np.sum(w * g, axis=-1)
    mom = np.einsum("...v,vd->...d", w * g, xi)
    u = mom / rho[..., None]
    xi2 = np.sum(xi * xi, axis=-1)
    rhoE = 0.5 * np.sum(w * (xi2 * g + h), axis=-1)
    T = (rhoE / rho - 0.5 * np.sum(u * u, axis=-1)) / gas.cv
    c = xi - u[..., None, :]
    c2 = np.sum(c * c, axis=-1)
    q = 0.5 * np.einsum("...v,...vd->...d", w * (c2 * g + h), c)
    P = np.einsum("...v,...va,...vb->...ab", w * g, c, c)
    return {"rho": rho, "mom": mom, "u": u, "rhoE": rhoE, "T": T, "p": rho * gas.R * T,
            "q": q, "P": P}


def compat_correct8(gS, hS, rho, u, T, q_tar, xi, w, gas: Gas):
    """Eight-moment linear compatibility correction of the model distribution (Sec. 3.3.1,
    D = 2 only).

    Eq. gh_model_correction with chi^g = g^S, chi^h = h^S, basis Eq. eq_eight_basis
    phi = [1, xi_x, xi_y, E_xi, E_c c_x, E_c c_y, c_x^2 - c_y^2, c_x c_y] with c = xi - u and
    E_c = 1/2 [(3-D+K) R T + c^2] (Eq. E_c_definition), joint matrix
    Eq. joint_gh_correction_matrix with the kernels of Eq. eq_eight_moment_constraint, and
    targets (rho, rho u, rho v, rho E, q_x^tar, q_y^tar, 0, 0): the collision invariants, the
    heat flux the model prescribes and a vanishing deviatoric stress.  One 8 x 8 system.
    """
    if gas.D != 2:
        raise ValueError("the eight-moment correction is two-dimensional")
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    q_tar = np.asarray(q_tar, dtype=np.float64)
    RT = gas.R * T
    xi2 = np.sum(xi * xi, axis=-1)
    cx = xi[:, 0] - u[..., 0:1]                 # (..., Nv)
    cy = xi[:, 1] - u[..., 1:2]
    c2 = cx * cx + cy * cy
    Exi = 0.5 * (gas.c_extra * RT[..., None] + xi2)
    Ec = 0.5 * (gas.c_extra * RT[..., None] + c2)
    shp = gS.shape
    phi = np.empty(shp[:-1] + (8, shp[-1]))
    phi[..., 0, :] = 1.0
    phi[..., 1, :] = xi[:, 0]
    phi[..., 2, :] = xi[:, 1]
    phi[..., 3, :] = Exi
    phi[..., 4, :] = Ec * cx
    phi[..., 5, :] = Ec * cy
    phi[..., 6, :] = cx * cx - cy * cy
    phi[..., 7, :] = cx * cy
    # kernels psi^g chi^g + psi^h chi^h of the eight constrained moments
    kern = np.empty_like(phi)
    kern[..., 0, :] = gS
    kern[..., 1, :] = xi[:, 0] * gS
    kern[..., 2, :] = xi[:, 1] * gS
    kern[..., 3, :] = 0.5 * (xi2 * gS + hS)
    kern[..., 4, :] = 0.5 * (c2 * gS + hS) * cx
    kern[..., 5, :] = 0.5 * (c2 * gS + hS) * cy
    kern[..., 6, :] = (cx * cx - cy * cy) * gS
    kern[..., 7, :] = cx * cy * gS
    A = np.einsum("...kv,...mv->...km", kern * w, phi)
    rhoE = rho * (0.5 * np.sum(u * u, axis=-1) + gas.cv * T)
    zero = np.zeros_like(rho)[..., None]
    tar = np.concatenate([rho[..., None], rho[..., None] * u, rhoE[..., None], q_tar, zero, zero], axis=-1)
    cur = np.sum(kern * w, axis=-1)
    a = np.linalg.solve(A, (tar - cur)[..., None])[..., 0]
    corr = np.einsum("...m,...mv->...v", a, phi)
    return gS + gS * corr, hS + hS * corr


def conserved(g, h, xi, w):
    """The collision-invariant moments (rho, rho u, rho E) stacked on the last axis.
    Eq. discrete_W."""
    rho = np.sum(w * g, axis=-1)
    mom = np.einsum("...v,vd->...d", w * g, xi)
    xi2 = np.sum(xi * xi, axis=-1)
    rhoE = 0.5 * np.sum(w * (xi2 * g + h), axis=-1)
    return np.concatenate([rho[..., None], mom, rhoE[..., None]], axis=-1)


def compat_correct4(gS, hS, rho, u, T, xi, w, gas: Gas):
    """Four-moment linear compatibility correction of the model distribution (Sec. 3.3.1).

    Eq. gh_model_correction with chi^g = g^S, chi^h = h^S (the equation after it), basis
    Eq. eq_four_basis phi = [1, xi_x, xi_y, E_xi] with E_xi = 1/2 [(3-D+K) R T + xi^2]
    (Eq. E_xi_definition), joint matrix Eq. joint_gh_correction_matrix with
    psi^g = [1, xi_x, xi_y, xi^2/2] and psi^h = [0, 0, 0, 1/2], and targets
    Eq. eq_four_moment_constraint (rho, rho u, rho v, rho E).  In 1-D the basis is
    [1, xi, E_xi].  The small system is solved by LU with partial pivoting.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    D = gas.D
    nm = D + 2
    RT = gas.R * T
    xi2 = np.sum(xi * xi, axis=-1)
    # basis phi_m(xi) (..., nm, Nv)
    Exi = 0.5 * (gas.c_extra * RT[..., None] + xi2)
    shp = gS.shape
    phi = np.empty(shp[:-1] + (nm, shp[-1]))
    phi[..., 0, :] = 1.0
    for d in range(D):
        phi[..., 1 + d, :] = xi[:, d]
    phi[..., D + 1, :] = Exi
    # kernels: rows k of psi^g * chi^g + psi^h * chi^h
    kern = np.empty_like(phi)
    kern[..., 0, :] = gS
    for d in range(D):
        kern[..., 1 + d, :] = xi[:, d] * gS
    kern[..., D + 1, :] = 0.5 * (xi2 * gS + hS)
    A = np.einsum("...kv,...mv->...km", kern * w, phi)
    rhoE = rho * (0.5 * np.sum(u * u, axis=-1) + gas.cv * T)
    tar = np.concatenate([rho[..., None], (rho[..., None] * u), rhoE[..., None]], axis=-1)
    cur = np.sum(kern * w, axis=-1)
    dM = tar - cur
    a = np.linalg.solve(A, dM[..., None])[..., 0]
    corr = np.einsum("...m,...mv->...v", a, phi)
    return gS + gS * corr, hS + hS * corr
