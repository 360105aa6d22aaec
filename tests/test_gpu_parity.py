"""GPU-vs-oracle parity of the single-space DUGKS step, through the C ABI.

Tolerances:
 * FP64 storage: the library and the oracle run the same FP64 algorithm with different
   summation orders; relative differences of a few 1e-13 per step (1e-10 here).
 * FP32 storage: per-velocity arithmetic and storage round at 6e-8; after a few steps the
   moments agree to 1e-5 relative (rho, T), 1e-5 sqrt(RT) for velocity, and the heat flux to
   1e-3 of its field maximum.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_moments, oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_35258_b300.solver import Solver  # noqa: E402
from paper_2609_35258_b300.mlvs import (RHO as M_RHO, U as M_U, V as M_V, T as M_T,  # noqa: E402
                                        QX as M_QX, QY as M_QY, SXX as M_SXX, SXY as M_SXY,
                                        SYY as M_SYY)


def _compare(gm, om, rtol_rho, atol_u, rtol_T, qfrac, D=2):
    rho_o, T_o = om[0], om[3]
    assert np.max(np.abs(gm[0] - rho_o) / rho_o) < rtol_rho
    assert np.max(np.abs(gm[1] - om[1])) < atol_u
    if D == 2:
        assert np.max(np.abs(gm[2] - om[2])) < atol_u
    assert np.max(np.abs(gm[3] - T_o) / T_o) < rtol_T
    qs = max(np.max(np.abs(om[4])), np.max(np.abs(om[5])), 1e-30)
    assert np.max(np.abs(gm[4] - om[4])) < qfrac * qs
    if D == 2:
        assert np.max(np.abs(gm[5] - om[5])) < qfrac * qs


@pytest.mark.parametrize("nx,ny", [(40, 20), (3, 2)])
def test_periodic_f64(nx, ny):
    desc = workloads.periodic_random(nx, ny, n_base=25, storage="f64")
    o = oracle_setup(desc)
    s = Solver(desc)
    assert abs(s.dt - o["dt"]) < 1e-15
    s.step(5)
    g, h = oracle_run(o, 5)
    _compare(s.moments(), oracle_moments(o, g, h), 1e-10, 1e-10, 1e-10, 1e-8)
    gg, hh = s.read_cells(0, nx * ny, 25 * 25)
    np.testing.assert_allclose(gg, g.reshape(nx * ny, -1), rtol=1e-9, atol=1e-12 * g.max())
    np.testing.assert_allclose(hh, h.reshape(nx * ny, -1), rtol=1e-9, atol=1e-12 * h.max())


def test_periodic_f32():
    desc = workloads.periodic_random(40, 20, n_base=25, storage="f32")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(5)
    g, h = oracle_run(o, 5)
    _compare(s.moments(), oracle_moments(o, g, h), 1e-5, 1e-5, 1e-5, 1e-3)
    gg, _ = s.read_cells(0, 40 * 20, 625)
    np.testing.assert_allclose(gg, g.reshape(800, -1), rtol=0, atol=2e-5 * g.max())


def test_cavity_f32_ragged():
    desc = workloads.cavity(36, n_base=25, Kn=0.075)
    desc["init"] = desc["init"][:, :36]
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(10)
    g, h = oracle_run(o, 10)
    _compare(s.moments(), oracle_moments(o, g, h), 1e-5, 1e-5, 1e-5, 1e-3)


def test_cavity_f64_walls():
    desc = workloads.cavity(20, n_base=25, Kn=0.075, storage="f64")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(8)
    g, h = oracle_run(o, 8)
    _compare(s.moments(), oracle_moments(o, g, h), 1e-10, 1e-10, 1e-10, 1e-7)


def test_sod_1d_f64_full_config():
    desc = workloads.sod_1d()           # 200 cells, 101 velocities, Kn = 1e-3, FP64, BGK
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(20)
    g, h = oracle_run(o, 20)
    gm = s.moments()
    om = oracle_moments(o, g, h)
    assert np.max(np.abs(gm[0] - om[0]) / om[0]) < 1e-10
    assert np.max(np.abs(gm[1] - om[1])) < 1e-10
    assert np.max(np.abs(gm[3] - om[3]) / om[3]) < 1e-10


def test_options_bgk_no_limiter_no_compat():
    desc = workloads.periodic_random(17, 9, n_base=25, storage="f64", Pr=1.0)
    desc["limiter"] = "none"
    o = oracle_setup(desc, compat=False)
    s = Solver(desc, compat_cell=0, compat_face=0)
    s.step(4)
    g, h = oracle_run(o, 4)
    _compare(s.moments(), oracle_moments(o, g, h), 1e-10, 1e-10, 1e-10, 1e-7)


def test_conservation_f64_periodic():
    desc = workloads.periodic_random(33, 17, n_base=25, storage="f64")
    s = Solver(desc)
    m0 = s.moments()
    s.step(50)
    m1 = s.moments()
    tot0 = np.array([m0[0].sum(), (m0[0] * m0[1]).sum(), (m0[0] * m0[2]).sum(), m0[6].sum()])
    tot1 = np.array([m1[0].sum(), (m1[0] * m1[1]).sum(), (m1[0] * m1[2]).sum(), m1[6].sum()])
    assert np.max(np.abs(tot1 - tot0)) < 1e-12 * np.max(np.abs(tot0))


# FP32 storage rounds phi~^{n+1} = phi~ + increment stochastically (the rounding error from
# Fast2Sum, the neighbour towards the exact sum taken with probability error/gap), so every
# stored value is unbiased with an error of at most one ulp, 2^-23 relative, standard deviation
# about 2^-24/sqrt(3) = 3.4e-8.  A domain total sum_cells sum_v w phi then moves by about
# 3.4e-8 / sqrt(N_eff) per step, N_eff the effective number of independent values (cells x
# velocities weighted by w phi: ~1e5 here), i.e. ~1e-10 per step, and as a random walk by
# ~1e-10 sqrt(steps) over a run.  The bound is 1e-10 per step times the steps, a margin of
# sqrt(steps) over the expected walk; the transport and collision terms telescope or conserve
# exactly, so anything systematic (weights that do not sum to one, rounded wall densities,
# correction sums that disagree with the evaluated model, increments lost to round-to-nearest
# near a steady state) grows linearly and exceeds it.
FP32_DRIFT_PER_STEP = 1e-10


def test_conservation_f32_periodic():
    desc = workloads.periodic_random(33, 17, n_base=25, storage="f32")
    s = Solver(desc)
    m0 = s.moments()
    s.step(50)
    m1 = s.moments()
    tot0 = np.array([m0[0].sum(), m0[6].sum()])
    tot1 = np.array([m1[0].sum(), m1[6].sum()])
    assert np.max(np.abs(tot1 - tot0) / tot0) < 50 * FP32_DRIFT_PER_STEP


def test_wall_mass_conservation_f64():
    """Diffuse walls carry no net mass flux: exact up to FP64 rounding."""
    desc = workloads.cavity(32, n_base=25, Kn=0.075, storage="f64")
    s = Solver(desc)
    m0 = s.moments()[0].sum()
    s.step(100)
    m1 = s.moments()[0].sum()
    assert abs(m1 - m0) / m0 < 1e-13


# Near a steady state round-to-nearest would lose the same sub-ulp increments every step (a
# drift growing linearly, measured 4e-8 to 1.1e-7 over 100 steps for 1024 cells); stochastic
# rounding keeps the drift a random walk within the per-step bound above, also over 2,000
# steps of the cavity settling.  The FP64 test above shows the wall treatment itself is exact.
@pytest.mark.parametrize("steps", [100, 2000])
def test_wall_mass_conservation_f32(steps):
    desc = workloads.cavity(32, n_base=25, Kn=0.075)
    s = Solver(desc)
    m0 = s.moments()[0].sum()
    s.step(steps)
    m1 = s.moments()[0].sum()
    assert abs(m1 - m0) / m0 < steps * FP32_DRIFT_PER_STEP


def test_uniform_bgk_fixed_point_gpu():
    desc = workloads.periodic_random(10, 10, n_base=25, storage="f64", Pr=1.0)
    desc["init"][..., 0] = 1.2
    desc["init"][..., 1] = 0.3
    desc["init"][..., 2] = -0.1
    desc["init"][..., 3] = 0.9
    s = Solver(desc)
    g0, h0 = s.read_cells(0, 100, 625)
    s.step(3)
    g1, h1 = s.read_cells(0, 100, 625)
    assert np.max(np.abs(g1 - g0)) < 1e-14 * np.max(g0)


def _oracle_stress(o, g, h):
    """Stress deviator of phi in the library's definition: 2 tau/(2 tau + dt) (P~ - p I)."""
    from oracle import dugks, kinetic
    m = kinetic.moments(g, h, o["sp"].xi, o["sp"].w, o["gas"])
    st = dugks.cell_state(g, h, o["sp"].xi, o["sp"].w, o["gas"], o["dt"])
    sf = 2.0 * st["tau"] / (2.0 * st["tau"] + o["dt"])
    P = m["P"]
    p = m["p"]
    return np.stack([(sf * (P[..., 0, 0] - p)).ravel(), (sf * P[..., 0, 1]).ravel(),
                     (sf * (P[..., 1, 1] - p)).ravel()])


def test_stress_output_f64():
    desc = workloads.periodic_random(12, 10, n_base=25, storage="f64")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(3)
    g, h = oracle_run(o, 3)
    sg = s.moments(M_SXX | M_SXY | M_SYY)
    so = _oracle_stress(o, g, h)
    scale = np.max(np.abs(so))
    assert scale > 1e-4
    np.testing.assert_allclose(sg, so, rtol=0, atol=1e-10 * scale)


# BF16 storage: every stored value keeps 8 significant bits, rounded stochastically (an
# unbiased rounding whose errors are independent from step to step).  A moment sums N_eff
# effective velocities, so its storage noise is about 2^-8 / sqrt(6 N_eff) per step: on the
# 101^2 grid (N_eff of a few hundred) the moments agree with the FP64 oracle to 1e-3 on the
# scales of the problem after a few steps -- rho and T relative, u in units of sqrt(RT),
# the heat flux in units of p sqrt(RT) and the stress deviator in units of p.  (On a 25^2
# grid the same noise reaches 2-4e-3.)
def test_bf16_storage_moments():
    desc = workloads.periodic_random(12, 8, n_base=101, storage="bf16")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(5)
    g, h = oracle_run(o, 5)
    gm = s.moments(M_RHO | M_U | M_V | M_T | M_QX | M_QY)
    om = oracle_moments(o, g, h)
    rho, T = om[0], om[3]
    p = rho * T
    cs = np.sqrt(T)
    assert np.max(np.abs(gm[0] - rho) / rho) < 1e-3
    assert np.max(np.abs(gm[3] - T) / T) < 1e-3
    assert np.max(np.abs(gm[1:3] - om[1:3]) / cs) < 1e-3
    assert np.max(np.abs(gm[4:6] - om[4:6]) / (p * cs)) < 1e-3
    sg = s.moments(M_SXX | M_SXY | M_SYY)
    so = _oracle_stress(o, g, h)
    assert np.max(np.abs(sg - so) / p) < 1e-3


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_supersonic_channel_freestream(walls, storage, tol):
    """Freestream inflow (Ma 2) and outflow sides; the bump is carried towards the outflow."""
    desc = workloads.supersonic_channel(30, 10, n_base=25, umax=8.0, storage=storage, walls=walls)
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(12)
    g, h = oracle_run(o, 12)
    om = oracle_moments(o, g, h)
    _compare(s.moments(), om, tol, tol * 3, tol, 100 * tol if storage == "f64" else 1e-3)
    assert np.max(np.abs(om[0] - desc["init"][..., 0].ravel())) > 1e-3
