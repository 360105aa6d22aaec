"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: closed-form Gaussian integrals, polynomial
exactness of the quadrature, the definitions of the transformed distributions (Sec. 2.2),
the Shakhov heat-flux property (Sec. 2.1), the compatibility-recovery test state of Sec. 4.1.1,
conservation of the finite-volume update, and a brute-force free-molecular advection.
"""

import numpy as np
import pytest

from oracle import dugks, kinetic, vspace
from paper_2609_35258_b300 import workloads
from tests.helpers import oracle_run, oracle_setup


# ---------------------------------------------------------------- quadrature (Sec. 2.3)

@pytest.mark.parametrize("n", [5, 9, 101])
def test_boole_polynomial_exactness(n):
    a, b = -3.0, 5.0
    x, w = vspace.newton_cotes_1d(n, a, b, "boole")
    for k in range(6):
        exact = (b ** (k + 1) - a ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) <= 1e-12 * max(1.0, abs(exact))
    if n == 5:   # degree 6 is not integrated exactly by one Boole panel
        exact6 = (b ** 7 - a ** 7) / 7
        assert abs(np.sum(w * x ** 6) - exact6) > 1e-6


def test_simpson_trapz_exactness():
    x, w = vspace.newton_cotes_1d(11, 0.0, 2.0, "simpson")
    assert abs(np.sum(w * x ** 3) - 4.0) < 1e-13
    x, w = vspace.newton_cotes_1d(11, 0.0, 2.0, "trapz")
    assert abs(np.sum(w * x) - 2.0) < 1e-13


@pytest.mark.parametrize("n,sizes", [(101, [101, 51, 25, 13]), (201, [201, 101, 51, 25]),
                                     (89, [89, 45, 23, 11])])
def test_level_sizes_and_nesting(n, sizes):
    for L, s in enumerate(sizes):
        g = vspace.axis_groups(n, L)
        assert len(g) == s
        assert sorted(i for grp in g for i in grp) == list(range(n))
        # symmetric under xi -> -xi
        assert [len(x) for x in g] == [len(x) for x in reversed(g)]
        if L > 0:   # each group is a union of level L-1 groups
            prev = vspace.axis_groups(n, L - 1)
            starts = {grp[0] for grp in prev}
            ends = {grp[-1] for grp in prev}
            for grp in g:
                assert grp[0] in starts and grp[-1] in ends


def test_merged_space_preserves_weight_and_first_moment():
    base = vspace.make_base(101, -6, 6, D=2)
    s0 = vspace.uniform_space(base, 0)
    for L in (1, 2, 3):
        s = vspace.uniform_space(base, L)
        assert abs(s.w.sum() - s0.w.sum()) < 1e-12
        # weighted mean coordinates reproduce the first moments of the base grid exactly
        np.testing.assert_allclose(s.w @ s.xi, s0.w @ s0.xi, atol=1e-12)


# ---------------------------------------------------------------- model (Sec. 2.1)

def _fine_space(D, n=401, um=12.0):
    base = vspace.make_base(n, -um, um, D=D)
    return vspace.uniform_space(base, 0)


@pytest.mark.parametrize("D", [1, 2])
def test_maxwellian_moments_closed_form(D):
    sp = _fine_space(D)
    gas = kinetic.Gas(D=D, K=0.0, R=1.0, Pr=1.0)
    rho, T = 1.3, 0.8
    u = np.array([0.4, -0.2])[:D]
    g, h = kinetic.maxwell_gh(np.array(rho), u, np.array(T), sp.xi, gas)
    m = kinetic.moments(g, h, sp.xi, sp.w, gas)
    assert abs(m["rho"] - rho) < 1e-12
    np.testing.assert_allclose(m["u"], u, atol=1e-12)
    assert abs(m["T"] - T) < 1e-12
    np.testing.assert_allclose(m["q"], 0.0, atol=1e-12)
    np.testing.assert_allclose(m["P"], rho * T * np.eye(D), atol=1e-11)
    # internal energy carried by h: (3 - D + K)/2 rho R T
    assert abs(0.5 * np.sum(sp.w * h) - 0.5 * (3 - D) * rho * T) < 1e-12


@pytest.mark.parametrize("D,K", [(2, 0.0), (1, 0.0), (2, 2.0)])
def test_shakhov_heat_flux_property(D, K):
    """The Shakhov distribution has the conserved moments of its state and heat flux (1-Pr) q."""
    sp = _fine_space(D)
    gas = kinetic.Gas(D=D, K=K, R=1.0, Pr=2.0 / 3.0)
    rho, T = 0.9, 1.1
    u = np.array([0.3, 0.1])[:D]
    q = np.array([0.05, -0.03])[:D]
    g, h = kinetic.shakhov_gh(np.array(rho), u, np.array(T), q, sp.xi, gas)
    m = kinetic.moments(g, h, sp.xi, sp.w, gas)
    assert abs(m["rho"] - rho) < 1e-12
    np.testing.assert_allclose(m["u"], u, atol=1e-12)
    assert abs(m["T"] - T) < 1e-11
    np.testing.assert_allclose(m["q"], (1 - gas.Pr) * q, atol=1e-11)


def test_compat_correction_E1_state():
    """Sec. 4.1.1: (rho, u, v, T, R) = (1, 1, 0.2, 1, 0.5) on a nonuniform quadtree grid; the
    four-moment linear correction brings the conserved moments to round-off."""
    base = vspace.make_base(33, -4.0, 4.0, D=2)
    N1 = len(vspace.axis_groups(33, 1))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    kappa = np.where(r < 3, 0, np.where(r < 5, 1, 2)).astype(np.int64)
    sp = vspace.kappa_space(base, kappa)
    assert sp.nv < base.n ** 2
    gas = kinetic.Gas(D=2, R=0.5, Pr=1.0)
    rho, u, T = np.array(1.0), np.array([1.0, 0.2]), np.array(1.0)
    g, h = kinetic.maxwell_gh(rho, u, T, sp.xi, gas)
    tar = np.array([1.0, 1.0, 0.2, 0.5 * (1.0 + 0.04) + 1.5 * 0.5 * 1.0])
    def eps(g, h):
        M = kinetic.conserved(g, h, sp.xi, sp.w)
        return np.max(np.abs(M - tar) / np.abs(tar))
    assert eps(g, h) > 1e-5
    gc, hc = kinetic.compat_correct4(g, h, rho, u, T, sp.xi, sp.w, gas)
    assert eps(gc, hc) < 1e-14


def test_compat_correction_E1_against_the_paper_table():
    """tests/golden/e1_compatibility.json: the four-moment correction brings eps_M to
    round-off (printed 1.11e-16); ours, on our quadtree grid for the same state, is within a
    few units in the last place of it.  The uncorrected value depends on the paper's grid (a
    figure only), so only its being far above round-off is checked."""
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e1_compatibility.json")))
    st = fx["state"]
    sp = _quadtree_E1_space()
    gas = kinetic.Gas(D=2, R=st["R"], Pr=1.0)
    rho, u, T = np.array(st["rho"]), np.array([st["u"], st["v"]]), np.array(st["T"])
    g, h = kinetic.maxwell_gh(rho, u, T, sp.xi, gas)
    tar = np.array([st["rho"], st["rho"] * st["u"], st["rho"] * st["v"],
                    st["rho"] * (0.5 * (st["u"] ** 2 + st["v"] ** 2) + 1.5 * st["R"] * st["T"])])
    eps = lambda g, h: np.max(np.abs(kinetic.conserved(g, h, sp.xi, sp.w) - tar) / np.abs(tar))
    gc, hc = kinetic.compat_correct4(g, h, rho, u, T, sp.xi, sp.w, gas)
    assert eps(gc, hc) <= 4 * fx["eps_M"]["four_moment_linear"]
    assert eps(g, h) > 1e6 * fx["eps_M"]["four_moment_linear"]


def _quadtree_E1_space():
    base = vspace.make_base(33, -4.0, 4.0, D=2)
    N1 = len(vspace.axis_groups(33, 1))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    kappa = np.where(r < 3, 0, np.where(r < 5, 1, 2)).astype(np.int64)
    return vspace.kappa_space(base, kappa)


def test_compat8_hits_heat_flux_and_isotropic_stress():
    """Sec. 3.3.1, eight constraints: on the nonuniform grid of the E1 test, a Shakhov model
    with a heat flux carries after the correction the conserved moments, the heat flux the
    model prescribes ((1 - Pr) q, the Shakhov property pinned above) and a vanishing deviatoric
    stress, measured with the moment routine (not the correction's own kernels)."""
    sp = _quadtree_E1_space()
    gas = kinetic.Gas(D=2, R=0.5, Pr=2.0 / 3.0)
    rho, u, T, q = np.array(1.0), np.array([1.0, 0.2]), np.array(1.0), np.array([0.05, -0.03])
    g, h = kinetic.shakhov_gh(rho, u, T, q, sp.xi, gas)
    q_tar = (1.0 - gas.Pr) * q
    gc, hc = kinetic.compat_correct8(g, h, rho, u, T, q_tar, sp.xi, sp.w, gas)
    m0 = kinetic.moments(g, h, sp.xi, sp.w, gas)
    m = kinetic.moments(gc, hc, sp.xi, sp.w, gas)
    p = rho * gas.R * T
    assert abs(m0["P"][0, 0] - m0["P"][1, 1]) > 1e-6 * p             # the uncorrected model is off
    assert abs(m["rho"] - rho) < 1e-14
    np.testing.assert_allclose(m["u"], u, atol=1e-14)
    assert abs(m["T"] - T) < 1e-13
    np.testing.assert_allclose(m["q"], q_tar, atol=1e-13)
    assert abs(m["P"][0, 0] - m["P"][1, 1]) < 1e-13 * p
    assert abs(m["P"][0, 1]) < 1e-13 * p


def test_compat8_is_compat4_for_a_symmetric_state_and_idempotent():
    """A gas at rest without heat flux on a grid symmetric in xi_x, xi_y and under their swap:
    the four extra constraints already hold and decouple, so the eight-moment correction is
    the four-moment one; a corrected model is left unchanged by a second correction."""
    base = vspace.make_base(25, -5.0, 5.0, D=2)
    for L in (0, 1):
        sp = vspace.uniform_space(base, L)
        gas = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0)
        rho, u, T = np.array(1.3), np.array([0.0, 0.0]), np.array(0.9)
        g, h = kinetic.maxwell_gh(rho, u, T, sp.xi, gas)
        g4, h4 = kinetic.compat_correct4(g, h, rho, u, T, sp.xi, sp.w, gas)
        g8, h8 = kinetic.compat_correct8(g, h, rho, u, T, np.zeros(2), sp.xi, sp.w, gas)
        assert np.max(np.abs(g4 - g)) > 1e-12 * np.max(g)             # the correction does act
        np.testing.assert_allclose(g8, g4, rtol=0, atol=1e-14 * np.max(g4))
        np.testing.assert_allclose(h8, h4, rtol=0, atol=1e-14 * np.max(h4))
    sp = _quadtree_E1_space()
    gas = kinetic.Gas(D=2, R=0.5, Pr=2.0 / 3.0)
    rho, u, T, q = np.array(1.0), np.array([1.0, 0.2]), np.array(1.0), np.array([0.05, -0.03])
    g, h = kinetic.shakhov_gh(rho, u, T, q, sp.xi, gas)
    args = (rho, u, T, (1.0 - gas.Pr) * q, sp.xi, sp.w, gas)
    g1, h1 = kinetic.compat_correct8(g, h, *args)
    g2, h2 = kinetic.compat_correct8(g1, h1, *args)
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-14 * np.max(g1))
    np.testing.assert_allclose(h2, h1, rtol=0, atol=1e-14 * np.max(h1))


def test_step_with_eight_moment_correction_conserves():
    """The step with the eight-moment correction at cells and faces: the four collision
    invariants are still among the constraints, so a periodic run conserves to round-off,
    and the result differs from the four-moment step."""
    desc = workloads.periodic_random(8, 6, n_base=25, amp=0.2)
    o = oracle_setup(desc)
    sp = o["sp"]
    W0 = kinetic.conserved(o["g"], o["h"], sp.xi, sp.w).sum(axis=(0, 1))
    opt8 = dugks.Options(compat_moments=8)
    g, h = o["g"], o["h"]
    for _ in range(10):
        g, h, _ = dugks.step(g, h, o["mesh"], sp.xi, sp.w, o["gas"], o["dt"], opt8)
    W1 = kinetic.conserved(g, h, sp.xi, sp.w).sum(axis=(0, 1))
    assert np.max(np.abs(W1 - W0)) < 1e-12 * np.max(np.abs(W0))
    g4, _ = oracle_run(o, 10)
    assert np.max(np.abs(g - g4)) > 1e-10 * np.max(g4)


# ---------------------------------------------------------------- DUGKS (Sec. 2.2)

def test_transformed_distribution_algebra():
    rng = np.random.default_rng(1)
    phi, phiS = rng.random(50), rng.random(50)
    tau, dt = 0.37, 0.11
    s = dt / 2
    Om = (phiS - phi) / tau
    phit = phi - dt / 2 * Om
    np.testing.assert_allclose(dugks.bar_plus(phit, phiS, tau, dt), phi + s / 2 * Om, rtol=1e-13)
    np.testing.assert_allclose(dugks.tilde_plus(phi + s / 2 * Om, phit), phi + dt / 2 * Om, rtol=1e-13)
    phib = phi - s / 2 * Om
    np.testing.assert_allclose(dugks.recover(phib, phiS, tau, s), phi, rtol=1e-13)


def test_discrete_heat_flux_relation():
    """Eq. discrete_q: the q recovered from phi~ equals the heat flux of phi."""
    sp = _fine_space(2)
    gas = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0, mu_ref=0.05)
    rho, u, T = np.array(1.0), np.array([0.2, -0.1]), np.array(1.0)
    qphi = np.array([0.04, 0.02])
    # a distribution phi with heat flux qphi: Shakhov form with Pr' such that (1-Pr') = 1
    g1 = kinetic.Gas(D=2, R=1.0, Pr=0.0)
    gphi, hphi = kinetic.shakhov_gh(rho, u, T, qphi, sp.xi, g1)
    m = kinetic.moments(gphi, hphi, sp.xi, sp.w, gas)
    np.testing.assert_allclose(m["q"], qphi, atol=1e-11)
    tau = kinetic.viscosity(T, gas) / (rho * gas.R * T)
    gS, hS = kinetic.shakhov_gh(rho, u, T, qphi, sp.xi, gas)
    dt = 0.02
    gt = gphi - dt / 2 * (gS - gphi) / tau
    ht = hphi - dt / 2 * (hS - hphi) / tau
    st = dugks.cell_state(gt, ht, sp.xi, sp.w, gas, dt)
    np.testing.assert_allclose(st["q"], qphi, atol=1e-11)
    assert abs(st["rho"] - 1.0) < 1e-12 and abs(st["T"] - 1.0) < 1e-11


def test_uniform_bgk_fixed_point():
    desc = workloads.periodic_random(6, 5, n_base=25, Pr=1.0)
    desc["init"][..., 0] = 1.2
    desc["init"][..., 1] = 0.3
    desc["init"][..., 2] = -0.1
    desc["init"][..., 3] = 0.9
    o = oracle_setup(desc)
    g, h = oracle_run(o, 3)
    assert np.max(np.abs(g - o["g"])) < 1e-14 * np.max(o["g"])
    assert np.max(np.abs(h - o["h"])) < 1e-14 * np.max(o["h"])


def test_shakhov_rest_fixed_point():
    desc = workloads.periodic_random(6, 5, n_base=25)
    desc["init"][..., 0] = 1.0
    desc["init"][..., 1:3] = 0.0
    desc["init"][..., 3] = 1.0
    o = oracle_setup(desc)
    g, h = oracle_run(o, 3)
    assert np.max(np.abs(g - o["g"])) < 1e-13 * np.max(o["g"])


def test_periodic_conservation():
    desc = workloads.periodic_random(8, 6, n_base=25, amp=0.2)
    o = oracle_setup(desc)
    sp = o["sp"]
    W0 = kinetic.conserved(o["g"], o["h"], sp.xi, sp.w).sum(axis=(0, 1))
    g, h = oracle_run(o, 30)
    W1 = kinetic.conserved(g, h, sp.xi, sp.w).sum(axis=(0, 1))
    assert np.max(np.abs(W1 - W0)) < 1e-12 * np.max(np.abs(W0))
    assert np.max(np.abs(g - o["g"])) > 1e-4   # the state did evolve


def test_wall_mass_conservation():
    desc = workloads.cavity(8, n_base=25, Kn=0.075)
    o = oracle_setup(desc)
    sp = o["sp"]
    M0 = kinetic.conserved(o["g"], o["h"], sp.xi, sp.w)[..., 0].sum()
    g, h = oracle_run(o, 20)
    M1 = kinetic.conserved(g, h, sp.xi, sp.w)[..., 0].sum()
    assert abs(M1 - M0) < 1e-13 * M0
    st = dugks.cell_state(g, h, sp.xi, sp.w, o["gas"], o["dt"])
    assert np.max(st["u"][..., 0]) > 1e-3   # the lid drives the flow


def _vanleer(a, b):
    if (a > 0 and b > 0) or (a < 0 and b < 0):
        return 2 * a * b / (a + b)
    return 0.0


def test_free_molecular_limit_matches_scalar_advection():
    """tau -> infinity: each velocity decouples into linear advection with the characteristic
    reconstruction; compare against a brute-force per-velocity loop (D = 1, 8 periodic cells)."""
    desc = workloads.periodic_random(8, 1, n_base=13, umax=4.0, dim=1, Pr=1.0)
    desc["mu_ref"] = 1e16
    o = oracle_setup(desc, compat=False)
    g0 = o["g"][0].copy()     # [nx, nv]
    xi = o["sp"].xi[:, 0]
    dt, dx = o["dt"], o["mesh"].dx
    s = dt / 2
    nx = 8
    g1, _ = oracle_run(o, 1)
    ref = np.zeros_like(g0)
    for v in range(len(xi)):
        f = g0[:, v]
        sig = [_vanleer(f[(i + 1) % nx] - f[i], f[i] - f[i - 1]) / dx for i in range(nx)]
        face = []
        for i in range(nx):   # face i between cells i-1 and i
            L, R = i - 1, i
            vL = f[L] + (dx / 2 - xi[v] * s) * sig[L]
            vR = f[R] + (-dx / 2 - xi[v] * s) * sig[R]
            face.append(vL if xi[v] > 0 else (vR if xi[v] < 0 else 0.5 * (vL + vR)))
        for i in range(nx):
            ref[i, v] = f[i] - dt / dx * xi[v] * (face[(i + 1) % nx] - face[i])
    np.testing.assert_allclose(g1[0], ref, rtol=1e-12, atol=1e-14 * np.max(np.abs(g0)))


def test_sod_oracle_wave_structure():
    """Kn = 1e-3 Sod: after t = 0.1 the density has the rarefaction/contact/shock ordering
    between the two initial states (qualitative check of the 1-D path)."""
    desc = workloads.sod_1d(ncell=100, n_base=61, umax=10.0)
    o = oracle_setup(desc)
    nsteps = int(round(0.1 / o["dt"]))
    g, h = oracle_run(o, nsteps)
    st = dugks.cell_state(g, h, o["sp"].xi, o["sp"].w, o["gas"], o["dt"])
    rho = st["rho"][0]
    assert rho[0] == pytest.approx(1.0, abs=1e-3) and rho[-1] == pytest.approx(0.125, abs=1e-3)
    assert np.all(np.diff(rho) <= 1e-3)           # monotone non-increasing left to right
    assert np.max(st["u"][0, :, 0]) > 0.5         # gas accelerated to the right


def _far_setup(bc, far, init, nb=25, umax=7.0, Pr=2.0 / 3.0):
    base = vspace.make_base(nb, -umax, umax, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2, R=1.0, Pr=Pr, mu_ref=kinetic.mu_ref_from_kn(0.1, 0.81))
    ny, nx = init.shape[:2]
    mesh = dugks.Mesh(nx, ny, 1.0 / nx, 1.0 / ny, bc=bc, far=far)
    g, h = dugks.initial_tilde(init[..., 0], init[..., 1:3], init[..., 3], sp.xi, sp.w, gas)
    dt = dugks.time_step(mesh, sp.xi, 0.5, 2)
    return sp, gas, mesh, g, h, dt


def test_uniform_freestream_is_a_fixed_point():
    """Freestream on every side at the state of the gas: nothing enters or leaves that differs
    from the interior, at subsonic and supersonic speeds (BGK: the discrete heat flux of a
    moving Maxwellian is not exactly zero, so a Shakhov state would drift by itself)."""
    F = dugks.FREE
    for u in (0.4, 3.0):
        far = (1.2, u, -0.3, 0.8)
        init = np.zeros((6, 8, 4))
        init[...] = far
        sp, gas, mesh, g, h, dt = _far_setup((F, F, F, F), far, init, Pr=1.0)
        g1, h1, _ = dugks.step(g, h, mesh, sp.xi, sp.w, gas, dt)
        assert np.max(np.abs(g1 - g)) < 1e-14 * np.max(g)
        assert np.max(np.abs(h1 - h)) < 1e-14 * np.max(h)


def test_freestream_sides_mirror_symmetry():
    """Inflow from the left at +u and the mirrored problem (inflow from the right at -u) give
    mirrored solutions: the inward normals of the two sides are consistent."""
    F, P = dugks.FREE, dugks.PERIODIC
    ny, nx = 4, 10
    x = (np.arange(nx) + 0.5) / nx
    init = np.zeros((ny, nx, 4))
    init[..., 0] = 1.0 + 0.2 * np.exp(-(x - 0.35) ** 2 / 0.01)
    init[..., 1] = 1.5
    init[..., 3] = 1.0
    sp, gas, mesh, g, h, dt = _far_setup((F, F, P, P), (1.0, 1.5, 0.0, 1.0), init)
    for _ in range(5):
        g, h, _ = dugks.step(g, h, mesh, sp.xi, sp.w, gas, dt)
    m = kinetic.moments(g, h, sp.xi, sp.w, gas)
    init2 = init[:, ::-1].copy()
    init2[..., 1] = -1.5
    sp, gas, mesh, g2, h2, dt = _far_setup((F, F, P, P), (1.0, -1.5, 0.0, 1.0), init2)
    for _ in range(5):
        g2, h2, _ = dugks.step(g2, h2, mesh, sp.xi, sp.w, gas, dt)
    m2 = kinetic.moments(g2, h2, sp.xi, sp.w, gas)
    np.testing.assert_allclose(m2["rho"][:, ::-1], m["rho"], rtol=1e-12)
    np.testing.assert_allclose(m2["u"][:, ::-1, 0], -m["u"][..., 0], atol=1e-12)
    np.testing.assert_allclose(m2["T"][:, ::-1], m["T"], rtol=1e-12)
    assert np.max(np.abs(m["rho"] - init[..., 0])) > 1e-3           # the bump moved


# ------------------------------------------------------------------ curvilinear meshes

def _curvi_vs_cartesian(bc, nx=8, ny=6, Lx=1.0, Ly=0.75, Pr=2.0 / 3.0):
    from oracle import curvi
    base = vspace.make_base(17, -5, 5, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2, R=1.0, Pr=Pr, mu_ref=kinetic.mu_ref_from_kn(0.1, 0.81))
    rng = np.random.default_rng(9)
    rho = 1.0 + 0.1 * rng.random((ny, nx))
    u = 0.2 * rng.standard_normal((ny, nx, 2))
    T = 1.0 + 0.1 * rng.random((ny, nx))
    g, h = dugks.initial_tilde(rho, u, T, sp.xi, sp.w, gas)
    dx, dy = Lx / nx, Ly / ny
    cart = dugks.Mesh(nx, ny, dx, dy, bc=bc, wall=((0, 0, 1.0), (0, 0, 1.0), (0.1, 0, 1.0), (0.2, 0, 1.1)),
                      far=(1.0, 0.3, -0.1, 0.9))
    Xn, Yn = np.meshgrid(np.arange(nx + 1) * dx, np.arange(ny + 1) * dy)
    cm = curvi.CurviMesh(Xn, Yn, bc=bc, wall=cart.wall, far=cart.far)
    dt = dugks.time_step(cart, sp.xi, 0.5, 2)
    assert abs(curvi.time_step(cm, sp.xi, 0.5) - dt) < 1e-15
    g1, h1, _ = dugks.step(g, h, cart, sp.xi, sp.w, gas, dt)
    g2, h2, _ = curvi.step(g, h, cm, sp.xi, sp.w, gas, dt)
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-13 * np.max(g1))
    np.testing.assert_allclose(h2, h1, rtol=0, atol=1e-13 * np.max(h1))


def test_curvilinear_step_on_cartesian_nodes_is_the_cartesian_step():
    P, W, F, Z = dugks.PERIODIC, dugks.WALL, dugks.FREE, dugks.ZEROGRAD
    for bc in ((P, P, P, P), (P, P, W, W), (F, F, W, W), (Z, Z, P, P)):
        _curvi_vs_cartesian(bc)


def test_ogrid_geometry_and_free_stream_preservation():
    """O-grid: positive areas summing to the annulus area, closed cells (the normals of a cell
    sum to zero with their lengths), and a uniform BGK flow with freestream sides inside and
    outside stays uniform."""
    from oracle import curvi
    X, Y = curvi.ogrid(32, 12, 1.0, 4.0)
    cm = curvi.CurviMesh(X, Y, bc=(dugks.PERIODIC, dugks.PERIODIC, dugks.FREE, dugks.FREE),
                         far=(1.0, 0.8, 0.3, 1.0))
    G = curvi.geometry(cm)
    assert np.all(G["area"] > 0)
    # polygon of 32 sides: area of the annulus between the inscribed polygons
    poly = 0.5 * 32 * np.sin(2 * np.pi / 32)
    assert abs(G["area"].sum() - poly * (4.0 ** 2 - 1.0)) < 1e-12
    closure = (G["ni"][:, 1:] * G["li"][:, 1:, None] - G["ni"][:, :-1] * G["li"][:, :-1, None]
               + G["nj"][1:] * G["lj"][1:, :, None] - G["nj"][:-1] * G["lj"][:-1, :, None])
    assert np.max(np.abs(closure)) < 1e-13
    base = vspace.make_base(17, -5, 5, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2, R=1.0, Pr=1.0, mu_ref=0.05)
    n = G["area"].shape
    g, h = dugks.initial_tilde(np.full(n, 1.0), np.broadcast_to([0.8, 0.3], n + (2,)).copy(), np.full(n, 1.0),
                               sp.xi, sp.w, gas)
    dt = curvi.time_step(cm, sp.xi, 0.5)
    g1, h1, _ = curvi.step(g, h, cm, sp.xi, sp.w, gas, dt)
    assert np.max(np.abs(g1 - g)) < 1e-13 * np.max(g)


# ------------------------------------------- uniform flow of Sec. 4.1.3 (golden values)

@pytest.mark.parametrize("kn", ["0.1", "10"])
def test_uniform_flow_conserved_moment_errors_match_the_paper(kn):
    """tests/golden/e3_uniform_flow.json: the uniform flow (rho, u, T) = (1, (0.1, 0), 1),
    R = 0.5, on the 89^2 Boole grid over +-4 sqrt(2RT), started from the discrete Maxwellian
    without correction and stepped with the four-moment correction: the deviations of the
    discrete rho, rho u_x and E from their exact values are the paper's printed UVS values
    (three digits), and they stay put over the steps (the correction conserves them)."""
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e3_uniform_flow.json")))
    ref = fx["uvs_four_moment"][kn]
    desc = workloads.uniform_flow(nx=100, ny=10, Kn=float(kn), storage="f64")
    # two cells of the same periodic mesh spacing carry the uniform state
    d2 = dict(desc)
    d2["nx"], d2["ny"], d2["Lx"], d2["Ly"] = 2, 1, 0.02, 0.01
    d2["init"] = desc["init"][:1, :2]
    o = oracle_setup(d2, compat=False)
    oc = oracle_setup(d2, compat=True)
    assert abs(o["dt"] - oracle_setup(desc, compat=False)["dt"]) < 1e-15
    xi, w, gas = o["sp"].xi, o["sp"].w, o["gas"]

    def errs(g, h):
        G, Hh = g[0, 0], h[0, 0]
        rho = np.sum(w * G)
        rhou = np.sum(w * xi[:, 0] * G)
        E = 0.5 * np.sum(w * ((xi ** 2).sum(1) * G + Hh))
        return np.array([abs(rho - 1.0), abs(rhou - 0.1), abs(E - (0.5 * 0.01 + 1.5 * 0.5))])

    g, h = o["g"], o["h"]
    e0 = errs(g, h)
    for _ in range(20):
        g, h, _ = dugks.step(g, h, oc["mesh"], xi, w, gas, oc["dt"], oc["opt"])
    e1 = errs(g, h)
    np.testing.assert_allclose(e1, e0, rtol=1e-5)
    np.testing.assert_allclose(e1, [ref["eps_rho"], ref["eps_rhoux"], ref["eps_E"]], rtol=1e-2)
