"""Pins of the multi-level parts of the oracle (Sec. 3.2-3.4).

Projection and mapping are checked against their defining properties (aggregation preserves
mass and energy, refinement inverts coarsening, the corrections hit their targets), the
repeated-projection test of Sec. 4.1.2 against its closed-form invariants, the criterion and
clustering against brute force and the limits the paper states, and the multi-level step
against the single-space oracle and exact conservation.
"""
import numpy as np
import pytest

from oracle import cluster, criterion, dugks, kinetic, mapping, mlvs, vspace
from paper_2609_35258_b300 import workloads
from tests.helpers import oracle_run, oracle_setup


def _rand_gh(sp, seed=0):
    rng = np.random.default_rng(seed)
    return 0.1 + rng.random(sp.nv), 0.1 + rng.random(sp.nv)


def test_projection_preserves_mass_energy_and_refine_inverts():
    base = vspace.make_base(33, -5, 5, D=2)
    fine, coarse = vspace.uniform_space(base, 0), vspace.uniform_space(base, 2)
    g, h = _rand_gh(fine)
    gc, hc = mapping.project(g, h, fine, coarse)
    x2f = np.sum(fine.xi ** 2, -1)
    x2c = np.sum(coarse.xi ** 2, -1)
    assert abs(np.sum(coarse.w * gc) - np.sum(fine.w * g)) < 1e-13
    assert abs(np.sum(coarse.w * (hc + x2c * gc)) - np.sum(fine.w * (h + x2f * g))) < 1e-12
    gr, hr = mapping.project(gc, hc, coarse, fine)
    g2, h2 = mapping.project(gr, hr, fine, coarse)
    np.testing.assert_allclose(g2, gc, rtol=1e-14)
    np.testing.assert_allclose(h2, hc, rtol=1e-13, atol=1e-14)


def test_correct4_hits_targets():
    base = vspace.make_base(33, -5, 5, D=2)
    src, dst = vspace.uniform_space(base, 0), vspace.uniform_space(base, 1)
    gas = kinetic.Gas(D=2, R=1.0)
    g, h = kinetic.maxwell_gh(np.array(1.1), np.array([0.3, -0.2]), np.array(0.9), src.xi, gas)
    g2, h2 = mapping.map4(g, h, src, dst, gas)
    np.testing.assert_allclose(kinetic.conserved(g2, h2, dst.xi, dst.w),
                               kinetic.conserved(g, h, src.xi, src.w), rtol=1e-13)


def _e2_initial(base, kind, eps):
    """Sec. 4.1.2 state (rho, U, V, T, R) = (1, 1, 0, 1, 0.5) with g = g_eq (1 + eps delta),
    delta orthogonalised on the initial space against (1, xi_x, xi_y, xi^2)."""
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2, R=0.5)
    rho, u, T = np.array(1.0), np.array([1.0, 0.0]), np.array(1.0)
    g, h = kinetic.maxwell_gh(rho, u, T, sp.xi, gas)
    g, h = kinetic.compat_correct4(g, h, rho, u, T, sp.xi, sp.w, gas)   # exact initial moments
    c = sp.xi - np.array([1.0, 0.0])
    d = c[:, 0] * (np.sum(c * c, -1) - 5 * 0.5) if kind == "heat" else c[:, 0] ** 2 - c[:, 1] ** 2
    B = np.stack([np.ones(sp.nv), sp.xi[:, 0], sp.xi[:, 1], np.sum(sp.xi ** 2, -1)])
    Wg = sp.w * g
    coef = np.linalg.solve((B * Wg) @ B.T, (B * Wg) @ d)
    d = d - coef @ B
    return sp, gas, g * (1 + eps * d), h


def _e2_sequence(base):
    return [(1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (0, 0)]


@pytest.mark.parametrize("kind", ["heat", "stress"])
@pytest.mark.parametrize("eps", [1e-5, 1e-3, 1e-1])
def test_repeated_projection_invariants(kind, eps):
    """Four-moment mapping keeps rho = 1, rho U = 1, rho E = 1.25 (Table of Sec. 4.1.2);
    nine-moment mapping also returns q_x and Pi_xx - Pi_yy to their initial values."""
    base = vspace.make_base(65, -6, 6, D=2)
    sp0, gas, g, h = _e2_initial(base, kind, eps)
    m0 = kinetic.moments(g, h, sp0.xi, sp0.w, gas)
    assert abs(m0["rho"] - 1) < 1e-12 and abs(m0["mom"][0] - 1) < 1e-12
    assert abs(m0["rhoE"] - 1.25) < 1e-12             # 1/2 rho U^2 + 3/2 rho R T
    cur, g4, h4, g9, h9 = sp0, g, h, g, h
    for Lx, Ly in _e2_sequence(base):
        nxt = vspace.aniso_space(base, Lx, Ly)
        g4, h4 = mapping.map4(g4, h4, cur, nxt, gas)
        g9, h9 = mapping.map9(g9, h9, cur, nxt)
        cur = nxt
    m4 = kinetic.moments(g4, h4, cur.xi, cur.w, gas)
    assert abs(m4["rho"] - 1) < 1e-12 and abs(m4["mom"][0] - 1) < 1e-12
    assert abs(m4["rhoE"] - 1.25) < 1e-12
    m9 = kinetic.moments(g9, h9, cur.xi, cur.w, gas)
    assert abs(m9["rhoE"] - 1.25) < 1e-12
    d0 = m0["P"][0, 0] - m0["P"][1, 1]
    d9 = m9["P"][0, 0] - m9["P"][1, 1]
    assert abs(m9["q"][0] - m0["q"][0]) < 1e-12 * max(1.0, abs(m0["q"][0]) / eps)
    assert abs(d9 - d0) < 1e-12 * max(1.0, abs(d0) / eps)
    if kind == "heat":
        assert abs(m0["q"][0]) > 0.1 * eps          # the perturbation carries a heat flux


def test_repeated_projection_against_the_paper_table():
    """tests/golden/e2_repeated_projection.json holds the 4- and 9-moment rows of the paper's
    table for the repeated projection sequence.  Our perturbation delta is normalised
    differently (q_x0 = 0.5 eps here, 0.7071 eps there), so what is compared is what does not
    depend on it: the basic moments as printed (three decimals), the constrained moment of a
    9-moment row back at its initial value (printed final / printed initial = 1.000) and the
    other higher moment unchanged; in the 4-moment rows the higher moments are not kept."""
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e2_repeated_projection.json")))
    base = vspace.make_base(65, -6, 6, D=2)
    for row in fx["rows"]:
        kind, eps = row["kind"], row["eps"]
        sp0, gas, g, h = _e2_initial(base, kind, eps)
        m0 = kinetic.moments(g, h, sp0.xi, sp0.w, gas)
        cur = sp0
        for Lx, Ly in _e2_sequence(base):
            nxt = vspace.aniso_space(base, Lx, Ly)
            g, h = mapping.map9(g, h, cur, nxt) if row["method"] == "9-moment" else mapping.map4(g, h, cur, nxt, gas)
            cur = nxt
        m = kinetic.moments(g, h, cur.xi, cur.w, gas)
        assert round(float(m["rho"]), 3) == row["rho"]
        assert round(float(m["mom"][0]), 3) == row["rhoU"]
        assert round(float(m["rhoE"]), 3) == row["rhoE"]
        dpi = lambda mm: mm["P"][0, 0] - mm["P"][1, 1]
        con, other = (("q_x", lambda mm: mm["q"][0]), dpi) if kind == "heat" else (("dPi", dpi), lambda mm: mm["q"][0])
        name, get = con
        if row["method"] == "9-moment":
            printed_ratio = row[name] / (fx["initial"][kind][name + "_over_eps"] * eps)
            assert round(float(get(m) / get(m0)), 3) == round(printed_ratio, 3) == 1.0
            assert abs(other(m) - other(m0)) < 1e-12
        elif eps <= 1e-3:
            assert abs(get(m) - get(m0)) > 10 * abs(get(m0))      # the table's "completely distorted"


# ------------------------------------------------------------------ criterion and clustering

def test_criterion_uniform_maxwellian():
    base = vspace.make_base(33, -6, 6, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2)
    g, h = kinetic.maxwell_gh(np.array(1.0), np.array([0.0, 0.0]), np.array(1.0), sp.xi, gas)
    g2, h2 = g.reshape(33, 33), h.reshape(33, 33)
    N1 = len(vspace.axis_groups(33, 1))
    kap = criterion.criterion_2d(g2, h2, base, np.zeros((N1, N1), int), 5e-3, 2.5e-3)
    # symmetric under xi -> -xi, fine at the centre, merged in the far tails
    np.testing.assert_array_equal(kap, kap[::-1, ::-1])
    np.testing.assert_array_equal(kap, kap.T)
    assert kap[N1 // 2, N1 // 2] == 0
    assert kap[0, 0] == 3
    # brute force: every level-1 block left fine has I_B >= C_merge
    M1, M2 = criterion._contrib(g2, h2, base)
    g1 = vspace.axis_groups(33, 1)
    for by in range(N1):
        for bx in range(N1):
            if kap[by, bx] == 0:
                sl = (slice(g1[by][0], g1[by][-1] + 1), slice(g1[bx][0], g1[bx][-1] + 1))
                assert max(M1[sl].sum(), M2[sl].sum()) >= 2.5e-3


def test_criterion_hysteresis_band():
    base = vspace.make_base(33, -6, 6, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2)
    g, h = kinetic.maxwell_gh(np.array(1.0), np.array([0.0, 0.0]), np.array(1.0), sp.xi, gas)
    g2, h2 = g.reshape(33, 33), h.reshape(33, 33)
    N1 = len(vspace.axis_groups(33, 1))
    big = 10.0       # every block in the band [C_merge, C_split]
    k_prev0 = criterion.criterion_2d(g2, h2, base, np.zeros((N1, N1), int), big, 0.0)
    k_prev3 = criterion.criterion_2d(g2, h2, base, np.full((N1, N1), 3), big, 0.0)
    assert np.all(k_prev0 == 0) and np.all(k_prev3 == 3)


def test_transport_test_only_rejects():
    base = vspace.make_base(33, -6, 6, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2)
    g, h = kinetic.maxwell_gh(np.array(1.0), np.array([0.5, 0.0]), np.array(1.0), sp.xi, gas)
    g2, h2 = g.reshape(33, 33), h.reshape(33, 33)
    N1 = len(vspace.axis_groups(33, 1))
    z = np.zeros((N1, N1), int)
    k_free = criterion.criterion_2d(g2, h2, base, z, 5e-3, 2.5e-3)
    k_tr = criterion.criterion_2d(g2, h2, base, z, 5e-3, 2.5e-3, eps_merge=1e-6)
    assert np.all(k_tr <= k_free)
    assert np.sum(k_tr) < np.sum(k_free)


def test_graded_distance_properties():
    a = np.zeros(10, int)
    b = np.full(10, 3)
    assert cluster.graded_distance(a, a) == 0
    assert cluster.graded_distance(a, b) == 1
    rng = np.random.default_rng(3)
    x, y = rng.integers(0, 4, 10), rng.integers(0, 4, 10)
    assert cluster.graded_distance(x, y) == cluster.graded_distance(y, x)
    assert cluster.graded_distance(x, y) == np.sum(np.abs(x - y)) / 30


def test_clustering_limits_and_enclosure():
    rng = np.random.default_rng(5)
    pats = rng.integers(0, 4, size=(6, 12))
    K = pats[rng.integers(0, 6, size=200)]
    lab1, rep1 = cluster.cluster(K, 1.0)
    assert rep1.shape[0] == 1 and np.all(lab1 == 0)
    lab0, rep0 = cluster.cluster(K, 0.0)
    assert rep0.shape[0] == len(np.unique(K, axis=0))
    for tau in (0.0, 0.1, 0.3, 1.0):
        lab, rep = cluster.cluster(K, tau)
        for c in range(rep.shape[0]):
            assert np.all(rep[c] <= K[lab == c])          # kappa_rep <= kappa_M for members
    # uniform requirement -> one space
    lab, rep = cluster.cluster(np.tile(pats[0], (50, 1)), 0.0)
    assert rep.shape[0] == 1


# ------------------------------------------------------------------ multi-level step

def _mlvs_from_desc(desc, levels_of_cell, Ls):
    o = oracle_setup(desc)
    book = mlvs.SpaceBook(o["base"])
    keys = [book.uniform(L) for L in Ls]
    init = desc["init"]
    st = mlvs.MLVSState.from_primitives(o["mesh"], o["gas"], book, [keys[l] for l in levels_of_cell],
                                        init[..., 0], init[..., 1:3], init[..., 3], o["dt"], o["opt"])
    return o, st


def test_single_level_mlvs_equals_uvs():
    desc = workloads.periodic_random(6, 5, n_base=13, umax=5.0)
    o, st = _mlvs_from_desc(desc, [0] * 30, [0])
    for _ in range(2):
        mlvs.step(st)
    g, h = oracle_run(o, 2)
    np.testing.assert_allclose(np.stack(st.g), g.reshape(30, -1), rtol=1e-12, atol=1e-15)


def test_single_level_mlvs_equals_uvs_walls():
    desc = workloads.cavity(5, n_base=13, umax=5.0)
    o, st = _mlvs_from_desc(desc, [0] * 25, [0])
    for _ in range(2):
        mlvs.step(st)
    g, h = oracle_run(o, 2)
    np.testing.assert_allclose(np.stack(st.g), g.reshape(25, -1), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("walls", [False, True])
def test_single_level_mlvs_equals_uvs_freestream(walls):
    """Freestream sides (and diffuse walls): the multi-level step on one space is the uniform
    step, whose freestream faces are pinned by the fixed-point and mirror tests."""
    desc = workloads.supersonic_channel(6, 4, mach=1.5, n_base=13, umax=6.0, walls=walls)
    o, st = _mlvs_from_desc(desc, [0] * 24, [0])
    for _ in range(2):
        mlvs.step(st)
    g, h = oracle_run(o, 2)
    np.testing.assert_allclose(np.stack(st.g), g.reshape(24, -1), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(np.stack(st.h), h.reshape(24, -1), rtol=1e-12, atol=1e-15)


def test_two_level_freestream_box_stays_mirror_symmetric():
    """A gas at rest between two freestream sides at rest, with a centred bump and the outer
    columns on the coarser space: the solution stays symmetric under x -> -x, so both sides'
    inward normals and the cross-level faces on either side are consistent."""
    nx, ny = 8, 4
    desc = workloads.supersonic_channel(nx, ny, mach=0.0, n_base=13, umax=5.0, walls=True)
    lev = [1 if (c % nx) in (0, 1, nx - 2, nx - 1) else 0 for c in range(nx * ny)]
    o, st = _mlvs_from_desc(desc, lev, [0, 1])
    for _ in range(3):
        mlvs.step(st)
    m = st.moments()
    rho = np.array([x["rho"] for x in m]).reshape(ny, nx)
    ux = np.array([x["u"][0] for x in m]).reshape(ny, nx)
    T = np.array([x["T"] for x in m]).reshape(ny, nx)
    np.testing.assert_allclose(rho[:, ::-1], rho, rtol=1e-12)
    np.testing.assert_allclose(ux[:, ::-1], -ux, atol=1e-12)
    np.testing.assert_allclose(T[:, ::-1], T, rtol=1e-12)
    assert np.max(np.abs(ux)) > 1e-4                     # the bump spreads outwards


def _cold_beam_on_coarse_space():
    """A narrow Maxwellian on the fine grid projected to level 2: the projection leaves
    moment defects that a correction must remove."""
    base = vspace.make_base(33, -6.0, 6.0, D=2)
    src, dst = vspace.uniform_space(base, 0), vspace.uniform_space(base, 2)
    gas = kinetic.Gas(D=2, R=1.0)
    g, h = kinetic.maxwell_gh(np.array(1.0), np.array([1.7, -0.4]), np.array(0.15), src.xi, gas)
    tar = kinetic.conserved(g, h, src.xi, src.w)
    gp, hp = mapping.project(g, h, src, dst)
    return gp, hp, tar, dst, gas


def test_exponential_correction_meets_targets_and_keeps_signs():
    """Eq. exponential_moment_correction: the corrected values meet the four targets, keep the
    sign of every provisional value (the factor is positive; a nonnegative g stays nonnegative)
    and leave zeros at zero, where the additive unit-weight correction of the same defect makes
    tails negative."""
    gp, hp, tar, dst, gas = _cold_beam_on_coarse_space()
    gp = np.where(gp < 1e-300, 0.0, gp)
    defect = np.abs(kinetic.conserved(gp, hp, dst.xi, dst.w) - tar) / np.abs(tar).max()
    assert defect.max() > 1e-4                                       # a real defect
    m = kinetic.moments(gp, hp, dst.xi, dst.w, gas)
    gl, hl = mapping.correct4(gp, hp, tar, m["T"], dst, gas)
    assert gl.min() < 0.0                                            # the additive correction goes negative
    ge, he = mapping.correct_exp4(gp, hp, tar, dst)
    M = kinetic.conserved(ge, he, dst.xi, dst.w)
    np.testing.assert_allclose(M, tar, rtol=1e-13, atol=1e-13 * np.abs(tar).max())
    assert gp.min() >= 0.0 and ge.min() >= 0.0                      # aggregation keeps g >= 0, and so does the factor
    assert np.all(ge[gp == 0.0] == 0.0)
    assert np.all(np.sign(ge) == np.sign(gp))
    assert np.all(np.sign(he) == np.sign(hp))                        # h = H - xi^2 g may be slightly negative after projection


def test_exponential_correction_without_defect_is_the_identity():
    base = vspace.make_base(17, -5.0, 5.0, D=2)
    sp = vspace.uniform_space(base, 1)
    g, h = _rand_gh(sp, seed=3)
    tar = kinetic.conserved(g, h, sp.xi, sp.w)
    ge, he = mapping.correct_exp4(g, h, tar, sp)
    np.testing.assert_allclose(ge, g, rtol=1e-13)
    np.testing.assert_allclose(he, h, rtol=1e-13)


def test_positive_mapping_fallback_on_a_level_switch():
    """The level switch of a cold narrow distribution to a coarse space: the four-moment
    linear mapping makes tails of g negative; with the fallback the exponential correction
    takes over, every value of g stays nonnegative and the conserved moments still match."""
    base = vspace.make_base(33, -6.0, 6.0, D=2)
    src, dst = vspace.uniform_space(base, 0), vspace.uniform_space(base, 2)
    gas = kinetic.Gas(D=2, R=1.0)
    g, h = kinetic.maxwell_gh(np.array(1.0), np.array([1.7, -0.4]), np.array(0.15), src.xi, gas)
    tar = kinetic.conserved(g, h, src.xi, src.w)
    gl, _ = mapping.map_state(g, h, src, dst, gas)
    gp, hp = mapping.map_state(g, h, src, dst, gas, positive=True)
    assert gl.min() < 0.0 <= g.min()
    assert gp.min() >= 0.0
    np.testing.assert_allclose(kinetic.conserved(gp, hp, dst.xi, dst.w), tar, rtol=1e-13, atol=1e-13)


def test_positive_mapping_keeps_exact_conservation(monkeypatch):
    """Two spaces with the fallback on: the exponential correction takes over for some mapped
    stencil states (counted), and the run still conserves to round-off."""
    calls = []
    exp4 = mapping.correct_exp4
    monkeypatch.setattr(mapping, "correct_exp4", lambda *a, **k: calls.append(1) or exp4(*a, **k))
    desc = workloads.periodic_random(8, 4, n_base=17, umax=5.0)
    lev = [0 if (c % 8) < 4 else 1 for c in range(32)]
    o, st = _mlvs_from_desc(desc, lev, [0, 1])
    st.opt = dugks.Options(positive_mapping=True)
    W0 = st.totals()
    for _ in range(4):
        mlvs.step(st)
    W1 = st.totals()
    assert len(calls) > 0
    assert np.max(np.abs(W1 - W0)) < 1e-12 * np.max(np.abs(W0))


def _raw9_totals(st):
    book = st.book
    return sum(mapping.raw9(g, h, book.space(k)) for g, h, k in zip(st.g, st.h, st.sp))


def test_nine_moment_flux_matching_conserves_raw_moments_without_collisions():
    """Free-molecular limit (Kn 1e12), two spaces on a periodic mesh: transport alone conserves
    the global sum of every velocity moment, so the nine raw moments (mass, momentum, energy,
    Gxx, Gyy, Gxy, Jx, Jy) are conserved to round-off exactly when every cross-level flux keeps
    all nine on both sides (Sec. 3.4, the nine-moment treatment); with the four-moment
    treatment the second moments drift."""
    desc = workloads.periodic_random(8, 4, n_base=17, umax=5.0, Kn=1e12)
    lev = [0 if (c % 8) < 4 else 1 for c in range(32)]
    drift = {}
    for nm in (4, 9):
        o, st = _mlvs_from_desc(desc, lev, [0, 1])
        st.opt = dugks.Options(map_moments=nm)
        R0 = _raw9_totals(st)
        for _ in range(4):
            mlvs.step(st)
        R1 = _raw9_totals(st)
        drift[nm] = np.abs(R1 - R0) / np.max(np.abs(R0))
    assert np.max(drift[9]) < 1e-13
    assert np.min(drift[4][4:]) > 1e-6                    # Gxx .. Jy are not matched by 4 moments
    assert np.max(drift[4][:4]) < 1e-13                   # the conserved ones are


def test_nine_moment_mapping_keeps_the_freestream_box_symmetric():
    nx, ny = 8, 4
    desc = workloads.supersonic_channel(nx, ny, mach=0.0, n_base=13, umax=5.0, walls=True)
    lev = [1 if (c % nx) in (0, 1, nx - 2, nx - 1) else 0 for c in range(nx * ny)]
    o, st = _mlvs_from_desc(desc, lev, [0, 1])
    st.opt = dugks.Options(map_moments=9)
    for _ in range(3):
        mlvs.step(st)
    m = st.moments()
    rho = np.array([x["rho"] for x in m]).reshape(ny, nx)
    ux = np.array([x["u"][0] for x in m]).reshape(ny, nx)
    np.testing.assert_allclose(rho[:, ::-1], rho, rtol=1e-12)
    np.testing.assert_allclose(ux[:, ::-1], -ux, atol=1e-12)


def test_two_level_conservation_and_flux_matching():
    """Mixed levels on a periodic density wave: cross-level faces conserve exactly (Sec. 3.4)."""
    desc = workloads.periodic_random(8, 4, n_base=17, umax=5.0)
    lev = [0 if (c % 8) < 4 else 1 for c in range(32)]
    o, st = _mlvs_from_desc(desc, lev, [0, 1])
    W0 = st.totals()
    for _ in range(4):
        mlvs.step(st)
    W1 = st.totals()
    assert np.max(np.abs(W1 - W0)) < 1e-12 * np.max(np.abs(W0))
    # the coarse side really is coarser
    assert st.book.space(st.sp[7]).nv < st.book.space(st.sp[0]).nv


def test_remap_preserves_moments():
    desc = workloads.periodic_random(4, 4, n_base=17, umax=5.0)
    o, st = _mlvs_from_desc(desc, [0] * 16, [0])
    before = st.totals()
    k1 = st.book.uniform(2)
    for c in range(0, 16, 2):
        mlvs.remap(st, c, k1)
    after = st.totals()
    np.testing.assert_allclose(after, before, rtol=1e-13)
