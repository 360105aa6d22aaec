"""The eight-moment compatibility correction (Sec. 3.3.1, Eq. eq_eight_basis and Eq.
eq_eight_moment_constraint) on the tile path, through the C ABI, against the oracle's step
with compat_moments = 8: cells and faces take the correction whose heat-flux target is the
Shakhov model's own heat flux (1 - Pr) q, freestream sides keep the four-moment correction.
Cartesian (a lid-driven cavity: walls, Shakhov Pr 2/3) and curvilinear (an O-grid with a wall
and a freestream side) on the uniform base space, and the cavity on one space cut from the base
grid (levels 0..2 of the quadtree, not a tensor product: the model sums come from the space's
rows), element by element against the oracle's step on that space.  Tolerances as the other
parity tests: FP64 1e-10, FP32 1e-5 on moments and 2e-5 of the largest value on f.  The FP64
runs also check that the four-moment correction misses the oracle by far more than the
tolerance, so that the comparison sees the correction.
"""
import dataclasses

import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_moments, oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import dugks, mlvs as omlvs, vspace  # noqa: E402
from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def _run(desc, steps, compat_moments):
    s = Solver(desc, compat_moments=compat_moments)
    s.step(steps)
    m = s.moments()
    s.close()
    return m


def _check(gm, om, tol):
    rho, T = om[0], om[3]
    assert np.max(np.abs(gm[0] - rho) / rho) < tol
    assert np.max(np.abs(gm[1:3] - om[1:3])) < 10 * tol
    assert np.max(np.abs(gm[3] - T) / T) < tol
    qs = np.max(np.abs(om[4:6]))
    assert np.max(np.abs(gm[4:6] - om[4:6])) < 100 * tol * qs


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_eight_moment_cavity_matches_oracle(storage, tol):
    desc = workloads.cavity(12, n_base=25, Kn=0.075, storage=storage)
    o = oracle_setup(desc)
    o["opt"] = dataclasses.replace(o["opt"], compat_moments=8)
    steps = 6
    gm = _run(desc, steps, 8)
    g, h = oracle_run(o, steps)
    om = oracle_moments(o, g, h)
    _check(gm, om, tol)
    if storage == "f64":   # the four-moment run is far outside the tolerance
        g4 = _run(desc, steps, 4)
        assert np.max(np.abs(g4[4:6] - om[4:6])) > 1e3 * 100 * tol * np.max(np.abs(om[4:6]))


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_eight_moment_ogrid_matches_oracle(storage, tol):
    desc = workloads.cylinder(24, 8, mach=2.0, Kn=0.1, n_base=25, umax=8.0, r_out=4.0, storage=storage)
    o = oracle_setup(desc)
    o["opt"] = dataclasses.replace(o["opt"], compat_moments=8)
    steps = 6
    gm = _run(desc, steps, 8)
    g, h = oracle_run(o, steps)
    om = oracle_moments(o, g, h)
    _check(gm, om, tol)
    assert np.max(np.abs(om[0] - 1.0)) > 1e-3          # the flow developed


def _cut_kappa(n_base):
    """Quadtree levels 0 near the origin, 1 around it, 2 outside: a space cut from the base grid."""
    N1 = len(vspace.axis_groups(n_base, 1))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    return np.where(r < N1 / 5, 0, np.where(r < N1 / 3, 1, 2)).astype(np.uint8)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 2e-5)])
def test_eight_moment_cut_space_matches_oracle(storage, tol):
    n = 12
    desc = workloads.cavity(n, n_base=25, Kn=0.075, storage=storage)
    ka = _cut_kappa(25)
    o = oracle_setup(desc)
    book = omlvs.SpaceBook(o["base"])
    S = book.space(book.get(ka.astype(np.int64)))
    s = Solver(desc, levels=(ka,), compat_moments=8)
    x, y, w = M.mlvs_level_info(s.h, 0)
    np.testing.assert_allclose(np.stack([x, y], 1), S.xi, rtol=0, atol=1e-13)
    nv = S.xi.shape[0]
    assert nv < 25 * 25                                   # a cut space
    g0, h0 = [], []
    for c in range(n * n):
        g, h = s.read_cells(c, 1, nv)
        g0.append(g[0].copy())
        h0.append(h[0].copy())
    steps = 6
    s.step(steps)
    G, H = np.stack(g0).reshape(n, n, nv), np.stack(h0).reshape(n, n, nv)
    opt8 = dataclasses.replace(o["opt"], compat_moments=8)
    G8, H8 = G, H
    for _ in range(steps):
        G8, H8, _ = dugks.step(G8, H8, o["mesh"], S.xi, S.w, o["gas"], o["dt"], opt8)
    ref_g, ref_h = G8.reshape(n * n, nv), H8.reshape(n * n, nv)
    gmax, hmax = np.max(np.abs(ref_g)), np.max(np.abs(ref_h))
    worst = 0.0
    for c in range(n * n):
        g, h = s.read_cells(c, 1, nv)
        worst = max(worst, np.max(np.abs(g[0] - ref_g[c])) / gmax, np.max(np.abs(h[0] - ref_h[c])) / hmax)
    s.close()
    assert worst < tol, worst
    if storage == "f64":   # the four-moment step is far outside the tolerance
        G4, H4 = G, H
        for _ in range(steps):
            G4, H4, _ = dugks.step(G4, H4, o["mesh"], S.xi, S.w, o["gas"], o["dt"], o["opt"])
        d4 = max(np.max(np.abs(G4 - G8)) / gmax, np.max(np.abs(H4 - H8)) / hmax)
        assert d4 > 1e3 * tol, d4


def test_eight_moment_needs_one_level():
    desc = workloads.cavity(8, n_base=25, storage="f64")
    with pytest.raises(M.MLVSError):
        Solver(desc, compat_moments=8, adaptive=1)
    with pytest.raises(M.MLVSError):
        Solver(desc, compat_moments=8, levels=(0, 1))


def _cross_kappa(n_base):
    """Level 0 on a band of blocks across every x, level 1 on a band across every y, levels
    2 and 3 elsewhere: a cut space whose rows draw on the groups of every level along both axes
    (about 180 distinct row entries on the 101^2 base)."""
    N1 = len(vspace.axis_groups(n_base, 1))
    mid = N1 // 2
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - mid, yy - mid)
    return np.where(np.abs(yy - mid) <= 2, 0,
                    np.where(np.abs(xx - mid) <= 2, 1, np.where(r < N1 / 3, 2, 3))).astype(np.uint8)


@pytest.mark.parametrize("compat_moments", [4, 8])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 2e-5)])
def test_row_sums_with_many_entries_match_oracle(compat_moments, storage, tol):
    """The row sums with many row entries (their shared memory per warp well above the pair
    moments' area) on a 101^2 base, against the oracle's step on that space."""
    n = 4
    desc = workloads.periodic_random(n, n, n_base=101, umax=6.0, storage=storage, amp=0.2)
    ka = _cross_kappa(101)
    o = oracle_setup(desc)
    book = omlvs.SpaceBook(o["base"])
    S = book.space(book.get(ka.astype(np.int64)))
    s = Solver(desc, levels=(ka,), compat_moments=compat_moments)
    nv = S.xi.shape[0]
    g0, h0 = [], []
    for c in range(n * n):
        g, h = s.read_cells(c, 1, nv)
        g0.append(g[0].copy())
        h0.append(h[0].copy())
    steps = 3
    s.step(steps)
    G, H = np.stack(g0).reshape(n, n, nv), np.stack(h0).reshape(n, n, nv)
    opt = dataclasses.replace(o["opt"], compat_moments=compat_moments)
    for _ in range(steps):
        G, H, _ = dugks.step(G, H, o["mesh"], S.xi, S.w, o["gas"], o["dt"], opt)
    ref_g, ref_h = G.reshape(n * n, nv), H.reshape(n * n, nv)
    gmax, hmax = np.max(np.abs(ref_g)), np.max(np.abs(ref_h))
    worst = 0.0
    for c in range(n * n):
        g, h = s.read_cells(c, 1, nv)
        worst = max(worst, np.max(np.abs(g[0] - ref_g[c])) / gmax, np.max(np.abs(h[0] - ref_h[c])) / hmax)
    s.close()
    assert worst < tol, worst
