"""The eight-moment compatibility correction (Sec. 3.3.1, Eq. eq_eight_basis and Eq.
eq_eight_moment_constraint) on the tile path, through the C ABI, against the oracle's step
with compat_moments = 8: cells and faces take the correction whose heat-flux target is the
Shakhov model's own heat flux (1 - Pr) q, freestream sides keep the four-moment correction.
Cartesian (a lid-driven cavity: walls, Shakhov Pr 2/3) and curvilinear (an O-grid with a wall
and a freestream side).  Tolerances as the other parity tests: FP64 1e-10, FP32 1e-5.  The FP64
cavity also checks that the four-moment run misses the oracle's heat flux by far more than the
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


def test_eight_moment_needs_one_uniform_level():
    desc = workloads.cavity(8, n_base=25, storage="f64")
    with pytest.raises(M.MLVSError):
        Solver(desc, compat_moments=8, adaptive=1)
    with pytest.raises(M.MLVSError):
        Solver(desc, compat_moments=8, levels=(0, 1))
