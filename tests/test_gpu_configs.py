"""The benchmark configurations at full size, in the launch configuration the benchmark uses.

* Sod shock tube (200 cells, 101 velocities, FP64, BGK, Kn 1e-3), all 500 steps against
  the oracle.
* The cavity of the benchmark (64^2 cells, 101^2 velocities, FP32): one step against the
  oracle over the whole mesh, then properties over more steps (wall mass conservation, the
  lid speed bounding the flow).
* 64 batched cavities (seeded Kn in [1e-3, 10], meshes 32^2 ... 128^2, 101^2 velocities),
  adapted to multi-level spaces and advanced together as one graph: per-instance mass
  conservation, and sampled instances identical to the same case run alone.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_moments, oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def test_sod_full_500_steps_f64():
    desc = workloads.sod_1d()
    o = oracle_setup(desc)
    s = Solver(desc)
    M.mlvs_set_graph(s.h, True)
    s.step(500)
    g, h = oracle_run(o, 500)
    gm = s.moments()
    om = oracle_moments(o, g, h)
    assert np.max(np.abs(gm[0] - om[0]) / om[0]) < 1e-9
    assert np.max(np.abs(gm[1] - om[1])) < 1e-9
    assert np.max(np.abs(gm[3] - om[3]) / om[3]) < 1e-9


def test_cavity_bench_size_one_step_against_oracle():
    desc = workloads.cavity(64, n_base=101, umax=6.0, Kn=0.075, storage="f32")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(1)
    g, h = oracle_run(o, 1)
    gm = s.moments()
    om = oracle_moments(o, g, h)
    assert np.max(np.abs(gm[0] - om[0]) / om[0]) < 1e-5
    assert np.max(np.abs(gm[1:3] - om[1:3])) < 1e-5
    assert np.max(np.abs(gm[3] - om[3]) / om[3]) < 1e-5
    # more steps: wall mass conservation (FP32 storage bound) and |u| below the lid speed
    m0 = gm[0].sum()
    M.mlvs_set_graph(s.h, True)
    s.step(200)
    m = s.moments()
    assert abs(m[0].sum() - m0) / m0 < 3e-7
    Uw = 0.16 * np.sqrt(5.0 / 3.0)
    assert np.max(np.hypot(m[1], m[2])) < Uw


def test_batched_cavities_full_size():
    descs = workloads.batched_cavities()
    assert len(descs) == 64 and {d["nx"] for d in descs} <= {32, 48, 64, 96, 128}
    hs = [Solver(d, adaptive=1) for d in descs]
    p = M.adapt_params(5e-3, 2.5e-3, 5e-5, 0.05, 2)
    M.mlvs_step_many([s.h for s in hs], 4, use_graph=True)
    for s in hs:
        M.mlvs_adapt(s.h, p)
    mass0 = [s.moments(M.RHO)[0].sum() for s in hs]
    st = M.mlvs_step_many([s.h for s in hs], 6, use_graph=True)
    assert st.cell_velocity_updates > 0
    for s, m0 in zip(hs, mass0):
        assert abs(s.moments(M.RHO)[0].sum() - m0) / m0 < 1e-6
    # sampled instances, re-run alone with the same adaptation, give the same fields
    for i in (0, 17, 63):
        a = Solver(descs[i], adaptive=1)
        a.step(4)
        M.mlvs_adapt(a.h, p)
        a.step(6)
        np.testing.assert_array_equal(a.moments(), hs[i].moments())
        a.close()
    for s in hs:
        s.close()
