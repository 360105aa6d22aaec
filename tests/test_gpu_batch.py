"""Batching, CUDA graphs and the chunking autotuner, through the C ABI.

A graph replays exactly the kernels of the regular path with the same arguments, so results
must be bit-identical to regular launches; the BF16 stochastic rounding draws its bits from a
device step counter, so replays do not repeat them.  A group of handles stepped together
(mlvs_step_many) must equal each handle stepped alone.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def _state(s, ncell, cap):
    g, h = s.read_cells(0, ncell, cap)
    return g, h


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_graph_steps_bit_identical(storage):
    desc = workloads.cavity(24, n_base=25, storage=storage)
    a, b = Solver(desc), Solver(desc)
    M.mlvs_set_graph(b.h, True)
    for n in (1, 4, 5, 2, 7):          # odd and even counts, moments calls in between
        a.step(n)
        b.step(n)
        np.testing.assert_array_equal(a.moments(), b.moments())
    ga, ha = _state(a, 576, 625)
    gb, hb = _state(b, 576, 625)
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ha, hb)
    st = b.step(6)
    assert st.launches > 0


def test_graph_with_levels_and_adaptation():
    desc = workloads.cavity(16, n_base=41, storage="f32")
    a, b = Solver(desc, adaptive=1), Solver(desc, adaptive=1)
    p = M.adapt_params(5e-3, 2.5e-3, 5e-5, 0.05, 2)
    for s in (a, b):
        M.mlvs_set_adaptation(s.h, p, 5)
    M.mlvs_set_graph(b.h, True)
    a.step(23)
    b.step(23)
    np.testing.assert_array_equal(a.moments(M.RHO | M.U | M.V | M.T | M.LEVEL),
                                  b.moments(M.RHO | M.U | M.V | M.T | M.LEVEL))


def test_step_many_equals_separate_steps():
    descs = [workloads.cavity(16, n_base=25, Kn=0.01), workloads.cavity(24, n_base=25, Kn=1.0),
             workloads.periodic_random(20, 12, n_base=25)]
    alone = [Solver(d) for d in descs]
    group = [Solver(d) for d in descs]
    for s in alone:
        s.step(9)
    st = M.mlvs_step_many([s.h for s in group], 9, use_graph=True)
    assert st.cell_velocity_updates == 9 * 625 * (256 + 576 + 240)
    for s1, s2 in zip(alone, group):
        np.testing.assert_array_equal(s1.moments(), s2.moments())
    # and once more without graphs
    st = M.mlvs_step_many([s.h for s in group], 3, use_graph=False)
    for s in alone:
        s.step(3)
    for s1, s2 in zip(alone, group):
        np.testing.assert_array_equal(s1.moments(), s2.moments())


def test_instances_in_one_handle_match_single_handles():
    desc = workloads.periodic_random(16, 8, n_base=25, storage="f64")
    init2 = np.stack([desc["init"], desc["init"][::-1].copy()])
    both = Solver(desc, n_instances=2, init=init2)
    M.mlvs_set_graph(both.h, True)
    one = Solver(desc)
    d2 = dict(desc)
    d2["init"] = desc["init"][::-1].copy()
    two = Solver(d2)
    for s in (both, one, two):
        s.step(6)
    np.testing.assert_allclose(both.moments(instance=0), one.moments(), rtol=0, atol=0)
    np.testing.assert_allclose(both.moments(instance=1), two.moments(), rtol=0, atol=0)


def test_autotune_keeps_conservation():
    desc = workloads.periodic_random(40, 24, n_base=25, storage="f64")
    s = Solver(desc)
    m0 = s.moments(M.RHO | M.RHOE)
    t, table = M.mlvs_autotune(s.h, 2)
    assert t in (148, 296, 444, 592, 888, 1184, 1776)
    assert np.all(table > 0)
    s.step(4)
    m1 = s.moments(M.RHO | M.RHOE)
    np.testing.assert_allclose(m1.sum(axis=1), m0.sum(axis=1), rtol=1e-12)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_chunking_changes_only_the_rounding(storage):
    """A different velocity chunking splits the moment sums differently: the results agree to
    rounding."""
    desc = workloads.cavity(20, n_base=25, storage=storage)
    a, b = Solver(desc), Solver(desc)
    M.mlvs_set_tuning(b.h, 148)
    a.step(3)
    b.step(3)
    M.mlvs_set_tuning(b.h, 1776)
    a.step(4)
    b.step(4)
    ma, mb = a.moments(), b.moments()
    tol = 1e-12 if storage == "f64" else 1e-6
    assert np.max(np.abs(ma - mb)) < tol * np.max(np.abs(ma))


def test_step_many_with_each_case_reclustering_on_its_own():
    """Independent cases with their own criterion thresholds, clustering thresholds and
    adaptation intervals (so their numbers of representative spaces change independently)
    advance through the batched launch exactly as they do alone."""
    descs = [workloads.cavity(16, n_base=41, storage="f32"), workloads.periodic_random(20, 12, n_base=41)]
    params = [(M.adapt_params(5e-3, 2.5e-3, 5e-5, 0.05, 2), 5), (M.adapt_params(1e-2, 5e-3, 0.0, 0.2, 3), 7)]
    alone = [Solver(d, adaptive=1) for d in descs]
    group = [Solver(d, adaptive=1) for d in descs]
    for s, (p, k) in zip(alone + group, params + params):
        M.mlvs_set_adaptation(s.h, p, k)
    for s in alone:
        s.step(23)
    M.mlvs_step_many([s.h for s in group], 23, use_graph=True)
    F = M.RHO | M.U | M.V | M.T | M.LEVEL
    for s1, s2 in zip(alone, group):
        np.testing.assert_array_equal(s1.moments(F), s2.moments(F))
