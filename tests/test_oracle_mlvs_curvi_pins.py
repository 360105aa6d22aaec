"""Pins of the oracle's multi-level step on curvilinear meshes (Sec. 3.4 on the O-grid step).

* On one space it is the uniform curvilinear step (itself pinned against the Cartesian step and
  the O-grid geometry), on an O-grid with a wall inside and a freestream side outside.
* On a Cartesian node grid with two spaces it is the Cartesian multi-level step (pinned against
  the uniform step and by exact conservation), with walls and with freestream sides.
* On a closed annulus (walls inside and outside) with three spaces, the area-weighted mass is
  conserved to rounding, which only holds if every face flux leaves one cell and enters the
  other with the same moments after the cross-level correction.
"""
import numpy as np
import pytest

from oracle import curvi, dugks, mapping, mlvs, mlvs_curvi
from paper_2609_35258_b300 import workloads
from tests.helpers import oracle_run, oracle_setup


def _state(desc, levels_of_cell, Ls):
    o = oracle_setup(desc)
    book = mlvs.SpaceBook(o["base"])
    keys = [book.uniform(L) for L in Ls]
    init = desc["init"]
    st = mlvs.MLVSState.from_primitives(o["mesh"], o["gas"], book, [keys[l] for l in levels_of_cell],
                                        init[..., 0], init[..., 1:3], init[..., 3], o["dt"], o["opt"])
    return o, st


def _with_nodes(desc):
    d = dict(desc)
    nx, ny = d["nx"], d["ny"]
    X, Y = np.meshgrid(np.arange(nx + 1) * d["Lx"] / nx, np.arange(ny + 1) * d["Ly"] / ny)
    d["nodes"] = np.stack([X, Y], axis=-1)
    return d


def test_single_space_is_the_curvilinear_step():
    desc = workloads.cylinder(12, 4, mach=2.0, Kn=0.1, n_base=13, umax=8.0, r_out=4.0, storage="f64")
    n = 48
    o, st = _state(desc, [0] * n, [0])
    assert isinstance(o["mesh"], curvi.CurviMesh)
    for _ in range(2):
        mlvs_curvi.step(st)
    g, h = oracle_run(o, 2)
    np.testing.assert_allclose(np.stack(st.g), g.reshape(n, -1), rtol=1e-12, atol=1e-14 * np.max(g))
    np.testing.assert_allclose(np.stack(st.h), h.reshape(n, -1), rtol=1e-12, atol=1e-14 * np.max(h))
    assert np.max(np.abs(g - o["g"])) > 1e-4 * np.max(g)          # the flow developed


@pytest.mark.parametrize("kind", ["cavity", "channel"])
def test_cartesian_nodes_two_spaces_are_the_cartesian_multilevel_step(kind):
    if kind == "cavity":
        desc = workloads.cavity(6, n_base=13, umax=5.0)
    else:
        desc = workloads.supersonic_channel(8, 4, mach=1.5, n_base=13, umax=6.0, walls=True)
    nx, ny = desc["nx"], desc["ny"]
    lev = [((c % nx) // 2 + (c // nx) // 2) % 2 for c in range(nx * ny)]
    _, a = _state(desc, lev, [0, 1])
    _, b = _state(_with_nodes(desc), lev, [0, 1])
    for _ in range(2):
        mlvs.step(a)
        mlvs_curvi.step(b)
    ga, gb = np.concatenate(a.g), np.concatenate(b.g)
    ha, hb = np.concatenate(a.h), np.concatenate(b.h)
    np.testing.assert_allclose(gb, ga, rtol=0, atol=1e-13 * np.max(np.abs(ga)))
    np.testing.assert_allclose(hb, ha, rtol=0, atol=1e-13 * np.max(np.abs(ha)))


def test_closed_annulus_with_three_spaces_conserves_mass():
    desc = workloads.cylinder(16, 5, mach=1.0, Kn=0.05, n_base=13, umax=6.0, r_out=3.0, storage="f64")
    desc["bc"] = ("periodic", "periodic", "wall", "wall")
    n = 80
    lev = [(c % 16) // 6 for c in range(n)]                      # spaces 0, 1, 2 around the annulus
    o, st = _state(desc, lev, [0, 1, 2])
    area = curvi.geometry(o["mesh"])["area"].ravel()
    tot0 = sum(a * m["rho"] for a, m in zip(area, st.moments()))
    for _ in range(3):
        mlvs_curvi.step(st)
    m = st.moments()
    tot1 = sum(a * x["rho"] for a, x in zip(area, m))
    assert abs(tot1 - tot0) < 1e-13 * tot0
    rho = np.array([x["rho"] for x in m])
    assert np.max(np.abs(rho - rho.mean())) > 1e-4                 # the flow is not uniform


def test_nine_moment_treatment_conserves_raw_moments_on_a_sheared_periodic_mesh():
    """Free-molecular limit (Kn 1e12) on a doubly periodic parallelogram mesh (sheared by 0.3,
    so faces are not axis-aligned and the y period moves x too), two spaces: the area-weighted
    sums of the nine raw moments are conserved to round-off with the nine-moment treatment,
    while the four-moment treatment lets the second moments and energy fluxes drift."""
    nx, ny = 8, 4
    desc = workloads.periodic_random(nx, ny, n_base=17, umax=5.0, Kn=1e12)
    dx, dy = desc["Lx"] / nx, desc["Ly"] / ny
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    desc["nodes"] = np.stack([i * dx + 0.3 * j * dy, j * dy], axis=-1)
    lev = [0 if (c % nx) < nx // 2 else 1 for c in range(nx * ny)]
    drift = {}
    for nm in (4, 9):
        o, st = _state(desc, lev, [0, 1])
        st.opt = dugks.Options(map_moments=nm)
        area = curvi.geometry(o["mesh"])["area"].ravel()

        def totals():
            return sum(a * mapping.raw9(g, h, st.book.space(k)) for a, g, h, k in zip(area, st.g, st.h, st.sp))

        R0 = totals()
        for _ in range(3):
            mlvs_curvi.step(st)
        drift[nm] = np.abs(totals() - R0) / np.max(np.abs(R0))
    assert np.max(drift[9]) < 1e-13
    assert np.min(drift[4][4:]) > 1e-7
