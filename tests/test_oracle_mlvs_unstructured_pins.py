"""Pins of the oracle's multi-level step on unstructured meshes (Sec. 3.4 on the unstructured
step; the two-cavity case of Sec. 4 runs MLVS on unstructured cells).

* On one space it is the unstructured step (itself pinned against the Cartesian step).
* On a Cartesian quad mesh with two spaces and unlimited gradients it is the Cartesian
  multi-level step with central slopes (walls and lid included).
* On the closed two-cavity mesh at the paper's density ratio with three spaces, the mass is
  conserved to round-off.
"""
import numpy as np

from oracle import dugks, kinetic, mlvs, mlvs_unstructured, unstructured as un, vspace
from paper_2609_35258_b300 import workloads
from tests.helpers import oracle_setup


def _two_cavity_state(levels_of_cell_fn, Ls):
    nodes, cells = workloads.two_cavities(2)
    mesh = un.UMesh(nodes, cells)
    G = un.geometry(mesh)
    base = vspace.make_base(13, -5.0, 5.0, D=2)
    gas = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0, mu_ref=kinetic.mu_ref_from_kn(0.05, 0.81))
    book = mlvs.SpaceBook(base)
    keys = [book.uniform(L) for L in Ls]
    nc = mesh.ncell
    rho = np.where(G["cen"][:, 0] < 0.0, 1.0, 1e-3)
    lev = [levels_of_cell_fn(G["cen"][c]) for c in range(nc)]
    dt = un.time_step(mesh, vspace.uniform_space(base, 0).xi, 0.5)
    st = mlvs.MLVSState.from_primitives(mesh, gas, book, [keys[l] for l in lev], rho, np.zeros((nc, 2)),
                                        np.ones(nc), dt, dugks.Options())
    return mesh, G, st


def test_single_space_is_the_unstructured_step():
    mesh, G, st = _two_cavity_state(lambda c: 0, [0])
    sp = st.book.space(st.sp[0])
    g, h = np.stack(st.g), np.stack(st.h)
    for _ in range(2):
        mlvs_unstructured.step(st)
        g, h, _ = un.step(g, h, mesh, sp.xi, sp.w, st.gas, st.dt, st.opt)
    np.testing.assert_allclose(np.stack(st.g), g, rtol=0, atol=1e-13 * np.max(g))
    np.testing.assert_allclose(np.stack(st.h), h, rtol=0, atol=1e-13 * np.max(h))


def test_cartesian_quads_two_spaces_are_the_cartesian_multilevel_step():
    desc = workloads.cavity(6, n_base=13, umax=5.0)
    desc["limiter"] = "none"
    n = desc["nx"]
    lev = [((c % n) // 2 + (c // n) // 2) % 2 for c in range(n * n)]
    o = oracle_setup(desc)
    book = mlvs.SpaceBook(o["base"])
    keys = [book.uniform(L) for L in (0, 1)]
    init = desc["init"]
    a = mlvs.MLVSState.from_primitives(o["mesh"], o["gas"], book, [keys[l] for l in lev], init[..., 0],
                                       init[..., 1:3], init[..., 3], o["dt"], o["opt"])
    nodes, cells = workloads.quad_mesh(np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1))
    tol = 1e-9
    side = lambda m: 0 if m[0] < tol else (1 if m[0] > 1 - tol else (2 if m[1] < tol else 3))
    mesh = un.UMesh(nodes, cells, wall_of=side, wall=desc["wall"])
    b = mlvs.MLVSState.from_primitives(mesh, o["gas"], book, [keys[l] for l in lev], init[..., 0].ravel(),
                                       init[..., 1:3].reshape(-1, 2), init[..., 3].ravel(), o["dt"], o["opt"])
    for _ in range(2):
        mlvs.step(a)
        mlvs_unstructured.step(b, limiter="none")
    ga, gb = np.concatenate(a.g), np.concatenate(b.g)
    np.testing.assert_allclose(gb, ga, rtol=0, atol=1e-13 * np.max(np.abs(ga)))
    np.testing.assert_allclose(np.concatenate(b.h), np.concatenate(a.h), rtol=0,
                               atol=1e-13 * np.max(np.abs(np.concatenate(a.h))))


def test_closed_two_cavities_with_three_spaces_conserve_mass():
    # fine in the left cavity, level 1 in the channel, level 2 in the right cavity
    mesh, G, st = _two_cavity_state(lambda x: 0 if x[0] < -0.5 else (1 if x[0] < 0.5 else 2), [0, 1, 2])
    area = G["area"]
    m0 = sum(a * m["rho"] for a, m in zip(area, st.moments()))
    for _ in range(3):
        mlvs_unstructured.step(st)
    rho = np.array([m["rho"] for m in st.moments()])
    assert abs(np.sum(area * rho) - m0) < 1e-13 * m0
    assert rho.min() > 0.0
    chan = (G["cen"][:, 0] > 0.0) & (G["cen"][:, 0] < 0.5)
    assert rho[chan].max() > 2e-3                               # gas crossed x = 0
