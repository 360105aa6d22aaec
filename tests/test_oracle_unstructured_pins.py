"""Pins of the oracle's DUGKS step on unstructured polygonal meshes (the two-cavity case of
Sec. 4 runs on unstructured cells).

* On a Cartesian quad mesh given as a cell list, with unlimited least-squares gradients, it is
  the Cartesian step with central slopes (least squares over the four face neighbours is the
  central difference; the reflected ghosts are the Cartesian ghost copies), walls and a moving
  lid included.
* A gas at rest in equilibrium between walls at its own temperature is a fixed point on a
  triangulated two-cavity mesh (every face normal direction, the limiter active).
* The closed two-cavity mesh with the paper's pressure ratio of 1000 conserves mass to
  round-off, on quads and on triangles.
"""
import numpy as np
import pytest

from oracle import dugks, kinetic, unstructured as un, vspace
from paper_2609_35258_b300 import workloads
from tests.helpers import oracle_setup


def test_cartesian_quads_with_central_gradients_are_the_cartesian_step():
    desc = workloads.cavity(6, n_base=13, umax=5.0)
    desc["limiter"] = "none"
    o = oracle_setup(desc)
    n = desc["nx"]
    nodes, cells = workloads.quad_mesh(np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1))
    tol = 1e-9

    def side(mid):
        x, y = mid
        return 0 if x < tol else (1 if x > 1 - tol else (2 if y < tol else 3))

    mesh = un.UMesh(nodes, cells, wall_of=side, wall=desc["wall"])
    sp = o["sp"]
    assert abs(un.time_step(mesh, sp.xi, desc["cfl"]) - o["dt"]) < 1e-15
    rng = np.random.default_rng(4)
    g = o["g"] * (1.0 + 0.05 * rng.random(o["g"].shape))          # a non-uniform start
    h = o["h"] * (1.0 + 0.05 * rng.random(o["h"].shape))
    ga, ha = g, h
    gb, hb = g.reshape(n * n, -1), h.reshape(n * n, -1)
    for _ in range(2):
        ga, ha, _ = dugks.step(ga, ha, o["mesh"], sp.xi, sp.w, o["gas"], o["dt"], o["opt"])
        gb, hb, _ = un.step(gb, hb, mesh, sp.xi, sp.w, o["gas"], o["dt"], o["opt"], limiter="none")
    np.testing.assert_allclose(gb, ga.reshape(n * n, -1), rtol=0, atol=1e-13 * np.max(ga))
    np.testing.assert_allclose(hb, ha.reshape(n * n, -1), rtol=0, atol=1e-13 * np.max(ha))


def _two_cavity_setup(tri, n_base=13):
    nodes, cells = workloads.two_cavities(2)
    if tri:
        nodes, cells = workloads.triangulate(nodes, cells)
    mesh = un.UMesh(nodes, cells)
    base = vspace.make_base(n_base, -5.0, 5.0, D=2)
    sp = vspace.uniform_space(base, 0)
    gas = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0, mu_ref=kinetic.mu_ref_from_kn(0.05, 0.81))
    return mesh, sp, gas


@pytest.mark.parametrize("tri", [False, True])
def test_gas_at_rest_between_walls_at_its_temperature_is_a_fixed_point(tri):
    """Trapezoid velocity grid on [-8, 8]^2 (the rule is exact to round-off for a Gaussian of
    unit variance), no correction: the Maxwellian's discrete moments are its own, so it is a
    discrete equilibrium, and walls at rest at T = 1 emit it back (rho_w = 1 by symmetry)."""
    mesh, _, gas = _two_cavity_setup(tri)
    sp = vspace.uniform_space(vspace.make_base(25, -8.0, 8.0, D=2, rule="trapz"), 0)
    nc = mesh.ncell
    g, h = kinetic.maxwell_gh(np.ones(nc), np.zeros((nc, 2)), np.ones(nc), sp.xi, gas)
    opt = dugks.Options(compat_cell=False, compat_face=False)
    dt = un.time_step(mesh, sp.xi, 0.5)
    g1, h1, _ = un.step(g, h, mesh, sp.xi, sp.w, gas, dt, opt)
    np.testing.assert_allclose(g1, g, rtol=0, atol=1e-14 * np.max(g))
    np.testing.assert_allclose(h1, h, rtol=0, atol=1e-14 * np.max(h))


@pytest.mark.parametrize("tri", [False, True])
def test_closed_two_cavities_conserve_mass(tri):
    """The paper's initial state: gas at rest at T = 1, density 1 left of x = 0 and 1e-3 right."""
    mesh, sp, gas = _two_cavity_setup(tri)
    G = un.geometry(mesh)
    nc = mesh.ncell
    rho = np.where(G["cen"][:, 0] < 0.0, 1.0, 1e-3)
    g, h = dugks.initial_tilde(rho, np.zeros((nc, 2)), np.ones(nc), sp.xi, sp.w, gas)
    dt = un.time_step(mesh, sp.xi, 0.5)
    m0 = np.sum(G["area"] * np.sum(sp.w * g, axis=-1))
    for _ in range(4):
        g, h, _ = un.step(g, h, mesh, sp.xi, sp.w, gas, dt)
    rho1 = np.sum(sp.w * g, axis=-1)
    assert abs(np.sum(G["area"] * rho1) - m0) < 1e-13 * m0
    right = (G["cen"][:, 0] > 0.0) & (G["cen"][:, 0] < 0.5)
    assert rho1[right].max() > 2e-3                             # gas crossed x = 0 into the thin side
    assert rho1.min() > 0.0
