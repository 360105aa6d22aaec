"""The unstructured-mesh step through the C ABI on the GPU against the oracle's unstructured
step (the two-cavity expansion runs on unstructured cells).

* Two-cavity meshes of quads and of triangles at the paper's density ratio of 1000: FP64
  within 1e-11 and FP32 within 2e-5 of the largest value after three steps.
* A quad cavity with a moving lid (a second wall index), FP64.
* The eight-moment compatibility correction at cells and faces, FP64 and FP32.
* The two-cavity mesh at full size (13,600 cells, close to the paper's 12,012) with 61^2
  velocities, FP32, 20 steps: the mass stays constant (closed walls) and the flow stays
  mirror-symmetric about the channel axis (the mesh and the initial state are).
"""
import numpy as np
import pytest

from tests.helpers import have_gpu
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from tests import test_ustep_emu as E  # noqa: E402
from oracle import unstructured as un  # noqa: E402


def _run_gpu(cfg, nodes, cells, W0, steps, edge_wall=None):
    h = M.mlvs_ucreate(cfg, nodes, cells, W0, edge_wall)
    try:
        M.mlvs_ustep(h, steps)
        g, hh = M.mlvs_uread(h, len(cells))
        return g, hh, M.mlvs_uinfo(h)[2]
    finally:
        M.mlvs_udestroy(h)


@pytest.mark.parametrize("tri", [False, True], ids=["quads", "triangles"])
def test_two_cavities_fp64(tri):
    nodes, cells, mesh, W0 = E._two_cavity(tri)
    g, h, dt = _run_gpu(E._cfg(M.F64, [(0.0, 0.0, 1.0)]), nodes, cells, W0, 3)
    go, ho, dto = E._run_oracle(mesh, W0, 3)
    assert dt == pytest.approx(dto, rel=1e-15)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-11 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-11 * np.max(np.abs(ho)))


def test_two_cavities_fp32():
    nodes, cells, mesh, W0 = E._two_cavity(True)
    g, h, _ = _run_gpu(E._cfg(M.F32, [(0.0, 0.0, 1.0)]), nodes, cells, W0, 3)
    go, ho, _ = E._run_oracle(mesh, W0, 3)
    np.testing.assert_allclose(g, go, rtol=0, atol=2e-5 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=2e-5 * np.max(np.abs(ho)))


def test_lid_driven_quads_with_two_walls():
    n = 8
    nodes, cells = workloads.quad_mesh(np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1))
    walls = [(0.0, 0.0, 1.0), (0.4, 0.0, 1.0)]
    top = lambda mid: 1 if mid[1] > 1.0 - 1e-9 else 0
    mesh = un.UMesh(nodes, cells, wall_of=top, wall=tuple(walls))
    edge_wall = [[top(0.5 * (nodes[c[k]] + nodes[c[(k + 1) % 4]])) for k in range(4)] for c in cells]
    W0 = np.tile([1.0, 0.0, 0.0, 1.0], (len(cells), 1))
    g, h, _ = _run_gpu(E._cfg(M.F64, walls), nodes, cells, W0, 3, edge_wall)
    go, ho, _ = E._run_oracle(mesh, W0, 3)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-11 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-11 * np.max(np.abs(ho)))


def test_full_size_two_cavities_conserve_mass_and_mirror_symmetry():
    nodes, cells = workloads.two_cavities(10)
    geo = M.mlvs_umesh_geometry(nodes, cells)
    nc = len(cells)
    assert nc == 13600
    W0 = np.zeros((nc, 4))
    W0[:, 0] = np.where(geo["cx"] < 0.0, 1.0, 1e-3)
    W0[:, 3] = 1.0
    h = M.mlvs_ucreate(E._cfg(M.F32, [(0.0, 0.0, 1.0)], n_base=61, umax=5.0, vpc=64), nodes, cells, W0)
    try:
        M.mlvs_ustep(h, 1)
        W1 = M.mlvs_ucells(h, nc)
        M.mlvs_ustep(h, 20)
        W2 = M.mlvs_ucells(h, nc)
    finally:
        M.mlvs_udestroy(h)
    m1, m2 = np.sum(geo["area"] * W1[0]), np.sum(geo["area"] * W2[0])
    assert abs(m2 - m1) < 1e-5 * m1
    right = geo["cx"] > 0.0                                     # gas crosses x = 0 into the thin side
    assert np.sum((geo["area"] * W2[0])[right]) > 1.2 * np.sum((geo["area"] * W1[0])[right])
    # mirror pairs (x, y) <-> (x, -y): density equal, v opposite.  The bounds are of the largest
    # value: FP32 rounding is relative to the dense side, and the generated mesh's centroids are
    # mirrored only to about 2e-13 (shoelace cancellation), which 21 steps of the expansion
    # amplify to 1e-8 even in FP64, in the oracle as in these passes.  The passes compiled for
    # the CPU give 4.7e-7 and 4.1e-5 on this mesh with 13^2 velocities.
    key = {(round(x, 9), round(y, 9)): i for i, (x, y) in enumerate(zip(geo["cx"], geo["cy"]))}
    mirror = np.array([key[(round(x, 9), round(-y, 9))] for x, y in zip(geo["cx"], geo["cy"])])
    np.testing.assert_allclose(W2[0][mirror], W2[0], rtol=0, atol=2e-5 * np.max(W2[0]))
    np.testing.assert_allclose(W2[2][mirror], -W2[2], rtol=0, atol=5e-4 * np.max(np.abs(W2[1])))


@pytest.mark.parametrize("storage,tol", [(M.F64, 1e-11), (M.F32, 2e-5)], ids=["f64", "f32"])
def test_eight_moment_correction(storage, tol):
    nodes, cells, mesh, W0 = E._two_cavity(True)
    cfg = E._cfg(storage, [(0.0, 0.0, 1.0)])
    cfg.compat_moments = 8
    g, h, _ = _run_gpu(cfg, nodes, cells, W0, 3)
    go, ho, _ = E._run_oracle(mesh, W0, 3, nmom=8)
    np.testing.assert_allclose(g, go, rtol=0, atol=tol * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=tol * np.max(np.abs(ho)))
