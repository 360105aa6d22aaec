"""The library's host construction of curvilinear geometry (J^{-T}, areas, face normals and
lengths, reconstruction offsets with reflected ghosts and periodic images, cell widths) against
the oracle's, on CPU through the C ABI."""
import numpy as np
import pytest

from oracle import curvi
from paper_2609_35258_b300 import mlvs as M
from paper_2609_35258_b300 import workloads


def _meshes():
    nodes = workloads.ogrid_nodes(24, 8, 1.0, 4.0)
    yield "ogrid", nodes, True, False
    nx, ny = 7, 5
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    yield "sheared", np.stack([0.2 * i + 0.07 * j, 0.15 * j], axis=-1), True, True
    rng = np.random.default_rng(11)
    xs = np.cumsum(np.r_[0.0, 0.1 + 0.1 * rng.random(nx)])
    ys = np.cumsum(np.r_[0.0, 0.1 + 0.1 * rng.random(ny)])
    X, Y = np.meshgrid(xs, ys)
    X[1:-1, 1:-1] += 0.02 * rng.standard_normal((ny - 1, nx - 1))
    Y[1:-1, 1:-1] += 0.02 * rng.standard_normal((ny - 1, nx - 1))
    yield "perturbed", np.stack([X, Y], axis=-1), False, False


@pytest.mark.parametrize("name,nodes,px,py", list(_meshes()), ids=lambda v: v if isinstance(v, str) else "")
def test_host_geometry_matches_oracle(name, nodes, px, py):
    ny, nx = nodes.shape[0] - 1, nodes.shape[1] - 1
    bc = ("periodic" if px else "wall",) * 2 + ("periodic" if py else "wall",) * 2
    mesh = curvi.CurviMesh(nodes[..., 0], nodes[..., 1], bc=bc)
    G = curvi.geometry(mesh)
    cenP = curvi._ghost_centroids(G, mesh)
    cg, fg, wd = M.mlvs_mesh_geometry(nodes, px, py)
    scale = np.max(np.abs(nodes))
    tol = dict(rtol=0, atol=1e-13)
    np.testing.assert_allclose(cg[:4].T, G["Jt"].reshape(-1, 4), rtol=1e-12, atol=1e-12 / scale)
    np.testing.assert_allclose(cg[4], G["area"].ravel(), rtol=1e-13)
    nfx = nx if px else nx + 1
    for j in range(ny):
        for p in range(nfx):
            f = j * nfx + p
            np.testing.assert_allclose(fg[0:2, f], G["ni"][j, p], **tol)
            np.testing.assert_allclose(fg[2, f], G["li"][j, p], rtol=1e-14)
            np.testing.assert_allclose(fg[3:5, f], G["bi"][j, p] - cenP[j + 2, p + 1], rtol=0, atol=1e-13 * scale)
            np.testing.assert_allclose(fg[5:7, f], G["bi"][j, p] - cenP[j + 2, p + 2], rtol=0, atol=1e-13 * scale)
    nfy = ny if py else ny + 1
    for p in range(nfy):
        for i in range(nx):
            f = nfx * ny + p * nx + i
            np.testing.assert_allclose(fg[0:2, f], G["nj"][p, i], **tol)
            np.testing.assert_allclose(fg[2, f], G["lj"][p, i], rtol=1e-14)
            np.testing.assert_allclose(fg[3:5, f], G["bj"][p, i] - cenP[p + 1, i + 2], rtol=0, atol=1e-13 * scale)
            np.testing.assert_allclose(fg[5:7, f], G["bj"][p, i] - cenP[p + 2, i + 2], rtol=0, atol=1e-13 * scale)
    longest = np.maximum(np.maximum(G["li"][:, :-1], G["li"][:, 1:]), np.maximum(G["lj"][:-1, :], G["lj"][1:, :]))
    np.testing.assert_allclose(wd, (G["area"] / longest).ravel(), rtol=1e-14)


def test_host_geometry_rejects_clockwise_cells():
    nodes = workloads.ogrid_nodes(8, 3, 1.0, 3.0)[:, ::-1].copy()        # reversed orientation
    with pytest.raises(M.MLVSError):
        M.mlvs_mesh_geometry(nodes, True, False)
