"""The library's host construction of unstructured-mesh geometry (areas, centroids, widths,
faces with their cells, normals, lengths and midpoints, each cell's signed faces, the inverse
least-squares normal matrices) against the oracle's, and its Hilbert cell order, on CPU
through the C ABI.  Pins of the oracle's least-squares matrices and gradients come first."""
import numpy as np
import pytest
from scipy.spatial import Delaunay

from oracle import unstructured as un
from paper_2609_35258_b300 import mlvs as M
from paper_2609_35258_b300 import workloads


def _ccw(nodes, cells):
    out = []
    for c in cells:
        P = nodes[list(c)]
        a = np.sum(P[:, 0] * np.roll(P[:, 1], -1) - np.roll(P[:, 0], -1) * P[:, 1])
        out.append(tuple(c) if a > 0 else tuple(c[::-1]))
    return out


def _meshes():
    yield "two_cavities_quads", *workloads.two_cavities(2)
    yield "two_cavities_triangles", *workloads.triangulate(*workloads.two_cavities(2))
    rng = np.random.default_rng(5)
    pts = np.vstack([rng.random((60, 2)), [[0, 0], [1, 0], [1, 1], [0, 1]]])
    yield "delaunay", pts, _ccw(pts, Delaunay(pts).simplices)
    nodes, quads = workloads.quad_mesh(np.linspace(0, 1, 5), np.linspace(0, 0.5, 3))
    nodes, tri = workloads.triangulate(nodes, quads[4:])
    yield "mixed", nodes, list(quads[:4]) + list(tri)


MESHES = list(_meshes())
IDS = [m[0] for m in MESHES]
ERR_ARG = next(k for k, v in M.STATUS.items() if v == "MLVS_ERR_ARG")


# -- pins of the oracle ------------------------------------------------------------------------

def test_oracle_normal_matrix_on_a_cartesian_grid_is_diagonal():
    """Every cell of a dx x dy grid sees offsets (+-dx, 0), (0, +-dy), the reflected ghosts at
    the boundary included: sum d d^T = diag(2 dx^2, 2 dy^2)."""
    dx, dy = 0.25, 0.1
    nodes, cells = workloads.quad_mesh(np.arange(5) * dx, np.arange(4) * dy)
    Ms = un.ls_normal_matrix(un.UMesh(nodes, cells))
    np.testing.assert_allclose(Ms, np.broadcast_to(np.diag([2 * dx * dx, 2 * dy * dy]), Ms.shape),
                               rtol=1e-13, atol=1e-16)


def test_oracle_gradients_are_exact_for_a_linear_field_in_interior_cells():
    """Least squares recovers the gradient of a linear field from exact neighbour differences
    (boundary cells see a zero ghost difference, so only interior cells are exact)."""
    _, nodes, cells = MESHES[2]
    mesh = un.UMesh(nodes, cells)
    G = un.geometry(mesh)
    a = np.array([[1.7, -0.4], [-2.0, 3.1]])                 # two velocities, two gradients
    P = 0.3 + G["cen"] @ a.T                                   # (Nc, 2)
    grad = un._gradients(P, mesh, "none")
    interior = [c for c, fs in enumerate(G["cell_faces"]) if all(G["fR"][f] >= 0 for f, _ in fs)]
    assert len(interior) > 20
    np.testing.assert_allclose(grad[interior], np.broadcast_to(a, (len(interior), 2, 2)), rtol=1e-11)


# -- library against the oracle ---------------------------------------------------------------

@pytest.mark.parametrize("name,nodes,cells", MESHES, ids=IDS)
def test_host_unstructured_geometry_matches_oracle(name, nodes, cells):
    mesh = un.UMesh(nodes, cells)
    G = un.geometry(mesh)
    g = M.mlvs_umesh_geometry(nodes, cells)
    scale = np.max(np.abs(nodes))
    np.testing.assert_allclose(g["area"], G["area"], rtol=1e-13)
    np.testing.assert_allclose(np.stack([g["cx"], g["cy"]], -1), G["cen"], rtol=0, atol=1e-14 * scale)
    # faces: same numbering (by node pair), same cells, normals out of L
    np.testing.assert_array_equal(g["L"], G["fL"])
    np.testing.assert_array_equal(g["R"], G["fR"])
    np.testing.assert_allclose(np.stack([g["nx"], g["ny"]], -1), G["fn"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(g["length"], G["fl"], rtol=1e-14)
    np.testing.assert_allclose(np.stack([g["midx"], g["midy"]], -1), G["fb"], rtol=0, atol=1e-15 * scale)
    # the edge's nodes in L's traversal direction give the same normal
    e = nodes[g["n1"]] - nodes[g["n0"]]
    np.testing.assert_allclose(np.stack([e[:, 1], -e[:, 0]], -1) / g["length"][:, None], G["fn"], atol=1e-14)
    # each cell's signed faces: the oracle's set, listed in the cell's edge order
    ptr, cf = g["cell_ptr"], g["cell_face"]
    for c, fs in enumerate(G["cell_faces"]):
        mine = cf[ptr[c]:ptr[c + 1]]
        assert sorted(mine) == sorted(f if s > 0 else -f - 1 for f, s in fs)
        poly = cells[c]
        for k, s in enumerate(mine):
            f = s if s >= 0 else -s - 1
            assert {poly[k], poly[(k + 1) % len(poly)]} == {g["n0"][f], g["n1"][f]}
    # widths give the oracle's time step; inverse normal matrices
    longest = np.array([max(G["fl"][f] for f, _ in fs) for fs in G["cell_faces"]])
    np.testing.assert_allclose(g["width"], G["area"] / longest, rtol=1e-14)
    Minv = np.linalg.inv(un.ls_normal_matrix(mesh))
    mine = np.stack([np.stack([g["mxx"], g["mxy"]], -1), np.stack([g["mxy"], g["myy"]], -1)], -2)
    np.testing.assert_allclose(mine, Minv, rtol=1e-12, atol=1e-12 * np.max(np.abs(Minv)))


def test_size_query_returns_the_face_count():
    nodes, cells = workloads.two_cavities(2)
    g = M.mlvs_umesh_geometry(nodes, cells)
    assert len(g["L"]) == len(un.geometry(un.UMesh(nodes, cells))["fL"])
    # Euler's formula for a planar mesh without holes: V - E + F = 1 (F = cells)
    assert len(nodes) - len(g["L"]) + len(cells) == 1


def _expect_arg_error(nodes, cells):
    with pytest.raises(M.MLVSError) as e:
        M.mlvs_umesh_geometry(nodes, cells)
    assert e.value.status == ERR_ARG


def test_rejects_mesh_defects():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [2.0, 0.5]])
    _expect_arg_error(nodes, [(0, 3, 2, 1)])                         # clockwise
    _expect_arg_error(nodes, [(0, 1, 7)])                            # node out of range
    _expect_arg_error(nodes, [(0, 1)])                               # fewer than three nodes
    _expect_arg_error(nodes, [(0, 1, 2), (1, 2, 3)])                 # shared edge, same direction
    _expect_arg_error(nodes, [(0, 1, 2), (2, 1, 4), (0, 2, 1)])      # an edge used three times
    _expect_arg_error(nodes, [(0, 1, 1, 2)])                         # a zero-length edge


def test_rejects_too_small_face_capacity():
    import ctypes as C
    nodes, cells = workloads.quad_mesh(np.linspace(0, 1, 3), np.linspace(0, 1, 3))
    xy = np.ascontiguousarray(nodes, dtype=np.float64)
    ptr = np.arange(0, 4 * len(cells) + 1, 4, dtype=np.int32)
    cn = np.ascontiguousarray(np.concatenate(cells), dtype=np.int32)
    nf = C.c_int()
    bufs = [np.zeros(64) for _ in range(2)] + [np.zeros(64, dtype=np.int32) for _ in range(3)]
    st = M._lib.mlvs_umesh_geometry(len(xy), xy.ctypes.data, len(cells), ptr.ctypes.data, cn.ctypes.data, 3,
                                    C.byref(nf), bufs[0].ctypes.data, bufs[2].ctypes.data, bufs[3].ctypes.data,
                                    bufs[4].ctypes.data, bufs[1].ctypes.data)
    assert st == ERR_ARG and nf.value == 12


# -- Hilbert order ----------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_hilbert_order_walks_a_power_of_two_grid_through_edge_neighbours(k):
    """On a 2^k x 2^k grid of unit cells the Hilbert curve visits every cell once, each next
    cell sharing an edge with the last (the curve's defining property), from a corner."""
    n = 2 ** k
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    perm = np.random.default_rng(k).permutation(n * n)
    cx, cy = (i.ravel() + 0.5)[perm], (j.ravel() + 0.5)[perm]
    order = M.mlvs_umesh_order(cx, cy)
    assert sorted(order) == list(range(n * n))
    steps = np.abs(np.diff(cx[order])) + np.abs(np.diff(cy[order]))
    np.testing.assert_array_equal(steps, 1.0)
    assert (cx[order[0]], cy[order[0]]) == (0.5, 0.5)


def test_hilbert_order_keeps_a_two_cavity_mesh_local():
    """17,408 triangles: consecutive cells are neighbours on average, and a block of 256
    consecutive cells spans about a square of 256 cells (a row-major block of the same size
    spans a strip across a cavity, and grows with the mesh)."""
    nodes, cells = workloads.triangulate(*workloads.two_cavities(8))
    g = M.mlvs_umesh_geometry(nodes, cells)
    order = M.mlvs_umesh_order(g["cx"], g["cy"])
    assert sorted(order) == list(range(len(cells)))
    h = np.sqrt(np.mean(g["area"]))
    assert np.mean(np.hypot(np.diff(g["cx"][order]), np.diff(g["cy"][order]))) < 2.0 * h

    def span(o):
        return np.median([np.ptp(g["cx"][o[b:b + 256]]) + np.ptp(g["cy"][o[b:b + 256]])
                          for b in range(0, len(o) - 256, 256)])

    assert span(order) < 48 * h
    assert span(order) < 0.6 * span(np.arange(len(cells)))
