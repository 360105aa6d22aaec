"""Checks of the synthetic input generators that build meshes (no kinetic arithmetic)."""
import numpy as np
import pytest

from paper_2609_35258_b300 import workloads


@pytest.mark.parametrize("m,tri", [(2, False), (4, False), (2, True)])
def test_two_cavity_mesh_is_conforming_and_closed(m, tri):
    nodes, cells = workloads.two_cavities(m)
    if tri:
        nodes, cells = workloads.triangulate(nodes, cells)
    h = 0.125 / m
    area, edges = 0.0, {}
    for poly in cells:
        P = nodes[list(poly)]
        Q = np.roll(P, -1, axis=0)
        a = 0.5 * np.sum(P[:, 0] * Q[:, 1] - Q[:, 0] * P[:, 1])
        assert a > 0.0                                          # counter-clockwise
        area += a
        for k in range(len(poly)):
            e = tuple(sorted((poly[k], poly[(k + 1) % len(poly)])))
            edges[e] = edges.get(e, 0) + 1
    assert abs(area - (2.0 + 1.0 * 0.125)) < 1e-12
    assert max(edges.values()) == 2                             # no edge shared by three cells
    boundary = [e for e, n in edges.items() if n == 1]
    perimeter = sum(np.hypot(*(nodes[a] - nodes[b])) for a, b in boundary)
    # two squares of side 1 and the channel's two long walls, minus the channel mouths
    assert abs(perimeter - (2 * 4.0 - 2 * 0.125 + 2 * 1.0)) < 1e-12
    assert len(np.unique(np.round(nodes / h).astype(np.int64), axis=0)) == len(nodes)   # no duplicate nodes


def test_two_cavity_cell_count_near_the_paper():
    _, cells = workloads.two_cavities(10)
    assert len(cells) == 13600                                  # the paper's mesh has 12,012 cells
    with pytest.raises(ValueError):
        workloads.two_cavities(3)


def test_cylinder_smooth_start():
    """The smooth start keeps the freestream's pressure (rho T = 1) and total enthalpy
    (T + u^2/5 for gamma = 5/3, R = 1) in every cell, is near rest at the wall and is the
    freestream far from it."""
    d = workloads.cylinder(64, 32, start="ramp")
    W = d["init"]
    u_inf = 5.0 * np.sqrt(5.0 / 3.0)
    assert np.allclose(W[..., 0] * W[..., 3], 1.0, rtol=1e-14)
    assert np.allclose(W[..., 3] + W[..., 1] ** 2 / 5.0, 1.0 + u_inf ** 2 / 5.0, rtol=1e-14)
    assert np.all(W[..., 2] == 0.0)
    assert np.all(W[0, :, 1] < 0.01 * u_inf) and np.allclose(W[-1, :, 1], u_inf, rtol=1e-12)
    assert np.all(np.diff(W[..., 1], axis=0) > 0.0)            # speed rises with the radius
    imp = workloads.cylinder(64, 32)["init"]
    assert np.all(imp[..., 1] == u_inf) and np.all(imp[..., 0] == 1.0)
    with pytest.raises(ValueError):
        workloads.cylinder(64, 32, start="nope")
