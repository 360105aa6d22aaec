"""Argument checks of the unstructured-mesh handle, on CPU: every defect of the mesh, the
configuration or the initial state is reported as MLVS_ERR_ARG before any device work, so
these run without a GPU."""
import numpy as np
import pytest

from paper_2609_35258_b300 import mlvs as M
from paper_2609_35258_b300 import workloads
from tests import test_ustep_emu as E

ERR_ARG = next(k for k, v in M.STATUS.items() if v == "MLVS_ERR_ARG")


def _mesh():
    nodes, cells = workloads.quad_mesh(np.linspace(0, 1, 4), np.linspace(0, 1, 4))
    W0 = np.tile([1.0, 0.0, 0.0, 1.0], (len(cells), 1))
    return nodes, cells, W0


def _expect_arg(cfg, nodes, cells, W0, edge_wall=None):
    with pytest.raises(M.MLVSError) as e:
        M.mlvs_ucreate(cfg, nodes, cells, W0, edge_wall)
    assert e.value.status == ERR_ARG, str(e.value)


def _good():
    return E._cfg(M.F64, [(0.0, 0.0, 1.0), (0.3, 0.0, 1.0)])


@pytest.mark.parametrize("field,value", [
    ("storage", M.BF16), ("storage", 7), ("limiter", M.LIMITER_VANLEER), ("compat_moments", 6),
    ("n_base", 12), ("n_base", 11), ("quadrature", 5), ("n_wall", 0), ("n_wall", 9), ("Pr", 0.0),
    ("R", -1.0), ("T_ref", 0.0), ("vpc", -3)])
def test_bad_configuration(field, value):
    nodes, cells, W0 = _mesh()
    cfg = _good()
    setattr(cfg, field, value)
    _expect_arg(cfg, nodes, cells, W0)


def test_no_viscosity_given():
    nodes, cells, W0 = _mesh()
    cfg = _good()
    cfg.mu_ref, cfg.Kn = 0.0, 0.0
    _expect_arg(cfg, nodes, cells, W0)


def test_bad_velocity_range_and_wall_temperature():
    nodes, cells, W0 = _mesh()
    cfg = _good()
    cfg.umin, cfg.umax = 2.0, 1.0
    _expect_arg(cfg, nodes, cells, W0)
    cfg = _good()
    cfg.wall[1][2] = 0.0
    _expect_arg(cfg, nodes, cells, W0)


def test_bad_mesh_and_initial_state():
    nodes, cells, W0 = _mesh()
    _expect_arg(_good(), nodes, [tuple(reversed(cells[0]))] + list(cells[1:]), W0)   # clockwise cell
    bad = W0.copy()
    bad[3, 0] = 0.0
    _expect_arg(_good(), nodes, cells, bad)                                           # rho = 0
    bad = W0.copy()
    bad[2, 3] = np.nan
    _expect_arg(_good(), nodes, cells, bad)                                           # T not finite
    with pytest.raises(ValueError):
        M.mlvs_ucreate(_good(), nodes, cells, W0[:-1])                               # wrong shape


def test_boundary_edge_naming_no_wall():
    nodes, cells, W0 = _mesh()
    edge_wall = [[0, 0, 0, 0] for _ in cells]
    edge_wall[0][0] = 2                                   # cell 0's bottom edge: only walls 0, 1 exist
    _expect_arg(_good(), nodes, cells, W0, edge_wall)
    edge_wall[0][0] = 0
    edge_wall[4][1] = 5                                   # an interior edge: ignored, so no error here
    cfg = _good()
    cfg.n_base = 4                                        # ... but the even base size is reported
    _expect_arg(cfg, nodes, cells, W0, edge_wall)
