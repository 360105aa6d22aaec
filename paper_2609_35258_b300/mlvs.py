"""Thin ctypes binding of the C ABI in include/mlvs.h (argument marshalling only).

Every step of the solver runs in libmlvs.so.  If the library is missing the import fails;
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmlvs.so")

MLVS_OK = 0
STATUS = {0: "MLVS_OK", -1: "MLVS_ERR_ARG", -2: "MLVS_ERR_OOM", -3: "MLVS_ERR_CUDA",
          -4: "MLVS_ERR_NONFINITE", -5: "MLVS_ERR_POSITIVITY", -6: "MLVS_ERR_SINGULAR",
          -7: "MLVS_ERR_TIMEOUT", -8: "MLVS_ERR_STATE"}
BC_PERIODIC, BC_ZEROGRAD, BC_WALL, BC_FREESTREAM = 0, 1, 2, 3
F64, F32, BF16 = 0, 1, 2
QUAD_BOOLE, QUAD_SIMPSON, QUAD_TRAPZ = 0, 1, 2
LIMITER_VANLEER, LIMITER_NONE, LIMITER_VENKAT = 0, 1, 2
RHO, U, V, T, QX, QY, LEVEL, RHOE, SXX, SXY, SYY = 1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024


class mlvs_config(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n_instances", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("Lx", C.c_double), ("Ly", C.c_double), ("bc", C.c_int * 4),
        ("wall", (C.c_double * 3) * 4), ("R", C.c_double), ("K_internal", C.c_double),
        ("Pr", C.c_double), ("omega", C.c_double), ("Kn", C.c_double), ("mu_ref", C.c_double),
        ("L_ref", C.c_double), ("T_ref", C.c_double), ("rho_ref", C.c_double),
        ("cfl", C.c_double), ("dt", C.c_double), ("storage", C.c_int), ("compat_cell", C.c_int),
        ("compat_face", C.c_int), ("limiter", C.c_int), ("init_W", C.POINTER(C.c_double)),
        ("stream", C.c_void_p), ("far", C.c_double * 4), ("mesh_kind", C.c_int),
        ("node_xy", C.POINTER(C.c_double)), ("positive_mapping", C.c_int), ("map_moments", C.c_int),
        ("compat_moments", C.c_int),
    ]


class mlvs_level_desc(C.Structure):
    _fields_ = [("uniform_L", C.c_int), ("kappa", C.POINTER(C.c_ubyte))]


class mlvs_step_stats(C.Structure):
    _fields_ = [("profile", C.c_int), ("dt", C.c_double), ("cell_velocity_updates", C.c_longlong),
                ("n_levels", C.c_int), ("launches", C.c_int), ("ms_total", C.c_float),
                ("ms_phase", C.c_float * 6)]


class mlvs_adapt_params(C.Structure):
    _fields_ = [("C_split", C.c_double), ("C_merge", C.c_double), ("eps_merge", C.c_double),
                ("tau_clust", C.c_double), ("max_level", C.c_int)]


class mlvs_adapt_stats(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_distinct", C.c_int), ("n_changed", C.c_int),
                ("updates_per_step", C.c_longlong), ("ms_criterion", C.c_float),
                ("ms_group", C.c_float), ("ms_remap", C.c_float), ("ms_total", C.c_float),
                ("n_interior_faces", C.c_int), ("n_cross_faces", C.c_int),
                ("n_exp_corrected", C.c_int), ("n_exp_failed", C.c_int)]


class mlvs_uconfig(C.Structure):
    _fields_ = [
        ("storage", C.c_int), ("R", C.c_double), ("K_internal", C.c_double), ("Pr", C.c_double),
        ("omega", C.c_double), ("mu_ref", C.c_double), ("T_ref", C.c_double), ("Kn", C.c_double),
        ("cfl", C.c_double),
        ("dt", C.c_double), ("compat_cell", C.c_int), ("compat_face", C.c_int), ("limiter", C.c_int),
        ("compat_moments", C.c_int), ("n_base", C.c_int), ("umin", C.c_double), ("umax", C.c_double),
        ("quadrature", C.c_int),
        ("n_wall", C.c_int), ("wall", (C.c_double * 3) * 8), ("vpc", C.c_int), ("stream", C.c_void_p),
    ]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libmlvs.so not built at {_LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(_LIB_PATH)
    H = C.c_void_p
    sig = {
        "mlvs_create": (C.c_int, [C.POINTER(mlvs_config), C.POINTER(H)]),
        "mlvs_set_velocity_levels": (C.c_int, [H, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                               C.POINTER(mlvs_level_desc), C.c_int]),
        "mlvs_step": (C.c_int, [H, C.c_int, C.POINTER(mlvs_step_stats)]),
        "mlvs_moments": (C.c_int, [H, C.c_int, C.c_uint, C.c_void_p, C.c_int]),
        "mlvs_read_cells": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
        "mlvs_time_step": (C.c_int, [H, C.POINTER(C.c_double)]),
        "mlvs_set_cell_levels": (C.c_int, [H, C.c_int, C.POINTER(C.c_int)]),
        "mlvs_level_info": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]),
        "mlvs_moments_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "mlvs_criterion": (C.c_int, [H, C.c_int, C.POINTER(mlvs_adapt_params), C.c_void_p, C.c_int]),
        "mlvs_adapt": (C.c_int, [H, C.POINTER(mlvs_adapt_params), C.POINTER(mlvs_adapt_stats)]),
        "mlvs_set_adaptation": (C.c_int, [H, C.POINTER(mlvs_adapt_params), C.c_int]),
        "mlvs_cluster": (C.c_int, [C.c_void_p, C.c_long, C.c_int, C.c_double, C.POINTER(C.c_int),
                                   C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
        "mlvs_level_kappa": (C.c_int, [H, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
        "mlvs_mesh_geometry": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]),
        "mlvs_umesh_geometry": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                          C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
        "mlvs_umesh_order": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
        "mlvs_ucreate": (C.c_int, [C.POINTER(mlvs_uconfig), C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(H)]),
        "mlvs_ustep": (C.c_int, [H, C.c_int, C.POINTER(C.c_float)]),
        "mlvs_uread": (C.c_int, [H, C.c_void_p, C.c_void_p]),
        "mlvs_ucells": (C.c_int, [H, C.c_void_p]),
        "mlvs_uinfo": (C.c_int, [H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "mlvs_udestroy": (None, [H]),
        "mlvs_space_points": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_int,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]),
        "mlvs_set_graph": (C.c_int, [H, C.c_int]),
        "mlvs_step_many": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.POINTER(mlvs_step_stats)]),
        "mlvs_autotune": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.c_void_p]),
        "mlvs_set_tuning": (C.c_int, [H, C.c_int]),
        "mlvs_mlp_create": (C.c_int, [C.c_void_p, C.POINTER(H)]),
        "mlvs_mlp_destroy": (None, [H]),
        "mlvs_mlp_set_weights": (C.c_int, [H, C.c_void_p, C.c_int]),
        "mlvs_mlp_get_weights": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_int]),
        "mlvs_mlp_forward": (C.c_int, [H, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
        "mlvs_mlp_gradient": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_float)]),
        "mlvs_mlp_train_step": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_float,
                                          C.POINTER(C.c_float)]),
        "mlvs_features": (C.c_int, [H, C.c_int, C.c_void_p, C.c_int]),
        "mlvs_criterion_levels": (C.c_int, [H, C.c_int, C.POINTER(mlvs_adapt_params), C.c_void_p]),
        "mlvs_adapt_mlp": (C.c_int, [H, H, C.POINTER(mlvs_adapt_params), C.c_float, C.POINTER(mlvs_adapt_stats)]),
        "mlvs_destroy": (None, [H]),
        "mlvs_last_error": (C.c_char_p, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("mlvs_create", "mlvs_set_velocity_levels", "mlvs_step", "mlvs_moments",
            "mlvs_read_cells", "mlvs_time_step", "mlvs_destroy", "mlvs_last_error")


class MLVSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, h):
    if st != MLVS_OK:
        msg = _lib.mlvs_last_error(h)
        raise MLVSError(st, msg.decode() if msg else "")


def mlvs_create(cfg: mlvs_config):
    h = C.c_void_p()
    _check(_lib.mlvs_create(C.byref(cfg), C.byref(h)), None)
    return h


def mlvs_set_velocity_levels(h, n_base, umin, umax, quadrature, levels, adaptive=0):
    arr = (mlvs_level_desc * len(levels))()
    keep = []
    for i, L in enumerate(levels):
        if isinstance(L, int):
            arr[i].uniform_L = L
            arr[i].kappa = None
        else:
            k = np.ascontiguousarray(L, dtype=np.uint8)
            keep.append(k)
            arr[i].uniform_L = -1
            arr[i].kappa = k.ctypes.data_as(C.POINTER(C.c_ubyte))
    _check(_lib.mlvs_set_velocity_levels(h, n_base, umin, umax, quadrature, len(levels), arr, adaptive), h)


def mlvs_step(h, n_steps=1, profile=False):
    st = mlvs_step_stats()
    st.profile = 1 if profile else 0
    _check(_lib.mlvs_step(h, n_steps, C.byref(st)), h)
    return st


def mlvs_moments(h, instance, fields, ncell, out=None):
    """Moments as a numpy [n_fields][ncell] array, or into a torch CUDA tensor `out`."""
    nf = bin(fields).count("1")
    if out is None:
        res = np.zeros((nf, ncell))
        _check(_lib.mlvs_moments(h, instance, fields, res.ctypes.data, 0), h)
        return res
    _check(_lib.mlvs_moments(h, instance, fields, C.c_void_p(out.data_ptr()), 1), h)
    return out


def mlvs_read_cells(h, instance, cell0, ncells, nv_cap):
    g = np.zeros(ncells * nv_cap)
    hh = np.zeros(ncells * nv_cap)
    nv = C.c_int()
    _check(_lib.mlvs_read_cells(h, instance, cell0, ncells, g.ctypes.data_as(C.POINTER(C.c_double)),
                                hh.ctypes.data_as(C.POINTER(C.c_double)), ncells * nv_cap,
                                C.byref(nv)), h)
    n = nv.value
    return g[: ncells * n].reshape(ncells, n), hh[: ncells * n].reshape(ncells, n)


def mlvs_time_step(h):
    dt = C.c_double()
    _check(_lib.mlvs_time_step(h, C.byref(dt)), h)
    return dt.value


def mlvs_moments_noalloc(g, h, nv, ncell, xi_x, xi_y, w_x, w_y, out, stream=None):
    """Allocation-free moments: every argument is a device pointer (int) or a tensor with
    data_ptr(); see include/mlvs.h for layouts."""
    def ptr(x):
        return C.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else x)
    _check(_lib.mlvs_moments_noalloc(ptr(g), ptr(h), nv, ncell, ptr(xi_x), ptr(xi_y), ptr(w_x),
                                     ptr(w_y), ptr(out), C.c_void_p(stream)), None)


def mlvs_set_cell_levels(h, instance, levels):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    _check(_lib.mlvs_set_cell_levels(h, instance, lv.ctypes.data_as(C.POINTER(C.c_int))), h)


def mlvs_level_info(h, level):
    nv = C.c_int()
    _check(_lib.mlvs_level_info(h, level, C.byref(nv), None, None, None, 0), h)
    n = nv.value
    x, y, w = np.zeros(n), np.zeros(n), np.zeros(n)
    P = C.POINTER(C.c_double)
    _check(_lib.mlvs_level_info(h, level, C.byref(nv), x.ctypes.data_as(P), y.ctypes.data_as(P),
                                w.ctypes.data_as(P), n), h)
    return x, y, w


def adapt_params(C_split, C_merge, eps_merge=0.0, tau_clust=0.05, max_level=3):
    return mlvs_adapt_params(C_split, C_merge, eps_merge, tau_clust, max_level)


def mlvs_level_kappa(h, level):
    nb = C.c_int()
    _check(_lib.mlvs_level_kappa(h, level, None, 0, C.byref(nb)), h)
    out = np.zeros(nb.value, dtype=np.uint8)
    _check(_lib.mlvs_level_kappa(h, level, out.ctypes.data, nb.value, C.byref(nb)), h)
    return out


def mlvs_criterion(h, instance, params, ncell, nb):
    """Masks [ncell][nb] (uint8) of the criterion for every cell of one instance."""
    out = np.zeros((ncell, nb), dtype=np.uint8)
    _check(_lib.mlvs_criterion(h, instance, C.byref(params), out.ctypes.data, 0), h)
    return out


def mlvs_adapt(h, params):
    st = mlvs_adapt_stats()
    _check(_lib.mlvs_adapt(h, C.byref(params), C.byref(st)), h)
    return st


def mlvs_set_adaptation(h, params, interval):
    _check(_lib.mlvs_set_adaptation(h, C.byref(params) if params is not None else None, interval), h)


def mlvs_cluster(kappa, tau):
    """Host grouping of masks [nrow][nb]: (labels [nrow], reps [ncluster][nb])."""
    k = np.ascontiguousarray(kappa, dtype=np.uint8)
    nrow, nb = k.shape
    labels = np.zeros(nrow, dtype=np.int32)
    cap = max(nrow, 1)
    reps = np.zeros((cap, nb), dtype=np.uint8)
    n = C.c_int()
    _check(_lib.mlvs_cluster(k.ctypes.data, nrow, nb, tau, labels.ctypes.data_as(C.POINTER(C.c_int)),
                             reps.ctypes.data, cap, C.byref(n)), None)
    return labels, reps[: n.value].copy()


def mlvs_mesh_geometry(node_xy, periodic_x, periodic_y):
    """Host-only: (cell_geo [5][nc], face_geo [7][nface], width [nc]) of a node grid
    node_xy [ny+1][nx+1][2], as a curvilinear handle builds it."""
    xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    ny, nx = xy.shape[0] - 1, xy.shape[1] - 1
    nfx = nx if periodic_x else nx + 1
    nfy = ny if periodic_y else ny + 1
    nc, nface = nx * ny, nfx * ny + nx * nfy
    cg, fg, wd = np.zeros((5, nc)), np.zeros((7, nface)), np.zeros(nc)
    _check(_lib.mlvs_mesh_geometry(nx, ny, int(bool(periodic_x)), int(bool(periodic_y)), xy.ctypes.data,
                                   cg.ctypes.data, fg.ctypes.data, wd.ctypes.data), None)
    return cg, fg, wd


def mlvs_umesh_geometry(node_xy, cells):
    """Host-only: geometry of an unstructured mesh (nodes [Nn][2], cells as counter-clockwise
    node lists) as a dict: cell rows area, cx, cy, width, mxx, mxy, myy (inverse least-squares
    normal matrix); cell_ptr, cell_face (f, or -f - 1 where the cell is R); per face L, R, n0,
    n1, nx, ny, length, midx, midy."""
    xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    ptr = np.zeros(len(cells) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(c) for c in cells])
    nodes = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in cells]))
    nc = len(cells)
    nf = C.c_int()
    args = (xy.shape[0], xy.ctypes.data, nc, ptr.ctypes.data, nodes.ctypes.data)
    _check(_lib.mlvs_umesh_geometry(*args, 0, C.byref(nf), None, None, None, None, None), None)
    m = nf.value
    cg, cf = np.zeros((7, nc)), np.zeros(int(ptr[-1]), dtype=np.int32)
    fc, fnd, fg = np.zeros((2, m), dtype=np.int32), np.zeros((2, m), dtype=np.int32), np.zeros((5, m))
    _check(_lib.mlvs_umesh_geometry(*args, m, C.byref(nf), cg.ctypes.data, cf.ctypes.data, fc.ctypes.data,
                                    fnd.ctypes.data, fg.ctypes.data), None)
    out = dict(zip(("area", "cx", "cy", "width", "mxx", "mxy", "myy"), cg))
    out.update(cell_ptr=ptr, cell_face=cf, L=fc[0], R=fc[1], n0=fnd[0], n1=fnd[1])
    out.update(zip(("nx", "ny", "length", "midx", "midy"), fg))
    return out


def mlvs_umesh_order(cx, cy):
    """Host-only: the cells in the order of a Hilbert curve through their centroids."""
    x = np.ascontiguousarray(cx, dtype=np.float64)
    y = np.ascontiguousarray(cy, dtype=np.float64)
    order = np.zeros(x.size, dtype=np.int32)
    _check(_lib.mlvs_umesh_order(x.size, x.ctypes.data, y.ctypes.data, order.ctypes.data), None)
    return order


def umesh_arrays(cells, edge_wall=None):
    """CSR (cell_ptr, cell_nodes) of a list of node tuples, and edge_wall flattened alike."""
    ptr = np.zeros(len(cells) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(c) for c in cells])
    nodes = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in cells]))
    ew = None
    if edge_wall is not None:
        ew = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.int32) for e in edge_wall]))
        if ew.size != nodes.size:
            raise ValueError("edge_wall needs one entry per cell edge")
    return ptr, nodes, ew


def mlvs_ucreate(cfg: mlvs_uconfig, node_xy, cells, init_W, edge_wall=None):
    """Unstructured handle: nodes [Nn][2], counter-clockwise cells (node tuples), init_W [Nc][4]
    = (rho, u, v, T), edge_wall per cell edge (None: wall 0 everywhere)."""
    xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    ptr, nodes, ew = umesh_arrays(cells, edge_wall)
    W0 = np.ascontiguousarray(init_W, dtype=np.float64)
    if W0.shape != (len(cells), 4):
        raise ValueError("init_W must be [n_cell][4]")
    h = C.c_void_p()
    _check(_lib.mlvs_ucreate(C.byref(cfg), xy.shape[0], xy.ctypes.data, len(cells), ptr.ctypes.data,
                             nodes.ctypes.data, None if ew is None else ew.ctypes.data, W0.ctypes.data,
                             C.byref(h)), None)
    return h


def mlvs_ustep(h, n_steps):
    """Advance n_steps steps; returns their device time in ms."""
    ms = C.c_float()
    _check(_lib.mlvs_ustep(h, n_steps, C.byref(ms)), None)
    return ms.value


def mlvs_uinfo(h):
    """(nv, n_face, dt) of an unstructured handle."""
    nv, nf, dt = C.c_int(), C.c_int(), C.c_double()
    _check(_lib.mlvs_uinfo(h, C.byref(nv), C.byref(nf), C.byref(dt)), None)
    return nv.value, nf.value, dt.value


def mlvs_uread(h, n_cell):
    """(g~, h~) as [n_cell][nv] FP64 arrays."""
    nv = mlvs_uinfo(h)[0]
    g, hh = np.zeros((n_cell, nv)), np.zeros((n_cell, nv))
    _check(_lib.mlvs_uread(h, g.ctypes.data, hh.ctypes.data), None)
    return g, hh


def mlvs_ucells(h, n_cell):
    """Cell state [11][n_cell] at the start of the last step (rho, u, v, T, qx, qy, rhoE, tau,
    sxx, sxy, syy)."""
    W = np.zeros((11, n_cell))
    _check(_lib.mlvs_ucells(h, W.ctypes.data), None)
    return W


def mlvs_udestroy(h):
    _lib.mlvs_udestroy(h)


def mlvs_space_points(n_base, umin, umax, quadrature, kappa):
    """Host-only: points (xi_x, xi_y) and weights of the space of a level-1 coarsening mask
    (made parent-child consistent first), as the library builds it."""
    k = np.ascontiguousarray(kappa, dtype=np.uint8).ravel()
    nv, n1 = C.c_int(), C.c_int()
    _check(_lib.mlvs_space_points(n_base, umin, umax, quadrature, k.ctypes.data, k.size, None, None, None, 0,
                                  C.byref(nv), C.byref(n1)), None)
    x, y, w = np.zeros(nv.value), np.zeros(nv.value), np.zeros(nv.value)
    _check(_lib.mlvs_space_points(n_base, umin, umax, quadrature, k.ctypes.data, k.size, x.ctypes.data,
                                  y.ctypes.data, w.ctypes.data, nv.value, C.byref(nv), C.byref(n1)), None)
    return x, y, w


def mlvs_set_graph(h, on=True):
    _check(_lib.mlvs_set_graph(h, 1 if on else 0), h)


def mlvs_step_many(handles, n_steps=1, use_graph=True):
    arr = (C.c_void_p * len(handles))(*[x.value for x in handles])
    st = mlvs_step_stats()
    _check(_lib.mlvs_step_many(arr, len(handles), n_steps, 1 if use_graph else 0, C.byref(st)), None)
    return st


def mlvs_autotune(h, steps=3):
    """(cta_target, ms per step of every candidate [7])"""
    t = C.c_int()
    table = np.zeros(7, dtype=np.float32)
    _check(_lib.mlvs_autotune(h, steps, C.byref(t), table.ctypes.data), h)
    return t.value, table


def mlvs_set_tuning(h, cta_target):
    _check(_lib.mlvs_set_tuning(h, cta_target), h)


N_SELECTOR_PARAMS = 5124


def _dptr(x):
    return C.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else x)


def mlvs_mlp_create(stream=None):
    m = C.c_void_p()
    _check(_lib.mlvs_mlp_create(stream, C.byref(m)), None)
    return m


def mlvs_mlp_destroy(m):
    _lib.mlvs_mlp_destroy(m)


def mlvs_mlp_set_weights(m, w):
    a = np.ascontiguousarray(w, dtype=np.float32)
    _check(_lib.mlvs_mlp_set_weights(m, a.ctypes.data, a.size), None)


def mlvs_mlp_get_weights(m):
    """(FP32 master weights, the BF16 weights as floats)"""
    master = np.zeros(N_SELECTOR_PARAMS, dtype=np.float32)
    b = np.zeros(N_SELECTOR_PARAMS, dtype=np.float32)
    _check(_lib.mlvs_mlp_get_weights(m, master.ctypes.data, b.ctypes.data, N_SELECTOR_PARAMS), None)
    return master, b


def mlvs_mlp_forward(m, X, n, logits=None, prob=None):
    """Device tensors: X [n][10] float32 -> logits / prob [n][4] float32 (asynchronous)."""
    _check(_lib.mlvs_mlp_forward(m, _dptr(X), n, _dptr(logits) if logits is not None else None,
                                 _dptr(prob) if prob is not None else None), None)


def mlvs_mlp_gradient(m, X, y, n, grad):
    loss = C.c_float()
    _check(_lib.mlvs_mlp_gradient(m, _dptr(X), _dptr(y), n, _dptr(grad), C.byref(loss)), None)
    return loss.value


def mlvs_mlp_train_step(m, X, y, n, lr, momentum=0.9):
    loss = C.c_float()
    _check(_lib.mlvs_mlp_train_step(m, _dptr(X), _dptr(y), n, lr, momentum, C.byref(loss)), None)
    return loss.value


def mlvs_features(h, instance, ncell):
    out = np.zeros((ncell, 10), dtype=np.float32)
    _check(_lib.mlvs_features(h, instance, out.ctypes.data, 0), h)
    return out


def mlvs_criterion_levels(h, instance, params, ncell):
    out = np.zeros(ncell, dtype=np.int32)
    _check(_lib.mlvs_criterion_levels(h, instance, C.byref(params), out.ctypes.data), h)
    return out


def mlvs_adapt_mlp(h, m, params, confidence):
    st = mlvs_adapt_stats()
    _check(_lib.mlvs_adapt_mlp(h, m, C.byref(params), confidence, C.byref(st)), h)
    return st


def mlvs_destroy(h):
    _lib.mlvs_destroy(h)


def mlvs_last_error(h=None):
    m = _lib.mlvs_last_error(h)
    return m.decode() if m else ""


def make_config(*, dim, nx, ny, Lx, Ly, bc, init_W, wall=((0, 0, 1),) * 4, R=1.0, K=0.0,
                Pr=2.0 / 3.0, omega=0.81, Kn=0.0, mu_ref=0.0, cfl=0.5, dt=0.0, storage=F32,
                compat_cell=1, compat_face=1, limiter=LIMITER_VANLEER, n_instances=1,
                stream=None, T_ref=1.0, L_ref=1.0, rho_ref=1.0, far=(1.0, 0.0, 0.0, 1.0), nodes=None,
                positive_mapping=0, map_moments=4, compat_moments=4):
    """Fill an mlvs_config.  init_W: float64 array [n_instances][ny][nx][4].  The returned
    config keeps a reference to init_W (attribute `_keep`)."""
    cfg = mlvs_config()
    cfg.dim, cfg.n_instances, cfg.nx, cfg.ny = dim, n_instances, nx, ny
    cfg.Lx, cfg.Ly = Lx, Ly
    for i in range(4):
        cfg.bc[i] = bc[i]
        for j in range(3):
            cfg.wall[i][j] = wall[i][j]
    cfg.R, cfg.K_internal, cfg.Pr, cfg.omega = R, K, Pr, omega
    cfg.Kn, cfg.mu_ref, cfg.L_ref, cfg.T_ref, cfg.rho_ref = Kn, mu_ref, L_ref, T_ref, rho_ref
    cfg.cfl, cfg.dt, cfg.storage = cfl, dt, storage
    cfg.compat_cell, cfg.compat_face, cfg.limiter = compat_cell, compat_face, limiter
    cfg.positive_mapping = positive_mapping
    cfg.map_moments = map_moments
    cfg.compat_moments = compat_moments
    W = np.ascontiguousarray(init_W, dtype=np.float64)
    cfg._keep = W
    cfg.init_W = W.ctypes.data_as(C.POINTER(C.c_double))
    cfg.stream = stream
    for j in range(4):
        cfg.far[j] = far[j]
    if nodes is not None:
        xy = np.ascontiguousarray(nodes, dtype=np.float64)    # [ny+1][nx+1][2]
        cfg._keep_nodes = xy
        cfg.mesh_kind = 1
        cfg.node_xy = xy.ctypes.data_as(C.POINTER(C.c_double))
    return cfg
