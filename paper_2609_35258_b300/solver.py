"""Convenience wrapper: a workload description -> one library handle (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import mlvs as M

_BC = {"periodic": M.BC_PERIODIC, "zerograd": M.BC_ZEROGRAD, "wall": M.BC_WALL,
       "freestream": M.BC_FREESTREAM}
_ST = {"f64": M.F64, "f32": M.F32, "bf16": M.BF16}
_RULE = {"boole": M.QUAD_BOOLE, "simpson": M.QUAD_SIMPSON, "trapz": M.QUAD_TRAPZ}
_LIM = {"vanleer": M.LIMITER_VANLEER, "none": M.LIMITER_NONE}


class Solver:
    def __init__(self, desc, levels=(0,), stream=None, storage=None, compat_cell=1, compat_face=1,
                 n_instances=1, init=None, adaptive=0, positive_mapping=0, map_moments=4, compat_moments=4):
        d = desc
        self.desc = d
        self.ncell = d["nx"] * d["ny"]
        init = d["init"] if init is None else init
        # init: [ny][nx][4] for every instance, or [n_instances][ny][nx][4]
        W = (np.ascontiguousarray(init) if init.ndim == 4
             else np.broadcast_to(init, (n_instances,) + init.shape).copy())
        if W.shape[0] != n_instances:
            raise ValueError("init has the wrong number of instances")
        self.cfg = M.make_config(
            dim=d["dim"], nx=d["nx"], ny=d["ny"], Lx=d["Lx"], Ly=d["Ly"],
            bc=[_BC[b] for b in d["bc"]], wall=d["wall"], init_W=W, R=d["R"], K=d["K"], Pr=d["Pr"],
            omega=d["omega"], Kn=d["Kn"] or 0.0, mu_ref=d["mu_ref"] or 0.0, cfl=d["cfl"],
            storage=_ST[storage or d["storage"]], compat_cell=compat_cell, compat_face=compat_face,
            limiter=_LIM[d["limiter"]], n_instances=n_instances, stream=stream,
            far=d.get("far", (1.0, 0.0, 0.0, 1.0)), nodes=d.get("nodes"), positive_mapping=positive_mapping,
            map_moments=map_moments, compat_moments=compat_moments)
        self.h = M.mlvs_create(self.cfg)
        M.mlvs_set_velocity_levels(self.h, d["n_base"], d["umin"], d["umax"], _RULE[d["rule"]],
                                   list(levels), adaptive)
        self.dt = M.mlvs_time_step(self.h)

    def step(self, n=1, profile=False):
        return M.mlvs_step(self.h, n, profile)

    def moments(self, fields=M.RHO | M.U | M.V | M.T | M.QX | M.QY | M.RHOE, instance=0):
        return M.mlvs_moments(self.h, instance, fields, self.ncell)

    def read_cells(self, cell0, ncells, nv_cap, instance=0):
        return M.mlvs_read_cells(self.h, instance, cell0, ncells, nv_cap)

    def close(self):
        if self.h:
            M.mlvs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
