"""The paper's workload index and runtime model of the multi-level organisation.

Sec. 3.5, Eq. composite_workload_index: I = r + lambda_cross f + lambda_upd N_upd^eq / N_cell,
with r = mean velocity points per cell / N_xi^UVS and f = N_cross / N_int (Eq.
normalized_performance_quantities).  Sec. 4.6, Eq. empirical_runtime_model: with the mesh,
the GPU and the adaptation interval fixed, t / t_UVS ~ r + lambda_cross f + c; the coefficient
of r is held at one and (lambda_cross, c) are fitted by least squares over a threshold sweep
(Eq. calibrated_runtime_model).  Eq. multilevel_runtime_criterion: a multi-level set beats
the single global adaptive space when f < (r_global - r) / lambda_cross.
"""
from __future__ import annotations

import numpy as np


def fit(r, f, t_rel):
    """Least-squares (lambda_cross, c) of t_rel - r = lambda_cross f + c.  Returns a dict with
    lambda_cross, c, r2 (coefficient of determination of the fitted part t_rel - r) and the
    model's t_rel per sample."""
    r, f, t_rel = (np.asarray(x, dtype=np.float64) for x in (r, f, t_rel))
    y = t_rel - r
    A = np.stack([f, np.ones_like(f)], axis=1)
    (lam, c), *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - (lam * f + c)
    tot = y - y.mean()
    r2 = 1.0 - float(res @ res) / float(tot @ tot) if float(tot @ tot) > 0 else float("nan")
    return {"lambda_cross": float(lam), "c": float(c), "r2": r2, "t_rel_model": r + lam * f + c}


def breakeven_cross_fraction(r_global, r, lambda_cross):
    """Largest cross-level face fraction at which a multi-level set with mean size r still
    beats the global adaptive space of mean size r_global."""
    return (r_global - r) / lambda_cross


def workload_index(r, f, lambda_cross, upd_fraction=0.0, lambda_upd=1.0):
    """I = r + lambda_cross f + lambda_upd (N_upd^eq / N_cell)."""
    return r + lambda_cross * f + lambda_upd * upd_fraction
