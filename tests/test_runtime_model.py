"""The runtime model of the multi-level organisation against the paper's own calibration
(Sec. 4.6, Table threshold_performance, tests/golden/threshold_runtime_model.json): fitted to
the printed sweep, the model gives the printed lambda_cross, c and R^2, the printed model
times and fitting errors, and the printed break-even cross-level fraction for tau 0.05."""
import json
import os

import numpy as np

from paper_2609_35258_b300 import runtime_model as RM

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "threshold_runtime_model.json")


def _table():
    d = json.load(open(GOLDEN))
    rows = np.array(d["rows"], dtype=np.float64)
    r = rows[:, 2] / d["N_xi_UVS"]
    f = rows[:, 3] / d["N_int"]
    return d, rows, r, f


def test_fit_reproduces_the_papers_calibration():
    d, rows, r, f = _table()
    # t_UVS from the f = 0 row's printed model time and the printed c
    t_uvs = rows[0, 5] / (r[0] + d["fit"]["c"])
    m = RM.fit(r, f, rows[:, 4] / t_uvs)
    assert abs(m["lambda_cross"] - d["fit"]["lambda_cross"]) < 5e-5
    assert abs(m["c"] - d["fit"]["c"]) < 5e-6
    assert abs(m["r2"] - d["fit"]["r2"]) < 5e-4
    np.testing.assert_allclose(m["t_rel_model"] * t_uvs, rows[:, 5], rtol=0, atol=0.06)
    err = 100.0 * (m["t_rel_model"] * t_uvs - rows[:, 4]) / rows[:, 4]
    np.testing.assert_allclose(err, rows[:, 6], rtol=0, atol=0.051)


def test_breakeven_fraction_at_tau_005():
    d, rows, r, f = _table()
    be = RM.breakeven_cross_fraction(r[0], r[2], d["fit"]["lambda_cross"])
    assert round(100.0 * be, 1) == d["breakeven_f_at_tau_0.05_percent"]
    assert f[2] < be                                   # the multi-level set wins at tau 0.05


def test_fit_is_exact_on_model_data_and_the_index_adds_its_terms():
    r = np.array([0.2, 0.15, 0.12, 0.11])
    f = np.array([0.0, 0.03, 0.06, 0.1])
    m = RM.fit(r, f, r + 0.5 * f + 0.02)
    assert abs(m["lambda_cross"] - 0.5) < 1e-12 and abs(m["c"] - 0.02) < 1e-12 and abs(m["r2"] - 1.0) < 1e-12
    assert RM.workload_index(0.1, 0.05, 0.3, 0.02, 2.0) == 0.1 + 0.3 * 0.05 + 2.0 * 0.02
