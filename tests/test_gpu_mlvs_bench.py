"""MLVS at the benchmarked configuration, element by element against the oracle.

The 64 x 64 lid-driven cavity on the 101^2 Boole base grid, f stored in FP32 (the benchmark's
MLVS leg): 200 UVS steps, then one adaptation with the cavity thresholds of Sec. 4 (C_split
5e-3, C_merge 2.5e-3, eps_merge 5e-5, tau_clust 0.05, blocks up to 4x4), which leaves the
cells on representative spaces cut from the base grid by the criterion (not tensor
products, so the split finalisation runs).  The oracle then takes the library's state on the
same spaces (its own construction of each space from the level's mask, checked point by point
against the library's) and both advance a few steps: the multi-level step of Sec. 3.4, or for
a single space the uniform step on that space.  Bounds: 2e-5 of the largest value on every
(cell, velocity) value, and the FP32 tolerance of the parity tests, 1e-5, on rho, u, v
(of sqrt(RT)) and T.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import dugks, kinetic, mlvs as omlvs, vspace  # noqa: E402
from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402

MLVS_PARAMS = (5e-3, 2.5e-3, 5e-5, 0.05, 2)
STEPS = 3


def test_mlvs_at_the_benchmarked_cavity_matches_the_oracle():
    n = 64
    desc = workloads.cavity(n, n_base=101, umax=6.0, Kn=0.075, storage="f32")
    ncell = n * n
    s = Solver(desc, adaptive=1)
    s.step(200)
    st = M.mlvs_adapt(s.h, M.adapt_params(*MLVS_PARAMS))
    nlev = st.n_levels
    lev = s.moments(M.LEVEL)[0].astype(int)
    o = oracle_setup(desc)
    book = omlvs.SpaceBook(o["base"])
    keys = []
    for L in range(nlev):
        k = M.mlvs_level_kappa(s.h, L).astype(np.int64).reshape(book.N1, book.N1)
        keys.append(book.get(k))
        S = book.space(keys[-1])
        x, y, w = M.mlvs_level_info(s.h, L)
        np.testing.assert_allclose(np.stack([x, y], 1), S.xi, rtol=0, atol=1e-13)
        np.testing.assert_allclose(w, S.w, rtol=1e-13)
        assert vspace.uniform_space(o["base"], 0).xi.shape[0] > S.xi.shape[0]   # a cut space
    # the library's state (FP32 values) as the oracle's FP64 state
    g0, h0 = [], []
    for c in range(ncell):
        g, h = s.read_cells(c, 1, 10201)
        g0.append(g[0].copy())
        h0.append(h[0].copy())
    s.step(STEPS)
    if nlev == 1:
        S = book.space(keys[0])
        G = np.stack(g0).reshape(n, n, -1)
        H = np.stack(h0).reshape(n, n, -1)
        for _ in range(STEPS):
            G, H, _ = dugks.step(G, H, o["mesh"], S.xi, S.w, o["gas"], o["dt"], o["opt"])
        ref_g, ref_h = G.reshape(ncell, -1), H.reshape(ncell, -1)
        spaces = [S] * ncell
    else:
        ost = omlvs.MLVSState(o["mesh"], o["gas"], book, [keys[lev[c]] for c in range(ncell)], g0, h0,
                              o["dt"], o["opt"])
        for _ in range(STEPS):
            omlvs.step(ost)
        ref_g, ref_h = ost.g, ost.h
        spaces = [book.space(keys[lev[c]]) for c in range(ncell)]
    gmax = max(np.max(np.abs(r)) for r in ref_g)
    hmax = max(np.max(np.abs(r)) for r in ref_h)
    worst = 0.0
    for c in range(ncell):
        g, h = s.read_cells(c, 1, 10201)
        worst = max(worst, np.max(np.abs(g[0] - ref_g[c])) / gmax, np.max(np.abs(h[0] - ref_h[c])) / hmax)
    assert worst < 2e-5, worst
    # moments
    m = s.moments(M.RHO | M.U | M.V | M.T)
    gas = o["gas"]
    for c in range(0, ncell, 7):
        S = spaces[c]
        mo = kinetic.moments(ref_g[c], ref_h[c], S.xi, S.w, gas)
        sRT = np.sqrt(gas.R * mo["T"])
        assert abs(m[0][c] - mo["rho"]) < 1e-5 * mo["rho"]
        assert abs(m[1][c] - mo["u"][0]) < 1e-5 * sRT
        assert abs(m[2][c] - mo["u"][1]) < 1e-5 * sRT
        assert abs(m[3][c] - mo["T"]) < 1e-5 * mo["T"]
    s.close()
