"""The library's host construction of a velocity space from a coarsening mask (parent-child
consistency, merged coordinates and weights) against the oracle's, on CPU through the C ABI."""
import numpy as np
import pytest

from oracle import vspace
from paper_2609_35258_b300 import mlvs as M

RULES = {"boole": M.QUAD_BOOLE, "simpson": M.QUAD_SIMPSON, "trapz": M.QUAD_TRAPZ}


def _sorted(x, y, w):
    o = np.lexsort((x, y))
    return x[o], y[o], w[o]


def _masks(n, seed):
    N1 = len(vspace.axis_groups(n, 1))
    rng = np.random.default_rng(seed)
    out = [np.full((N1, N1), L, dtype=np.int64) for L in range(4)]
    out.append(rng.integers(0, 4, size=(N1, N1)))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    out.append(np.where(r < N1 / 6, 0, np.where(r < N1 / 3, 1, np.where(xx > N1 // 2, 3, 2))).astype(np.int64))
    return out


@pytest.mark.parametrize("n,umax,rule", [(101, 6.0, "boole"), (201, 15.0, "boole"), (41, 5.0, "simpson"),
                                         (25, 8.0, "trapz")])
def test_host_space_matches_oracle(n, umax, rule):
    base = vspace.make_base(n, -umax, umax, D=2, rule=rule)
    for seed, kappa in enumerate(_masks(n, n)):
        sp = vspace.kappa_space(base, vspace.enforce_consistency(kappa, n))
        x, y, w = M.mlvs_space_points(n, -umax, umax, RULES[rule], kappa.astype(np.uint8))
        assert len(w) == sp.nv, (seed, len(w), sp.nv)
        xo, yo, wo = _sorted(sp.xi[:, 0].copy(), sp.xi[:, 1].copy(), sp.w.copy())
        xl, yl, wl = _sorted(x, y, w)
        np.testing.assert_allclose(xl, xo, rtol=0, atol=1e-13 * umax)
        np.testing.assert_allclose(yl, yo, rtol=0, atol=1e-13 * umax)
        np.testing.assert_allclose(wl, wo, rtol=1e-13)
        assert abs(w.sum() - (2 * umax) ** 2) < 1e-12 * (2 * umax) ** 2


def test_host_space_rejects_bad_input():
    with pytest.raises(M.MLVSError):
        M.mlvs_space_points(100, -5.0, 5.0, M.QUAD_BOOLE, np.zeros(4, dtype=np.uint8))      # even size
    with pytest.raises(M.MLVSError):
        M.mlvs_space_points(25, -5.0, 5.0, M.QUAD_BOOLE, np.zeros(5, dtype=np.uint8))       # not n1 * n1
    with pytest.raises(M.MLVSError):
        M.mlvs_space_points(25, -5.0, 5.0, M.QUAD_BOOLE, np.full(169, 4, dtype=np.uint8))   # level above 3
