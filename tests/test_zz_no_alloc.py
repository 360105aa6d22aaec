"""mlvs_moments_noalloc against mlvs_moments, through the C ABI (collected last on purpose).

The allocation-free entry point serves callers that must not have the library allocate device
memory (a process that reserves its GPU memory up front, or work recorded into a CUDA graph).
It keeps its partial sums in a fixed file-scope device array instead of handle-owned buffers.
The test feeds it the distributions of a running handle and checks, on two calls in a row, that
its (rho, rho u, rho v, rho E) agree with the handle's own moments within the FP32 tolerance of
the parity tests (1e-5 relative).
"""
import numpy as np
import pytest

from tests.helpers import have_gpu
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import torch  # noqa: E402

from oracle import vspace  # noqa: E402
from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def _axes(desc):
    base = vspace.make_base(desc["n_base"], desc["umin"], desc["umax"], D=2, rule=desc["rule"])
    n = base.n
    xi_x = np.tile(base.x, n)            # v = iy * n + ix
    xi_y = np.repeat(base.x, n)
    w_x = np.tile(base.w, n)
    w_y = np.repeat(base.w, n)
    dev = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in (xi_x, xi_y, w_x, w_y)]
    return n * n, dev


def _noalloc_vs_handle(s, nv, axes):
    ncell = s.ncell
    g, h = s.read_cells(0, ncell, nv)
    gd = torch.tensor(g.T.copy(), dtype=torch.float32, device="cuda")
    hd = torch.tensor(h.T.copy(), dtype=torch.float32, device="cuda")
    out = torch.full((4, ncell), float("nan"), dtype=torch.float64, device="cuda")
    M.mlvs_moments_noalloc(gd, hd, nv, ncell, *axes, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    m = s.moments(M.RHO | M.U | M.V | M.RHOE)
    ref = np.stack([m[0], m[0] * m[1], m[0] * m[2], m[3]])
    # relative for rho and rho E; momentum against rho sqrt(R T) (R = T = 1 here), the
    # parity tests' 1e-5 sqrt(R T) velocity tolerance
    scale = np.maximum(np.abs(ref), np.abs(ref[0]))
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref) / scale) < 1e-5


def test_noalloc_matches_handle_moments_twice():
    desc = workloads.cavity(48, n_base=25, Kn=0.075)
    s = Solver(desc)
    nv, axes = _axes(desc)
    s.step(3)
    _noalloc_vs_handle(s, nv, axes)
    s.step(2)
    _noalloc_vs_handle(s, nv, axes)


def _numpy_moments(g, h, xi_x, xi_y, w_x, w_y):
    """(rho, rho u, rho v, rho E) of FP32 arrays [nv][ncell], summed in FP64."""
    w = (w_x.astype(np.float64) * w_y.astype(np.float64))[:, None]
    x, y = xi_x.astype(np.float64)[:, None], xi_y.astype(np.float64)[:, None]
    g, h = g.astype(np.float64), h.astype(np.float64)
    return np.stack([np.sum(w * g, 0), np.sum(w * x * g, 0), np.sum(w * y * g, 0),
                     np.sum(0.5 * w * ((x * x + y * y) * g + h), 0)])


def _call(g, h, axes):
    nv, ncell = g.shape
    dev = [torch.tensor(a, device="cuda") for a in (g, h, *axes)]
    out = torch.full((4, ncell), float("nan"), dtype=torch.float64, device="cuda")
    M.mlvs_moments_noalloc(*dev[:2], nv, ncell, *dev[2:], out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_sizes_against_numpy():
    """Fewer velocities than chunks (nv = 5: most chunks empty, their rows still written), the
    largest accepted cell count, and a large call followed by a smaller one that must not pick
    up the larger call's partial sums."""
    rng = np.random.default_rng(20261202)

    def case(nv, ncell):
        g = rng.random((nv, ncell), dtype=np.float32)
        h = rng.random((nv, ncell), dtype=np.float32)
        axes = [rng.standard_normal(nv).astype(np.float32) for _ in range(2)] + \
               [rng.random(nv, dtype=np.float32) for _ in range(2)]
        got = _call(g, h, axes)
        ref = _numpy_moments(g, h, *axes)
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / scale) < 1e-12

    case(5, 300)
    case(37, 16384)
    case(3, 1000)
    case(40, 200)


def test_noalloc_rejects_too_many_cells():
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MLVSError) as e:
        M.mlvs_moments_noalloc(dummy, dummy, 1, 16385, dummy, dummy, dummy, dummy, out)
    assert e.value.status == -1
