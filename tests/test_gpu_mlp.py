"""Level selector (10-64-64-4 network) through the C ABI, against the oracle.

The library's forward and backward passes read BF16 weights and accumulate in FP32; the
oracle evaluates the same BF16 values in FP64, so logits agree to FP32 accumulation error
(1e-5 of their scale) and gradients to 1e-4 of their largest entry.  The end-to-end test
trains the network on criterion labels and shows what it gains: the selector's adaptation
agrees with the criterion's on most cells and costs less time.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import torch  # noqa: E402

from oracle import dugks, mlp as omlp  # noqa: E402
from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def _weights(seed):
    rng = np.random.default_rng(seed)
    w = omlp.init_weights(seed) + 0.05 * rng.normal(size=omlp.N_PARAM)
    return w.astype(np.float32)


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, omlp.N_IN)).astype(np.float32)
    y = rng.integers(0, omlp.N_OUT, size=n).astype(np.int32)
    return X, y


def test_forward_matches_oracle():
    X, _ = _data(3, 300)
    w = _weights(1)
    m = M.mlvs_mlp_create()
    M.mlvs_mlp_set_weights(m, w)
    master, wb = M.mlvs_mlp_get_weights(m)
    np.testing.assert_array_equal(master, w)
    np.testing.assert_array_equal(wb, omlp.bf16_round(w))      # nearest-even BF16 copy
    Xd = torch.from_numpy(X).cuda()
    lg = torch.zeros(300, 4, device="cuda")
    pr = torch.zeros(300, 4, device="cuda")
    M.mlvs_mlp_forward(m, Xd, 300, lg, pr)
    torch.cuda.synchronize()
    ref = omlp.forward(wb.astype(np.float64), X.astype(np.float64))[-1]
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(lg.cpu().numpy() - ref)) < 1e-5 * scale
    np.testing.assert_allclose(pr.cpu().numpy(), omlp.softmax(ref), rtol=0, atol=1e-5)
    M.mlvs_mlp_destroy(m)


def test_gradient_matches_oracle():
    n = 300                                 # not a multiple of the 64-sample blocks
    X, y = _data(4, n)
    m = M.mlvs_mlp_create()
    M.mlvs_mlp_set_weights(m, _weights(2))
    _, wb = M.mlvs_mlp_get_weights(m)
    g = torch.zeros(M.N_SELECTOR_PARAMS, device="cuda")
    loss = M.mlvs_mlp_gradient(m, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), n, g)
    lref, gref = omlp.loss_and_grad(wb.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss - lref) < 1e-5 * max(1.0, lref)
    assert np.max(np.abs(g.cpu().numpy() - gref)) < 1e-4 * np.max(np.abs(gref))
    M.mlvs_mlp_destroy(m)


def test_train_step_matches_oracle_update():
    n = 256
    X, y = _data(5, n)
    w = _weights(3)
    m = M.mlvs_mlp_create()
    M.mlvs_mlp_set_weights(m, w)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    loss = M.mlvs_mlp_train_step(m, Xd, yd, n, 0.05, 0.9)
    master, _ = M.mlvs_mlp_get_weights(m)
    lref, gref = omlp.loss_and_grad(omlp.bf16_round(w), X.astype(np.float64), y)
    wref, _ = omlp.sgd_momentum(w.astype(np.float64), np.zeros(omlp.N_PARAM), gref, 0.05, 0.9)
    assert abs(loss - lref) < 1e-5 * max(1.0, lref)
    assert np.max(np.abs(master - wref)) < 1e-6
    # and it learns: 200 more steps on the same batch lower the loss
    for _ in range(200):
        last = M.mlvs_mlp_train_step(m, Xd, yd, n, 0.05, 0.9)
    assert last < 0.8 * loss
    M.mlvs_mlp_destroy(m)


@pytest.mark.parametrize("kind", ["periodic", "walls"])
def test_features_match_oracle(kind):
    if kind == "periodic":
        desc = workloads.periodic_random(12, 10, n_base=25, storage="f64", amp=0.3)
    else:
        desc = workloads.cavity(10, n_base=25, storage="f64")
    o = oracle_setup(desc)
    g, h = oracle_run(o, 3)
    s = Solver(desc)
    s.step(3)
    ncell = desc["nx"] * desc["ny"]
    F = M.mlvs_features(s.h, 0, ncell)
    st = dugks.cell_state(g, h, o["sp"].xi, o["sp"].w, o["gas"], o["dt"])
    per = kind == "periodic"
    Fo = omlp.features(st["rho"], st["u"][..., 0], st["u"][..., 1], st["T"], st["q"][..., 0], st["q"][..., 1],
                       o["mesh"].dx, o["mesh"].dy, per, per, R=o["gas"].R, T_ref=1.0,
                       mu_ref=o["gas"].mu_ref, omega=o["gas"].omega)
    assert np.max(np.abs(F - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5


def _labelled(desc, levels, p, steps=(0, 4, 4)):
    s = Solver(desc, levels=levels, adaptive=0)
    n = desc["nx"] * desc["ny"]
    Xs, ys = [], []
    for k in steps:
        if k:
            s.step(k)
        Xs.append(M.mlvs_features(s.h, 0, n))
        ys.append(M.mlvs_criterion_levels(s.h, 0, p, n))
    s.close()
    return np.concatenate(Xs), np.concatenate(ys)


def test_selector_learns_criterion_levels_and_saves_time():
    nb = 41
    levels = list(workloads.radial_levels(nb))
    p = M.adapt_params(5e-3, 2.5e-3, 0.0, 0.05, 3)
    train, held = workloads.SELECTOR_TRAIN, workloads.SELECTOR_HELD
    X, y = [], []
    for amp, Kn, seed in train:
        d = workloads.periodic_random(24, 24, n_base=nb, amp=amp, Kn=Kn, seed=seed)
        a, b = _labelled(d, levels, p)
        X.append(a)
        y.append(b)
    X, y = np.concatenate(X), np.concatenate(y)
    assert len(np.unique(y)) >= 3
    m = M.mlvs_mlp_create()
    M.mlvs_mlp_set_weights(m, workloads.selector_init())
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    first = M.mlvs_mlp_train_step(m, Xd, yd, len(y), 0.02, 0.9)
    for _ in range(1500):
        last = M.mlvs_mlp_train_step(m, Xd, yd, len(y), 0.02, 0.9)
    assert last < 0.5 * first
    # held-out accuracy
    for amp, Kn, seed in held:
        d = workloads.periodic_random(24, 24, n_base=nb, amp=amp, Kn=Kn, seed=seed)
        Xh, yh = _labelled(d, levels, p, steps=(0,))
        pr = torch.zeros(len(yh), 4, device="cuda")
        M.mlvs_mlp_forward(m, torch.from_numpy(Xh).cuda(), len(yh), None, pr)
        torch.cuda.synchronize()
        pr = pr.cpu().numpy()
        assert np.mean(np.argmax(pr, 1) == yh) > 0.85
    # adaptation on a held-out case: selector (with fallback) vs criterion
    amp, Kn, seed = held[0]
    d = workloads.periodic_random(64, 64, n_base=nb, amp=amp, Kn=Kn, seed=seed)
    a = Solver(d, levels=levels, adaptive=0)
    b = Solver(d, levels=levels, adaptive=0)
    a.step(2)
    b.step(2)
    for _ in range(2):                          # the second call of each is the timed one
        sa = M.mlvs_adapt(a.h, p)
        sb = M.mlvs_adapt_mlp(b.h, m, p, 0.9)
    la = a.moments(M.LEVEL)[0]
    lb = b.moments(M.LEVEL)[0]
    assert np.mean(la == lb) > 0.9
    assert sb.n_distinct < 0.3 * 4096           # cells that fell back to the criterion
    assert sb.ms_total < sa.ms_total
    # the solutions stay close
    a.step(10)
    b.step(10)
    ma, mb = a.moments(M.RHO | M.T), b.moments(M.RHO | M.T)
    assert np.max(np.abs(ma - mb) / ma) < 1e-3
    M.mlvs_mlp_destroy(m)
