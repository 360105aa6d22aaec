"""Pins of the oracle's level-selector network against things other than itself:
finite differences of the loss, closed forms of softmax cross-entropy, BF16 rounding of
known values, and the features of states whose gradients are known."""
import numpy as np

from oracle import mlp


def _batch(seed, n=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.N_IN))
    y = rng.integers(0, mlp.N_OUT, size=n)
    return X, y


def test_gradient_matches_finite_differences():
    X, y = _batch(1)
    w = mlp.init_weights(7) + 0.01 * np.random.default_rng(2).normal(size=mlp.N_PARAM)
    _, g = mlp.loss_and_grad(w, X, y)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(640, 12, replace=False),                      # W1
                          640 + rng.choice(64, 4, replace=False),                  # b1
                          704 + rng.choice(4096, 12, replace=False),               # W2
                          4800 + rng.choice(64, 4, replace=False),                 # b2
                          4864 + rng.choice(256, 8, replace=False),                # W3
                          5120 + np.arange(4)])                                    # b3
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAM)
        e[i] = h
        fd = (mlp.loss_and_grad(w + e, X, y)[0] - mlp.loss_and_grad(w - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i])), i


def test_zero_network_closed_forms():
    X, y = _batch(4, n=40)
    w = np.zeros(mlp.N_PARAM)
    loss, g = mlp.loss_and_grad(w, X, y)
    assert abs(loss - np.log(4.0)) < 1e-15            # uniform softmax over four classes
    freq = np.bincount(y, minlength=4) / len(y)
    np.testing.assert_allclose(g[-4:], 0.25 - freq, atol=1e-15)
    assert np.all(g[:-4] == 0.0)                       # no signal through zero weights


def test_training_separates_linear_classes():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(400, mlp.N_IN))
    y = (X[:, 0] > 0).astype(int) + 2 * (X[:, 1] > 0).astype(int)
    w = mlp.init_weights(11)
    v = np.zeros_like(w)
    losses = []
    for _ in range(300):
        loss, g = mlp.loss_and_grad(w, X, y)
        losses.append(loss)
        w, v = mlp.sgd_momentum(w, v, g, 0.05, 0.9)
    assert losses[-1] < 0.1 * losses[0]
    acc = np.mean(np.argmax(mlp.forward(w, X)[-1], axis=1) == y)
    assert acc > 0.97


def test_bf16_rounding_of_known_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0 + 2 ** -7, 1e-3])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                                 # tie: to the even mantissa
    assert r[2] == 1.0 + 2 * 2 ** -7                   # tie: 1.0078125 is odd, 1.015625 even
    assert r[3] == -2.5
    assert r[4] == 3.0                                 # spacing 2^-6 above 2: 3 + 2^-7 is a tie, 3.0 even
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3          # half a unit in the last place


def test_features_of_uniform_and_ramped_states():
    ny, nx = 6, 8
    rho = np.full((ny, nx), 1.3)
    u = np.full((ny, nx), 0.2)
    v = np.full((ny, nx), -0.1)
    T = np.full((ny, nx), 0.9)
    z = np.zeros((ny, nx))
    F = mlp.features(rho, u, v, T, z, z, 0.1, 0.1, True, True, R=1.0, T_ref=1.0, mu_ref=0.05, omega=0.81)
    np.testing.assert_allclose(F[:, 0], np.log(1.3))
    np.testing.assert_allclose(F[:, 1:3], np.tile([0.2, -0.1], (ny * nx, 1)))
    np.testing.assert_allclose(F[:, 6:9], 0.0, atol=1e-15)
    mu = 0.05 * 0.9 ** 0.81
    lam = mu / (1.3 * 0.9) * np.sqrt(np.pi * 0.9 / 2)
    np.testing.assert_allclose(F[:, 9], np.log10(lam))
    # a density ramp along x with clamped ends: interior gradient exact, half at the ends
    rho2 = np.tile(1.0 + 0.1 * np.arange(nx), (ny, 1))
    F2 = mlp.features(rho2, z, z, T, z, z, 0.5, 0.5, False, False, R=1.0, T_ref=1.0, mu_ref=0.05, omega=0.81)
    g = F2[:, 6].reshape(ny, nx) * rho2 / 0.5
    np.testing.assert_allclose(g[:, 1:-1], 0.2, rtol=1e-12)
    np.testing.assert_allclose(g[:, [0, -1]], 0.1, rtol=1e-12)


def test_curvilinear_features_reduce_to_cartesian():
    rng = np.random.default_rng(8)
    ny, nx, dx, dy = 5, 7, 0.2, 0.1
    f = [1.0 + 0.1 * rng.random((ny, nx)) for _ in range(4)]
    q = [0.01 * rng.standard_normal((ny, nx)) for _ in range(2)]
    Jt = np.zeros((ny, nx, 4))
    Jt[..., 0], Jt[..., 3] = 1.0 / dx, 1.0 / dy
    width = np.full((ny, nx), min(dx, dy))
    for px, py in ((True, True), (False, True), (False, False)):
        a = mlp.features(f[0], f[1], f[2], f[3], q[0], q[1], dx, dy, px, py, R=1.0, T_ref=1.0,
                         mu_ref=0.05, omega=0.81)
        b = mlp.features_curvi(f[0], f[1], f[2], f[3], q[0], q[1], Jt, width, px, py, R=1.0, T_ref=1.0,
                               mu_ref=0.05, omega=0.81)
        np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-15)
