"""Learned level selector (oracle; test infrastructure only).

A multilayer perceptron 10 -> 64 -> 64 -> 4 with ReLU activations maps local features of a
cell to logits over four velocity levels; it is trained with softmax cross-entropy on labels
produced by the criterion of Sec. 3.2 (the level the fixed-level-set rule assigns from the
cell's mask).  This is not part of the paper's method; the library adds it as a cheaper
stand-in for the criterion, with the criterion as fallback below a confidence threshold.

Everything here is plain FP64 numpy.  The library keeps the weights in BF16 for the forward
and backward passes (FP32 accumulation) and an FP32 master copy for the update; the oracle
takes the BF16-rounded weights as given values (they are exact in FP64) so the two compute
the same function.

Parameter layout (5,124 values): W1 [64][10], b1 [64], W2 [64][64], b2 [64], W3 [4][64], b3 [4].

Features of a cell (Sec. 2.1 moments; gradients by central differences over the mesh with
the neighbours wrapped on periodic sides and clamped on the others, i.e. the ghost-copy
reading of the boundaries):
  0 log rho          1 u / sqrt(R T_ref)     2 v / sqrt(R T_ref)     3 log(T / T_ref)
  4 q_x / (rho (RT)^1.5)                     5 q_y / (rho (RT)^1.5)
  6 dx |grad rho| / rho                      7 dx |grad T| / T
  8 dx |grad u| / sqrt(RT)  (Frobenius norm of the velocity gradient)
  9 log10 Kn_local, Kn_local = lambda / L_ref, lambda = (mu / p) sqrt(pi R T / 2)
with dx = min(dx, dy).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 10, 64, 4
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    """Parameter vector to named arrays (selector; no counterpart in the paper)."""
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    """Named arrays to the parameter vector (selector; no counterpart in the paper)."""
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64.
    Selector; no counterpart in the paper."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_weights(seed):
    """He-uniform weights, zero biases (a fixed recipe shared with the tests).
    Selector; no counterpart in the paper."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[1])
            p[name] = rng.uniform(-lim, lim, size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def forward(w, X):
    """Activations of a batch X [n][10]: (z1, h1, z2, h2, logits).
    Selector; no counterpart in the paper."""
    p = unpack(w)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    logits = h2 @ p["W3"].T + p["b3"]
    return z1, h1, z2, h2, logits


def softmax(logits):
    """Row-wise softmax of the logits (selector; no counterpart in the paper)."""
    m = logits - np.max(logits, axis=1, keepdims=True)
    e = np.exp(m)
    return e / np.sum(e, axis=1, keepdims=True)


def loss_and_grad(w, X, y):
    """Mean softmax cross-entropy over the batch and its gradient with respect to w.
    Selector; no counterpart in the paper."""
    n = X.shape[0]
    p = unpack(w)
    z1, h1, z2, h2, logits = forward(w, X)
    P = softmax(logits)
    loss = -np.mean(np.log(P[np.arange(n), y]))
    d3 = P.copy()
    d3[np.arange(n), y] -= 1.0
    d3 /= n                                       # d loss / d logits
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ p["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def sgd_momentum(w, v, grad, lr, mu):
    """v <- mu v + grad;  w <- w - lr v.  (selector; no counterpart in the paper)."""
    v = mu * v + grad
    return w - lr * v, v


def features(rho, u, v, T, qx, qy, dx, dy, periodic_x, periodic_y, R, T_ref, mu_ref, omega, L_ref=1.0):
    """The ten features of every cell of a [ny][nx] mesh, returned as [ny*nx][10].
    Selector, no counterpart in the paper; moments of Sec. 2.1."""
    def ddx(f):
        if periodic_x:
            fp, fm = np.roll(f, -1, axis=1), np.roll(f, 1, axis=1)
        else:
            fp = np.concatenate([f[:, 1:], f[:, -1:]], axis=1)
            fm = np.concatenate([f[:, :1], f[:, :-1]], axis=1)
        return (fp - fm) / (2.0 * dx)

    def ddy(f):
        if f.shape[0] == 1:
            return np.zeros_like(f)
        if periodic_y:
            fp, fm = np.roll(f, -1, axis=0), np.roll(f, 1, axis=0)
        else:
            fp = np.concatenate([f[1:], f[-1:]], axis=0)
            fm = np.concatenate([f[:1], f[:-1]], axis=0)
        return (fp - fm) / (2.0 * dy)

    h = min(dx, dy) if rho.shape[0] > 1 else dx
    RT = R * T
    gr = np.hypot(ddx(rho), ddy(rho))
    gT = np.hypot(ddx(T), ddy(T))
    gu = np.sqrt(ddx(u) ** 2 + ddy(u) ** 2 + ddx(v) ** 2 + ddy(v) ** 2)
    mu = mu_ref * (T / T_ref) ** omega
    lam = mu / (rho * RT) * np.sqrt(np.pi * RT / 2.0)
    c = np.sqrt(R * T_ref)
    F = np.stack([np.log(rho), u / c, v / c, np.log(T / T_ref),
                  qx / (rho * RT ** 1.5), qy / (rho * RT ** 1.5),
                  h * gr / rho, h * gT / T, h * gu / np.sqrt(RT), np.log10(lam / L_ref)], axis=-1)
    return F.reshape(-1, N_IN)


def features_curvi(rho, u, v, T, qx, qy, Jt, width, periodic_x, periodic_y, R, T_ref, mu_ref, omega,
                   L_ref=1.0):
    """The same features on a structured curvilinear mesh: gradients from central differences
    along the index directions (neighbours wrapped or clamped) turned physical with the cell's
    J^{-T} [ny][nx][4] (row-major), and the cell width |V| / max |S| [ny][nx] for dx.  On a
    Cartesian mesh this is `features`.
    Selector, no counterpart in the paper; moments of Sec. 2.1."""
    def d_i(f):
        if periodic_x:
            fp, fm = np.roll(f, -1, axis=1), np.roll(f, 1, axis=1)
        else:
            fp = np.concatenate([f[:, 1:], f[:, -1:]], axis=1)
            fm = np.concatenate([f[:, :1], f[:, :-1]], axis=1)
        return 0.5 * (fp - fm)

    def d_j(f):
        if periodic_y:
            fp, fm = np.roll(f, -1, axis=0), np.roll(f, 1, axis=0)
        else:
            fp = np.concatenate([f[1:], f[-1:]], axis=0)
            fm = np.concatenate([f[:1], f[:-1]], axis=0)
        return 0.5 * (fp - fm)

    def grad(f):
        a, b = d_i(f), d_j(f)
        return Jt[..., 0] * a + Jt[..., 1] * b, Jt[..., 2] * a + Jt[..., 3] * b

    RT = R * T
    gr = np.hypot(*grad(rho))
    gT = np.hypot(*grad(T))
    ux, uy = grad(u)
    vx, vy = grad(v)
    gu = np.sqrt(ux ** 2 + uy ** 2 + vx ** 2 + vy ** 2)
    mu = mu_ref * (T / T_ref) ** omega
    lam = mu / (rho * RT) * np.sqrt(np.pi * RT / 2.0)
    c = np.sqrt(R * T_ref)
    F = np.stack([np.log(rho), u / c, v / c, np.log(T / T_ref),
                  qx / (rho * RT ** 1.5), qy / (rho * RT ** 1.5),
                  width * gr / rho, width * gT / T, width * gu / np.sqrt(RT), np.log10(lam / L_ref)], axis=-1)
    return F.reshape(-1, N_IN)
