"""Seeded synthetic workloads shaped like the paper's benchmarks.

Each function returns a plain description: mesh, boundary kinds, gas constants, velocity
grid and the initial primitive fields (rho, u, v, T) per cell, or (for unstructured meshes)
nodes and cells.  Nothing here evaluates the kinetic method; the same description feeds the
CUDA library and the test-side oracle.

Units are dimensionless: R = 1, T_ref = 1, rho_ref = 1, L_ref = 1, so velocity ranges are
multiples of sqrt(R T_ref).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20261202


def _desc(name, dim, nx, ny, Lx, Ly, bc, init, *, wall=((0.0, 0.0, 1.0),) * 4, R=1.0, K=0.0,
          Pr=2.0 / 3.0, omega=0.81, Kn=None, mu_ref=None, n_base=101, umin=-6.0, umax=6.0,
          rule="boole", cfl=0.5, storage="f32", limiter="vanleer"):
    return {"name": name, "dim": dim, "nx": nx, "ny": ny, "Lx": Lx, "Ly": Ly, "bc": tuple(bc),
            "wall": tuple(tuple(float(x) for x in w) for w in wall), "R": R, "K": K, "Pr": Pr,
            "omega": omega, "Kn": Kn, "mu_ref": mu_ref, "n_base": n_base, "umin": umin,
            "umax": umax, "rule": rule, "cfl": cfl, "storage": storage, "limiter": limiter,
            "init": np.ascontiguousarray(init, dtype=np.float64)}


def sod_1d(ncell=200, n_base=101, umax=10.0, Kn=1e-3, storage="f64"):
    """1-D shock tube: (rho, p) = (1, 1) | (0.125, 0.1) at rest on [0, 1], BGK, gamma = 5/3."""
    x = (np.arange(ncell) + 0.5) / ncell
    rho = np.where(x < 0.5, 1.0, 0.125)
    p = np.where(x < 0.5, 1.0, 0.1)
    init = np.zeros((1, ncell, 4))
    init[0, :, 0] = rho
    init[0, :, 3] = p / rho
    return _desc("sod1d", 1, ncell, 1, 1.0, 1.0, ("zerograd", "zerograd", "periodic", "periodic"),
                 init, Pr=1.0, Kn=Kn, n_base=n_base, umin=-umax, umax=umax, storage=storage)


def cavity(n=64, n_base=101, umax=6.0, Kn=0.075, lid_mach=0.16, storage="f32"):
    """Lid-driven cavity on [0,1]^2, diffuse isothermal walls at T_w = 1, gas at rest, T = 1.

    The lid (y-high side) moves at U_w = Ma sqrt(gamma R T_w), gamma = 5/3; Shakhov Pr = 2/3.
    """
    Uw = lid_mach * math.sqrt(5.0 / 3.0)
    init = np.zeros((n, n, 4))
    init[..., 0] = 1.0
    init[..., 3] = 1.0
    wall = ((0.0, 0.0, 1.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0), (Uw, 0.0, 1.0))
    return _desc("cavity", 2, n, n, 1.0, 1.0, ("wall",) * 4, init, wall=wall, Kn=Kn,
                 n_base=n_base, umin=-umax, umax=umax, storage=storage)


def supersonic_channel(nx=48, ny=16, mach=2.0, n_base=41, umax=8.0, Kn=0.05, storage="f32", walls=False):
    """Channel flow: freestream inflow at x-low (rho, T = 1, u = Ma sqrt(gamma R T), gamma = 5/3),
    freestream outflow side at x-high, periodic (or diffuse walls at T = 1) in y.  The gas
    starts as the freestream with a density and temperature bump at the channel centre."""
    u = mach * math.sqrt(5.0 / 3.0)
    x = (np.arange(nx) + 0.5) / nx * (nx / ny)
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    bump = np.exp(-((X - 0.5 * nx / ny) ** 2 + (Y - 0.5) ** 2) / 0.02)
    init = np.zeros((ny, nx, 4))
    init[..., 0] = 1.0 + 0.3 * bump
    init[..., 1] = u
    init[..., 3] = 1.0 + 0.2 * bump
    ybc = ("wall", "wall") if walls else ("periodic", "periodic")
    d = _desc("supersonic_channel", 2, nx, ny, nx / ny, 1.0, ("freestream", "freestream") + ybc, init,
              Kn=Kn, n_base=n_base, umin=-umax, umax=umax, storage=storage)
    d["far"] = (1.0, u, 0.0, 1.0)
    return d


def ogrid_nodes(ntheta, nr, r_in=1.0, r_out=11.0):
    """Nodes [nr+1][ntheta+1][2] of an O-grid around a cylinder of radius r_in: ntheta cells
    around (the node index i runs clockwise so that cells are counter-clockwise with j
    outward; column ntheta repeats column 0), nr cells out to r_out, geometrically stretched
    with the first cell height r_in 2 pi / ntheta (square cells at the wall)."""
    h0 = r_in * 2.0 * math.pi / ntheta
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        if h0 * (q ** nr - 1.0) / (q - 1.0) > r_out - r_in:
            hi = q
        else:
            lo = q
    q = 0.5 * (lo + hi)
    r = r_in + h0 * (q ** np.arange(nr + 1) - 1.0) / (q - 1.0)
    r[-1] = r_out
    th = -2.0 * math.pi * np.arange(ntheta + 1) / ntheta
    R, TH = np.meshgrid(r, th, indexing="ij")
    xy = np.stack([R * np.cos(TH), R * np.sin(TH)], axis=-1)
    xy[:, -1] = xy[:, 0]
    return xy


def cylinder(ntheta=256, nr=128, mach=5.0, Kn=0.1, n_base=201, umax=15.0, r_out=11.0, storage="f32",
             start="impulsive", ramp=2.0):
    """Flow past a cylinder of radius 1 on an O-grid: periodic around, a diffuse wall at
    T_w = T_inf on the cylinder (j = 0), freestream (rho, T = 1, u = Ma sqrt(gamma R T),
    gamma = 5/3) at the outer boundary.  start = "impulsive": the gas starts as the freestream
    everywhere.  start = "ramp": the speed rises from zero at the wall to the freestream's over
    about `ramp` radii, u = u_inf (1 - exp(-((r - 1) / ramp)^2)), at the freestream's total
    enthalpy (T = T_inf + (u_inf^2 - u^2) / (2 c_p), c_p = 5R/2) and pressure (rho T = 1): the
    gas near the cylinder starts near its stagnation state instead of striking the wall at the
    freestream speed and leaving a near-vacuum behind it."""
    u = mach * math.sqrt(5.0 / 3.0)
    nodes = ogrid_nodes(ntheta, nr, 1.0, r_out)
    init = np.zeros((nr, ntheta, 4))
    init[..., 0] = 1.0
    init[..., 1] = u
    init[..., 3] = 1.0
    if start == "ramp":
        c = 0.25 * (nodes[:-1, :-1] + nodes[1:, :-1] + nodes[:-1, 1:] + nodes[1:, 1:])   # cell centres
        r = np.hypot(c[..., 0], c[..., 1])
        uc = u * (1.0 - np.exp(-((r - 1.0) / ramp) ** 2))
        T = 1.0 + (u * u - uc * uc) / 5.0
        init[..., 1] = uc
        init[..., 3] = T
        init[..., 0] = 1.0 / T
    elif start != "impulsive":
        raise ValueError("start must be 'impulsive' or 'ramp'")
    d = _desc("cylinder", 2, ntheta, nr, 1.0, 1.0, ("periodic", "periodic", "wall", "freestream"), init,
              Kn=Kn, n_base=n_base, umin=-umax, umax=umax, storage=storage)
    d["far"] = (1.0, u, 0.0, 1.0)
    d["nodes"] = nodes
    return d


def periodic_random(nx, ny, n_base=25, umax=6.0, seed=SEED, amp=0.2, Kn=0.1, Pr=2.0 / 3.0,
                    storage="f32", dim=2, bc=None):
    """Smooth random periodic fields: a few seeded Fourier modes of rho, u, v, T."""
    rng = np.random.default_rng(seed)
    y = (np.arange(ny) + 0.5) / ny
    x = (np.arange(nx) + 0.5) / nx
    X, Y = np.meshgrid(x, y)
    init = np.zeros((ny, nx, 4))
    base = (1.0, 0.0, 0.0, 1.0)
    scale = (amp, 0.3 * amp * 2, 0.3 * amp * 2, amp)
    for f in range(4):
        field = np.full_like(X, base[f])
        for _ in range(3):
            kx, ky = rng.integers(0, 3, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(-1, 1) * scale[f]
            field += a * np.sin(2 * np.pi * (kx * X + (ky * Y if dim == 2 else 0)) + ph)
        init[..., f] = field
    if dim == 1:
        init[..., 2] = 0.0
    if bc is None:
        bc = ("periodic",) * 4
    return _desc("periodic_random", dim, nx, ny, 1.0, 1.0 if dim == 2 else 1.0, bc, init, Kn=Kn,
                 Pr=Pr, n_base=n_base, umin=-umax, umax=umax, storage=storage)


def uniform_flow(nx=100, ny=10, n_base=89, R=0.5, Kn=0.1, storage="f32"):
    """Uniform flow on the periodic box [0,1] x [0,0.1]: rho = 1, u = (0.1, 0), T = 1."""
    init = np.zeros((ny, nx, 4))
    init[..., 0] = 1.0
    init[..., 1] = 0.1
    init[..., 3] = 1.0
    um = 4.0 * math.sqrt(2.0 * R * 1.0)
    return _desc("uniform", 2, nx, ny, 1.0, 0.1, ("periodic",) * 4, init, R=R, Kn=Kn,
                 n_base=n_base, umin=-um, umax=um, storage=storage)


def sine_wave(nx=100, ny=10, n_base=89, R=0.5, Kn=0.1, storage="f32"):
    """Density wave at constant pressure: rho = 1 + 0.2 sin(2 pi x), u = (0.1, 0), p = 0.5."""
    x = (np.arange(nx) + 0.5) / nx
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
    init = np.zeros((ny, nx, 4))
    init[..., 0] = rho[None, :]
    init[..., 1] = 0.1
    init[..., 3] = (0.5 / (rho * R))[None, :]
    um = 4.0 * math.sqrt(2.0 * R * 1.0)
    return _desc("sine", 2, nx, ny, 1.0, 0.1, ("periodic",) * 4, init, R=R, Kn=Kn,
                 n_base=n_base, umin=-um, umax=um, storage=storage)


def batched_cavities(n_inst=64, seed=SEED, sizes=(32, 48, 64, 96, 128)):
    """Independent cavity instances: Kn log-uniform in [1e-3, 10], grid size drawn from sizes."""
    rng = np.random.default_rng(seed)
    kn = 10.0 ** rng.uniform(-3.0, 1.0, size=n_inst)
    n = rng.choice(np.asarray(sizes), size=n_inst)
    return [cavity(int(n[i]), Kn=float(kn[i])) for i in range(n_inst)]


def radial_levels(n_base, radii=((4.75, 99.0, 99.0), (4.0, 5.0, 99.0), (3.25, 4.25, 5.25)), umin=-6.0, umax=6.0):
    """Four velocity levels for the selector: level 0 fine everywhere, level L = 1..3 fine
    inside radius r1 of the origin and coarsened to 1, 2, 3 beyond r1, r2, r3 (units of
    sqrt(R T_ref)).  Returned as coarsening-index arrays over the 2x2 blocks of the base grid
    ([N1][N1] uint8), the radius of a block taken at its index distance from the centre block
    times the block width 2 (umax - umin) / (n_base - 1)."""
    c = (n_base - 1) // 2
    N1 = 2 * max(c // 2, 1) + 1
    width = 2.0 * (umax - umin) / (n_base - 1)
    b = np.arange(N1) - N1 // 2
    BX, BY = np.meshgrid(b, b)
    R = np.hypot(BX, BY) * width
    out = [np.zeros((N1, N1), dtype=np.uint8)]
    for r1, r2, r3 in radii:
        k = np.zeros((N1, N1), dtype=np.uint8)
        k[R > r1] = 1
        k[R > r2] = 2
        k[R > r3] = 3
        out.append(k)
    return out


def selector_init(seed=SEED):
    """He-uniform initial weights of the 10-64-64-4 selector (biases zero), flat [5124]
    in the layout W1 [64][10], b1 [64], W2 [64][64], b2 [64], W3 [4][64], b3 [4]."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, 10), (64, 64), (4, 64)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


# smooth random states for the selector's training data (density and temperature stay above
# 0.3 for these amplitudes and seeds), each at two Knudsen numbers; two held-out cases
SELECTOR_TRAIN = [(amp, Kn, seed) for amp, seed in ((0.2, 1), (0.2, 2), (0.2, 3), (0.35, 2), (0.35, 3),
                                                    (0.5, 2), (0.5, 3)) for Kn in (0.01, 1.0)]
SELECTOR_HELD = [(0.35, 1.0, 4), (0.2, 0.01, 4)]


# ------------------------------------------------------------------ unstructured meshes

def quad_mesh(x_edges, y_edges):
    """Nodes and counter-clockwise quads of a tensor grid, cells in row-major order."""
    nx, ny = len(x_edges) - 1, len(y_edges) - 1
    X, Y = np.meshgrid(x_edges, y_edges)
    nodes = np.stack([X.ravel(), Y.ravel()], axis=-1)
    idx = lambda i, j: j * (nx + 1) + i
    cells = [(idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)) for j in range(ny) for i in range(nx)]
    return nodes, cells


def two_cavities(m, L=1.0, channel=1.0, width=0.125):
    """Two square cavities of side L joined by a channel (length `channel`, width `width`),
    centred on x = 0: square cells of side width / m on three blocks that share their nodes
    (m even, so that the channel walls at +-width/2 are grid lines of the cavities).
    Returns (nodes, cells)."""
    if m % 2:
        raise ValueError("m must be even")
    h = width / m
    n_cav, n_ch = int(round(L / h)), int(round(channel / h))
    xs_left = -0.5 * channel - L + h * np.arange(n_cav + 1)
    xs_ch = -0.5 * channel + h * np.arange(n_ch + 1)
    xs_right = 0.5 * channel + h * np.arange(n_cav + 1)
    ys_cav = -0.5 * L + h * np.arange(n_cav + 1)
    ys_ch = -0.5 * width + h * np.arange(m + 1)
    key = lambda x, y: (int(np.floor(x / h + 0.5)), int(np.floor(y / h + 0.5)))
    nodes, index = [], {}

    def node(x, y):
        k = key(x, y)
        if k not in index:
            index[k] = len(nodes)
            nodes.append((x, y))
        return index[k]

    cells = []
    for xs, ys in ((xs_left, ys_cav), (xs_ch, ys_ch), (xs_right, ys_cav)):
        for j in range(len(ys) - 1):
            for i in range(len(xs) - 1):
                cells.append((node(xs[i], ys[j]), node(xs[i + 1], ys[j]), node(xs[i + 1], ys[j + 1]),
                              node(xs[i], ys[j + 1])))
    return np.array(nodes), cells


def triangulate(nodes, cells):
    """Each quad split into two triangles along alternating diagonals."""
    tri = []
    for k, (a, b, c, d) in enumerate(cells):
        if k % 2 == 0:
            tri += [(a, b, c), (a, c, d)]
        else:
            tri += [(a, b, d), (b, c, d)]
    return nodes, tri
