"""The library's Cartesian step, tile kernels included, run on the CPU against the oracle's
Cartesian step (Sec. 2.2).  The tile kernels (MODE 0 face sums and MODE 1 update: shared-memory
staging of a 16 x 16 tile with its two-cell halo, slopes, upwind faces and barrier rounds of two
velocities) run on emulated thread blocks (tests/emu/tile_emu.cpp), with the initialisation,
chunk-sum and finalisation kernels the handle launches around them.  FP64, 1e-13 of the largest
value after two steps (FP32 on the cavity, 1e-5), on meshes that leave partial tiles: doubly periodic, a lid-driven cavity
(walls, one moving), and a supersonic channel (freestream inflow and outflow, walls).  On a space
cut from the base grid the finalisation takes its split path, whose velocity sums run one warp
per point from the space's row tables (warp shuffles emulated): the cavity with the four- and the
eight-moment correction against the oracle's step on that space, FP64 1e-12 and FP32 2e-5."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import dugks, vspace
from tests.helpers import oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
BC = {"periodic": 0, "zerograd": 1, "wall": 2, "freestream": 3}
RULE = {"boole": 0, "simpson": 1, "trapz": 2}
LIM = {"vanleer": 0, "none": 1}


def _build(fp32):
    out = os.path.join(tempfile.mkdtemp(prefix="tile_emu_"), "emu.so")
    subprocess.run(["g++", "-std=c++20", "-O1", "-fPIC", "-shared", "-I", CUDA_INC, *(["-DEMU_FP32"] if fp32 else []),
                    os.path.join(HERE, "emu", "tile_emu.cpp"), "-o", out, "-lpthread"],
                   check=True, capture_output=True)
    L = C.CDLL(out)
    P = C.c_void_p
    L.emu_tile_run.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, P, P, P, C.c_int, C.c_double,
                               C.c_double, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, P, P, C.c_int,
                               C.c_int, P, C.c_int, C.c_int, P, C.POINTER(C.c_int)]
    return L


@pytest.fixture(scope="module")
def lib():
    return _build(False)


@pytest.fixture(scope="module")
def lib32():
    return _build(True)


def _emu(lib, desc, o, steps, vpc, nv, kappa=None, compat_moments=4, split=False):
    """The emulated step's distributions [ny][nx][nv] (g, h) after `steps` steps."""
    nx, ny = desc["nx"], desc["ny"]
    gas = o["gas"]
    bc = np.array([BC[b] for b in desc["bc"]], dtype=np.int32)
    wall = np.ascontiguousarray(np.array(desc["wall"], dtype=np.float64).reshape(12))
    gas6 = np.array([gas.R, gas.K, gas.Pr, gas.omega, gas.mu_ref, gas.T_ref])
    far = np.array(desc.get("far", (1.0, 0.0, 0.0, 1.0)), dtype=np.float64)
    W0 = np.ascontiguousarray(desc["init"].reshape(-1, 4), dtype=np.float64)
    out = np.zeros((2, nv, nx * ny))
    nvo = C.c_int()
    kp = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.uint8)
    err = lib.emu_tile_run(nx, ny, desc["Lx"], desc["Ly"], bc.ctypes.data, wall.ctypes.data, gas6.ctypes.data,
                           desc["n_base"], desc["umin"], desc["umax"], RULE[desc["rule"]], o["dt"],
                           int(o["opt"].compat_cell), int(o["opt"].compat_face), LIM[desc["limiter"]],
                           far.ctypes.data, W0.ctypes.data, steps, vpc,
                           None if kp is None else kp.ctypes.data, compat_moments, int(split), out.ctypes.data,
                           C.byref(nvo))
    assert err == 0 and nvo.value == nv
    return out[0].T.reshape(ny, nx, nv), out[1].T.reshape(ny, nx, nv)


def _run(lib, desc, steps, vpc):
    o = oracle_setup(desc)
    g_o, h_o = oracle_run(o, steps)
    g, h = _emu(lib, desc, o, steps, vpc, g_o.shape[-1])
    return g, h, g_o, h_o


@pytest.mark.parametrize("case", ["periodic", "cavity", "channel"])
def test_tile_kernels_match_the_oracle(lib, case):
    if case == "periodic":
        desc = workloads.periodic_random(20, 12, n_base=13, storage="f64")
    elif case == "cavity":
        desc = workloads.cavity(18, n_base=13, umax=5.0, storage="f64")
    else:
        desc = workloads.supersonic_channel(20, 6, mach=1.5, n_base=13, umax=6.0, walls=True, storage="f64")
    g, h, g_o, h_o = _run(lib, desc, 2, vpc=40)                  # 169 velocities: a ragged last chunk
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-13 * np.max(np.abs(g_o)))
    np.testing.assert_allclose(h, h_o, rtol=0, atol=1e-13 * np.max(np.abs(h_o)))


def test_tile_kernels_fp32_match_the_oracle(lib32):
    """FP32 storage and arithmetic (the benchmark's): within 1e-5 of the largest value."""
    desc = workloads.cavity(18, n_base=13, umax=5.0, storage="f32")
    g, h, g_o, h_o = _run(lib32, desc, 2, vpc=40)
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-5 * np.max(np.abs(g_o)))
    np.testing.assert_allclose(h, h_o, rtol=0, atol=1e-5 * np.max(np.abs(h_o)))


def test_row_sum_layout_keeps_the_fp64_sums_aligned(lib, lib32):
    """The warp areas of the finalisation's row sums (FP32 and FP64 storage): every warp's area
    holds the prefix sums of NO orders (three compensated) over n1 + 4 slots, and above the
    lanes' padded pair moments (NE rows of 33) the NE sums as FP64 at an offset that keeps them
    8-byte aligned in every warp: an even count of values per warp and an even offset."""
    for L in (lib, lib32):
        for NO in (8, 10):
            ne = NO * (NO + 1) // 2
            pd = L.emu_row_pd(NO)
            assert pd % 2 == 0 and pd >= ne * 33
            for n1 in range(1, 700):
                v = L.emu_row_smem_values(n1, NO)
                assert v % 2 == 0, (n1, NO, v)
                assert v >= (NO + 3) * (n1 + 4) and v >= pd + 2 * ne, (n1, NO, v)


def _cut_kappa(n_base):
    """Quadtree levels 0 near the origin, 1 around it, 2 outside: a space cut from the base grid."""
    N1 = len(vspace.axis_groups(n_base, 1))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    return np.where(r < N1 / 5, 0, np.where(r < N1 / 3, 1, 2)).astype(np.uint8)


@pytest.mark.parametrize("compat_moments,fp32", [(4, False), (8, False), (8, True)])
def test_tile_step_on_a_cut_space_matches_the_oracle(lib, lib32, compat_moments, fp32):
    """The step on a space cut from the base grid (not a tensor product): the finalisation's
    split path with the velocity sums from the space's rows (warp shuffles emulated), the four-
    or eight-moment correction at cells and faces, walls on every side; from the emulation's
    own initial state, against the oracle's step on that space with the same correction."""
    import dataclasses

    from oracle import mlvs as omlvs
    desc = workloads.cavity(8, n_base=25, Kn=0.075, storage="f64")
    ka = _cut_kappa(25)
    o = oracle_setup(desc)
    book = omlvs.SpaceBook(o["base"])
    S = book.space(book.get(ka.astype(np.int64)))
    nv = S.xi.shape[0]
    assert nv < 25 * 25
    L = lib32 if fp32 else lib
    tol = 2e-5 if fp32 else 1e-12
    g0, h0 = _emu(L, desc, o, 0, 64, nv, ka, compat_moments)
    steps = 2
    g1, h1 = _emu(L, desc, o, steps, 64, nv, ka, compat_moments)
    opt = dataclasses.replace(o["opt"], compat_moments=compat_moments)
    G, H = g0, h0
    for _ in range(steps):
        G, H, _ = dugks.step(G, H, o["mesh"], S.xi, S.w, o["gas"], o["dt"], opt)
    assert np.max(np.abs(g1 - G)) < tol * np.max(np.abs(G))
    assert np.max(np.abs(h1 - H)) < tol * np.max(np.abs(H))


@pytest.mark.parametrize("case", ["periodic", "cavity"])
def test_split_finalisation_on_the_uniform_space_matches_the_oracle(lib, case):
    """The split finalisation on the tensor-product space (the handle's path for launches of
    fewer than 4,096 points): the one-axis sums split over a warp's lanes and merged with exact
    TwoSum compensation (warp shuffles emulated), FP64, against the oracle's step."""
    desc = (workloads.periodic_random(10, 6, n_base=13, storage="f64") if case == "periodic"
            else workloads.cavity(8, n_base=13, umax=5.0, storage="f64"))
    o = oracle_setup(desc)
    g_o, h_o = oracle_run(o, 2)
    g, h = _emu(lib, desc, o, 2, 64, g_o.shape[-1], split=True)
    assert np.max(np.abs(g - g_o)) < 1e-13 * np.max(np.abs(g_o))
    assert np.max(np.abs(h - h_o)) < 1e-13 * np.max(np.abs(h_o))
