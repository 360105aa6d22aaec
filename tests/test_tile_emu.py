"""The library's Cartesian step, tile kernels included, run on the CPU against the oracle's
Cartesian step (Sec. 2.2).  The tile kernels (MODE 0 face sums and MODE 1 update: shared-memory
staging of a 16 x 16 tile with its two-cell halo, slopes, upwind faces and barrier rounds of two
velocities) run on emulated thread blocks (tests/emu/tile_emu.cpp), with the initialisation,
chunk-sum and finalisation kernels the handle launches around them.  FP64, 1e-13 of the largest
value after two steps (FP32 on the cavity, 1e-5), on meshes that leave partial tiles: doubly periodic, a lid-driven cavity
(walls, one moving), and a supersonic channel (freestream inflow and outflow, walls)."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

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
                               C.c_int, P, C.POINTER(C.c_int)]
    return L


@pytest.fixture(scope="module")
def lib():
    return _build(False)


@pytest.fixture(scope="module")
def lib32():
    return _build(True)


def _run(lib, desc, steps, vpc):
    o = oracle_setup(desc)
    g_o, h_o = oracle_run(o, steps)
    nx, ny = desc["nx"], desc["ny"]
    gas = o["gas"]
    bc = np.array([BC[b] for b in desc["bc"]], dtype=np.int32)
    wall = np.ascontiguousarray(np.array(desc["wall"], dtype=np.float64).reshape(12))
    gas6 = np.array([gas.R, gas.K, gas.Pr, gas.omega, gas.mu_ref, gas.T_ref])
    far = np.array(desc.get("far", (1.0, 0.0, 0.0, 1.0)), dtype=np.float64)
    W0 = np.ascontiguousarray(desc["init"].reshape(-1, 4), dtype=np.float64)
    nv = g_o.shape[-1]
    out = np.zeros((2, nv, nx * ny))
    nvo = C.c_int()
    err = lib.emu_tile_run(nx, ny, desc["Lx"], desc["Ly"], bc.ctypes.data, wall.ctypes.data, gas6.ctypes.data,
                           desc["n_base"], desc["umin"], desc["umax"], RULE[desc["rule"]], o["dt"],
                           int(o["opt"].compat_cell), int(o["opt"].compat_face), LIM[desc["limiter"]],
                           far.ctypes.data, W0.ctypes.data, steps, vpc, out.ctypes.data, C.byref(nvo))
    assert err == 0 and nvo.value == nv
    return out[0].T.reshape(ny, nx, nv), out[1].T.reshape(ny, nx, nv), g_o, h_o


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
