"""The library's mapping kernel k_map (projection plus the four-moment correction of Sec. 3.3.2,
Eqs. hierarchical_projection_operator ... mapping_h_residual_correction in its four-moment form;
a CTA of 256 threads reducing over the velocity stripes of G columns in shared memory) run on
the CPU with emulated thread blocks (tests/emu/cta_shim.hpp), against the oracle's projection
and additive correction with the source's moments and temperature as targets (FP64, 1e-12 of
the largest value).  Columns: cylinder post-shock states and random smooth states, mapped
between two masked spaces both ways and from the base grid onto a masked space, with every
column count per CTA (8, 4, 2, 1) and a ragged last group."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import kinetic, mapping, vspace
from tests import test_expmap_emu as X

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(prefix="kmap_emu_"), "emu.so")
    subprocess.run(["g++", "-std=c++20", "-O1", "-fPIC", "-shared", "-I", CUDA_INC,
                    os.path.join(HERE, "emu", "kmap_emu.cpp"), "-o", out, "-lpthread"],
                   check=True, capture_output=True)
    L = C.CDLL(out)
    L.emu_kmap.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]
    return L


spaces = X.spaces


def _columns(bsp, state, src, n):
    rng = np.random.default_rng(3)
    cols = []
    for k in range(n):
        if k % 2 == 0:
            g, h = state(0.02 + 0.3 * rng.random())
        else:
            u = rng.normal(0.0, 1.0, 2)
            g, h = kinetic.maxwell_gh(np.array(0.5 + rng.random()), u, np.array(1.0 + 4.0 * rng.random()),
                                      bsp.xi, X.GAS)
        cols.append(mapping.project(g, h, bsp, src) if src is not bsp else (g, h))
    return cols


def _oracle(cols, src, dst):
    out = []
    for g, h in cols:
        m = kinetic.moments(g, h, src.xi, src.w, X.GAS)
        tar = np.concatenate([[m["rho"]], m["rho"] * m["u"], [m["rhoE"]]])
        gp, hp = mapping.project(g, h, src, dst)
        out.append(mapping.correct4(gp, hp, tar, m["T"], dst, X.GAS))
    return out


@pytest.mark.parametrize("G", [8, 4, 2, 1])
@pytest.mark.parametrize("route", ["A_to_B", "B_to_A", "base_to_A"])
def test_k_map_matches_the_oracle(lib, spaces, G, route):
    bsp, state, A, B = spaces
    src, dst = {"A_to_B": (A, B), "B_to_A": (B, A), "base_to_A": (bsp, A)}[route]
    n = 11                                                       # ragged against every G
    cols = _columns(bsp, state, src, n)
    off, idx, wgt = X._csr(src, dst)
    sv, tv = X._vt(src), X._vt(dst)
    S = np.ascontiguousarray(np.stack([np.stack([g for g, _ in cols], -1), np.stack([h for _, h in cols], -1)]))
    D = np.zeros((2, dst.nv, n))
    assert lib.emu_kmap(src.nv, sv.ctypes.data, dst.nv, tv.ctypes.data, off.ctypes.data, idx.ctypes.data,
                        wgt.ctypes.data, S.ctypes.data, D.ctypes.data, n, X.GAS.R, X.GAS.K, G) == 0
    for k, (ge, he) in enumerate(_oracle(cols, src, dst)):
        np.testing.assert_allclose(D[0, :, k], ge, rtol=0, atol=1e-12 * np.max(np.abs(ge)))
        np.testing.assert_allclose(D[1, :, k], he, rtol=0, atol=1e-12 * np.max(np.abs(he)))
