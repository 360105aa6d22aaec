"""The library's per-item state mappings, run on the CPU (the functions its CUDA kernels call,
compiled as host C++): the positivity fallback against the oracle's exponential correction
(Sec. 3.3.2, Eq. exponential_moment_correction; `mapping.correct_exp4`), and the nine-moment
mapping against the oracle's (`mapping.map9`; Eqs. mapping_nine_targets ...
mapping_h_residual_correction), both ways between two masked spaces, which keeps the nine raw
moments of the source to 1e-12.

A post-shock state of the Mach 5 cylinder (hot Maxwellian carrying a cold beam) lives on one
masked space and moves to another with the additive four-moment correction, which leaves
negative tails; the fallback must replace that result by the oracle's exponential one (FP64,
1e-12 of the largest value), keep the additive result where it has no negative value, and keep
it where the projection itself is negative (the oracle's rule)."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import criterion, kinetic, mapping, vspace

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
GAS = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0, omega=0.81, mu_ref=1e-3)


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(prefix="expmap_emu_"), "emu.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CUDA_INC,
                    os.path.join(HERE, "emu", "expmap_emu.cpp"), "-o", out], check=True, capture_output=True)
    L = C.CDLL(out)
    for fn in (L.emu_expmap, L.emu_map9):
        fn.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                       C.c_void_p, C.c_void_p]
    return L


@pytest.fixture(scope="module")
def spaces():
    base = vspace.make_base(81, -15.0, 15.0, D=2)
    bsp = vspace.uniform_space(base, 0)
    n = base.n
    N1 = len(vspace.axis_groups(n, 1))

    def state(frac):
        g1, h1 = kinetic.maxwell_gh(np.array(4.0 * (1 - frac)), np.array([0.6, 0.0]), np.array(8.0), bsp.xi, GAS)
        g2, h2 = kinetic.maxwell_gh(np.array(4.0 * frac), np.array([5.92, 0.0]), np.array(1.0), bsp.xi, GAS)
        return g1 + g2, h1 + h2

    def space(frac):
        g, h = state(frac)
        k = criterion.criterion_2d(g.reshape(n, n), h.reshape(n, n), base, np.zeros((N1, N1), dtype=np.int64),
                                   0.01, 0.005, eps_merge=None, max_level=3)
        return vspace.kappa_space(base, k)

    return bsp, state, space(0.2), space(0.05)


def _vt(sp):
    return np.ascontiguousarray(np.stack([sp.xi[:, 0], sp.xi[:, 1], sp.w, np.ones_like(sp.w)]))


def _csr(src, dst):
    P = mapping.projection_matrix(src, dst)
    off = np.zeros(dst.nv + 1, dtype=np.int32)
    idx, wgt = [], []
    for i in range(dst.nv):
        nz = np.nonzero(P[i])[0]
        idx += list(nz)
        wgt += list(P[i, nz])
        off[i + 1] = len(idx)
    return off, np.asarray(idx, dtype=np.int32), np.asarray(wgt, dtype=np.float64)


def _run(lib, A, B, gA, hA, gl, hl, fn="emu_expmap"):
    off, idx, wgt = _csr(A, B)
    sv, tv = _vt(A), _vt(B)
    src = np.ascontiguousarray(np.concatenate([gA, hA]))
    dst = np.ascontiguousarray(np.concatenate([gl, hl]))
    code = getattr(lib, fn)(A.nv, sv.ctypes.data, B.nv, tv.ctypes.data, off.ctypes.data, idx.ctypes.data,
                            wgt.ctypes.data, src.ctypes.data, dst.ctypes.data)
    return code, dst[:B.nv], dst[B.nv:]


def _remap(A, B, gA, hA):
    m = kinetic.moments(gA, hA, A.xi, A.w, GAS)
    tar = np.concatenate([[m["rho"]], m["rho"] * m["u"], [m["rhoE"]]])
    gp, hp = mapping.project(gA, hA, A, B)
    gl, hl = mapping.correct4(gp, hp, tar, m["T"], B, GAS)
    return gp, hp, gl, hl, tar


@pytest.mark.parametrize("frac", [0.2, 0.1, 0.05])
def test_negative_additive_remaps_become_the_exponential_correction(lib, spaces, frac):
    bsp, state, A, B = spaces
    gA, hA = mapping.project(*state(frac), bsp, A)              # a positive state on A
    assert gA.min() >= 0.0
    gp, hp, gl, hl, tar = _remap(A, B, gA, hA)
    assert gl.min() < 0.0 <= gp.min()                           # the case the fallback is for
    ge, he = mapping.correct_exp4(gp, hp, tar, B)
    code, g, h = _run(lib, A, B, gA, hA, gl, hl)
    assert code == 1
    np.testing.assert_allclose(g, ge, rtol=0, atol=1e-12 * np.max(ge))
    np.testing.assert_allclose(h, he, rtol=0, atol=1e-12 * np.max(he))
    assert g.min() >= 0.0


def test_positive_additive_result_is_kept(lib, spaces):
    bsp, state, A, B = spaces
    gA, hA = mapping.project(*state(0.1), bsp, A)
    gp, hp, gl, hl, _ = _remap(A, B, gA, hA)
    gl, hl = np.abs(gl), np.abs(hl)                             # a result without negative values
    code, g, h = _run(lib, A, B, gA, hA, gl, hl)
    assert code == 0
    np.testing.assert_array_equal(g, gl)
    np.testing.assert_array_equal(h, hl)


def test_negative_projection_keeps_the_additive_result(lib, spaces):
    bsp, state, A, B = spaces
    gA, hA = mapping.project(*state(0.1), bsp, A)
    gA = gA.copy()
    gA[np.argmin(gA)] = -1e-3 * gA.max()                        # a source that is already negative
    gp, hp, gl, hl, _ = _remap(A, B, gA, hA)
    assert gp.min() < 0.0
    code, g, _ = _run(lib, A, B, gA, hA, gl, hl)
    assert code == 0
    np.testing.assert_array_equal(g, gl)


@pytest.mark.parametrize("frac", [0.2, 0.05])
@pytest.mark.parametrize("direction", ["A_to_B", "B_to_A"])
def test_nine_moment_mapping_matches_the_oracle(lib, spaces, frac, direction):
    bsp, state, A, B = spaces
    if direction == "B_to_A":
        A, B = B, A
    gA, hA = mapping.project(*state(frac), bsp, A)
    ge, he = mapping.map9(gA, hA, A, B)
    code, g, h = _run(lib, A, B, gA, hA, np.zeros(B.nv), np.zeros(B.nv), fn="emu_map9")
    assert code == 1
    np.testing.assert_allclose(g, ge, rtol=0, atol=1e-12 * np.max(np.abs(ge)))
    np.testing.assert_allclose(h, he, rtol=0, atol=1e-12 * np.max(np.abs(he)))
    R0, R1 = mapping.raw9(gA, hA, A), mapping.raw9(g, h, B)
    np.testing.assert_allclose(R1, R0, rtol=0, atol=1e-12 * np.max(np.abs(R0)))
