"""The library's unstructured-step passes run on the CPU against the oracle's unstructured step.
The per-element functions the CUDA kernels loop over, and the same step sequence, are
compiled as host C++ (tests/emu).  Cases:
  * two-cavity meshes of quads and of triangles at the paper's density ratio of 1000, FP64;
  * a quad cavity with a moving lid, a second wall index, FP64;
  * the triangulated two-cavity mesh in FP32;
  * the eight-moment compatibility correction at cells and faces (FP64 and FP32), which the
    four-moment run differs from by far more than the bound;
  * one run under AddressSanitizer, which checks every buffer access of every pass.
Velocity sums run in a different order than the oracle's and the FP32 case rounds every
operation, so the bounds are 1e-12 (FP64) and 1e-5 (FP32) of the largest value (measured:
1.3e-15 and 1.1e-6)."""
import ctypes as C
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from oracle import dugks, kinetic, unstructured as un, vspace
from paper_2609_35258_b300 import mlvs as M
from paper_2609_35258_b300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
EMU = os.path.join(HERE, "emu")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def _compile(asan, contract=False):
    """contract: let the compiler fuse a * b + c into one rounding, as nvcc does for device
    code, so that a sign decision that depends on an unfused product shows up on the CPU."""
    out = os.path.join(tempfile.mkdtemp(prefix="ustep_emu_"), "emu.so")
    flags = ["-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer"] if asan else ["-O2"]
    if contract:
        flags += ["-mfma", "-ffp-contract=off", "-DEMU_CONTRACT"]
    cmd = ["g++", "-std=c++17", *flags, "-fPIC", "-shared", "-I", CUDA_INC,
           os.path.join(EMU, "ustep_emu.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _bind(path):
    lib = C.CDLL(path)
    lib.emu_create.restype = C.c_void_p
    lib.emu_create.argtypes = [C.POINTER(M.mlvs_uconfig), C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_char_p, C.c_int]
    lib.emu_step.argtypes = [C.c_void_p, C.c_int]
    lib.emu_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.emu_dt.restype = C.c_double
    lib.emu_dt.argtypes = [C.c_void_p]
    lib.emu_nv.argtypes = [C.c_void_p]
    lib.emu_destroy.argtypes = [C.c_void_p]
    return lib


@pytest.fixture(scope="module")
def emu():
    return _bind(_compile(asan=False))


GAS = kinetic.Gas(D=2, R=1.0, Pr=2.0 / 3.0, omega=0.81, mu_ref=kinetic.mu_ref_from_kn(0.05, 0.81), T_ref=1.0)


def _cfg(storage, walls, n_base=13, umax=5.0, limiter=M.LIMITER_VENKAT, vpc=32):
    c = M.mlvs_uconfig()
    c.storage = storage
    c.R, c.K_internal, c.Pr, c.omega, c.mu_ref, c.T_ref = GAS.R, GAS.K, GAS.Pr, GAS.omega, GAS.mu_ref, GAS.T_ref
    c.cfl, c.dt = 0.5, 0.0
    c.compat_cell = c.compat_face = 1
    c.limiter = limiter
    c.n_base, c.umin, c.umax, c.quadrature = n_base, -umax, umax, M.QUAD_BOOLE
    c.n_wall = len(walls)
    for k, w in enumerate(walls):
        for j in range(3):
            c.wall[k][j] = w[j]
    c.vpc = vpc
    return c


def _run_emu(lib, cfg, nodes, cells, W0, steps, edge_wall=None):
    xy = np.ascontiguousarray(nodes, dtype=np.float64)
    ptr, cn, ew = M.umesh_arrays(cells, edge_wall)
    W0 = np.ascontiguousarray(W0, dtype=np.float64)
    msg = C.create_string_buffer(256)
    e = lib.emu_create(C.byref(cfg), len(xy), xy.ctypes.data, len(cells), ptr.ctypes.data, cn.ctypes.data,
                       None if ew is None else ew.ctypes.data, W0.ctypes.data, msg, 256)
    assert e, msg.value.decode()
    try:
        assert lib.emu_step(e, steps) == 0
        nv = lib.emu_nv(e)
        g, h = np.zeros((len(cells), nv)), np.zeros((len(cells), nv))
        lib.emu_read(e, g.ctypes.data, h.ctypes.data)
        return g, h, lib.emu_dt(e)
    finally:
        lib.emu_destroy(e)


def _run_oracle(mesh, W0, steps, n_base=13, umax=5.0, limiter="venkat", nmom=4):
    sp = vspace.uniform_space(vspace.make_base(n_base, -umax, umax, D=2), 0)
    g, h = dugks.initial_tilde(W0[:, 0], W0[:, 1:3], W0[:, 3], sp.xi, sp.w, GAS)
    dt = un.time_step(mesh, sp.xi, 0.5)
    for _ in range(steps):
        g, h, _ = un.step(g, h, mesh, sp.xi, sp.w, GAS, dt, dugks.Options(compat_moments=nmom), limiter=limiter)
    return g, h, dt


def _two_cavity(tri):
    nodes, cells = workloads.two_cavities(2)
    if tri:
        nodes, cells = workloads.triangulate(nodes, cells)
    mesh = un.UMesh(nodes, cells)
    cen = un.geometry(mesh)["cen"]
    W0 = np.zeros((len(cells), 4))
    W0[:, 0] = np.where(cen[:, 0] < 0.0, 1.0, 1e-3)
    W0[:, 3] = 1.0
    return nodes, cells, mesh, W0


@pytest.fixture(scope="module")
def emu_fma():
    return _bind(_compile(asan=False, contract=True))


@pytest.mark.parametrize("tri", [False, True], ids=["quads", "triangles"])
@pytest.mark.parametrize("contract", [False, True], ids=["ieee", "fma"])
def test_two_cavities_fp64_match_the_oracle(emu, emu_fma, tri, contract):
    """The "fma" build contracts products into fused multiply-adds wherever the source leaves
    it free to, as the GPU build does.  The triangles' diagonal faces have n = (1, -1)/sqrt(2),
    so velocities with xi_x = xi_y are tangential to them: xi.n must come out as an exact zero
    (the mean of both sides), which a fused product would turn into a rounding residue whose
    sign picks one side."""
    nodes, cells, mesh, W0 = _two_cavity(tri)
    g, h, dt = _run_emu(emu_fma if contract else emu, _cfg(M.F64, [(0.0, 0.0, 1.0)]), nodes, cells, W0, 3)
    go, ho, dto = _run_oracle(mesh, W0, 3)
    assert dt == pytest.approx(dto, rel=1e-15)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-12 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-12 * np.max(np.abs(ho)))
    assert np.max(np.abs(g - dugks.initial_tilde(W0[:, 0], W0[:, 1:3], W0[:, 3], *_space(), GAS)[0])) > 1e-3


def _space(n_base=13, umax=5.0):
    sp = vspace.uniform_space(vspace.make_base(n_base, -umax, umax, D=2), 0)
    return sp.xi, sp.w


def test_lid_driven_quads_with_two_walls_match_the_oracle(emu):
    n = 8
    nodes, cells = workloads.quad_mesh(np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1))
    walls = [(0.0, 0.0, 1.0), (0.4, 0.0, 1.0)]
    top = lambda mid: 1 if mid[1] > 1.0 - 1e-9 else 0
    mesh = un.UMesh(nodes, cells, wall_of=top, wall=tuple(walls))
    edge_wall = [[top(0.5 * (nodes[c[k]] + nodes[c[(k + 1) % 4]])) for k in range(4)] for c in cells]
    W0 = np.tile([1.0, 0.0, 0.0, 1.0], (len(cells), 1))
    g, h, _ = _run_emu(emu, _cfg(M.F64, walls), nodes, cells, W0, 3, edge_wall)
    go, ho, _ = _run_oracle(mesh, W0, 3)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-12 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-12 * np.max(np.abs(ho)))
    xi, w = _space()
    u = np.sum(w * g * xi[:, 0], axis=1) / np.sum(w * g, axis=1)
    assert u.max() > 1e-3                                        # the lid drags the gas along


def test_unlimited_gradients_match_the_oracle(emu):
    nodes, cells, mesh, W0 = _two_cavity(True)
    W0[:, 0] = np.where(mesh.geo["cen"][:, 0] < 0.0, 1.0, 0.5)
    g, h, _ = _run_emu(emu, _cfg(M.F64, [(0.0, 0.0, 1.0)], limiter=M.LIMITER_NONE), nodes, cells, W0, 2)
    go, ho, _ = _run_oracle(mesh, W0, 2, limiter="none")
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-12 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-12 * np.max(np.abs(ho)))


def test_two_cavities_fp32_match_the_oracle(emu):
    nodes, cells, mesh, W0 = _two_cavity(True)
    g, h, _ = _run_emu(emu, _cfg(M.F32, [(0.0, 0.0, 1.0)]), nodes, cells, W0, 3)
    go, ho, _ = _run_oracle(mesh, W0, 3)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-5 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-5 * np.max(np.abs(ho)))


CHILD = r"""
import ctypes as C, sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from tests import test_ustep_emu as T
lib = T._bind(sys.argv[1])
nodes, cells, mesh, W0 = T._two_cavity(True)
for st in (T.M.F64, T.M.F32):
    T._run_emu(lib, T._cfg(st, [(0.0, 0.0, 1.0)], n_base=9, vpc=20), nodes, cells, W0, 2)
print("clean")
"""


def test_every_pass_stays_inside_its_buffers_under_address_sanitizer():
    so = _compile(asan=True)
    libasan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan):
        pytest.skip("libasan is not available to preload")
    env = dict(os.environ, LD_PRELOAD=libasan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0")
    root = os.path.dirname(HERE)
    r = subprocess.run([sys.executable, "-c", CHILD, so, root], env=env, capture_output=True, text=True,
                       timeout=600, cwd=root)
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-3000:]


def test_knudsen_number_gives_the_oracles_reference_viscosity(emu):
    """mu_ref <= 0 with Kn set: the library's VHS relation gives the oracle's mu_ref, so the
    run equals the one with mu_ref given."""
    nodes, cells, _, W0 = _two_cavity(True)
    by_mu = _cfg(M.F64, [(0.0, 0.0, 1.0)])
    by_kn = _cfg(M.F64, [(0.0, 0.0, 1.0)])
    by_kn.mu_ref, by_kn.Kn = 0.0, 0.05
    a = _run_emu(emu, by_mu, nodes, cells, W0, 2)
    b = _run_emu(emu, by_kn, nodes, cells, W0, 2)
    np.testing.assert_allclose(b[0], a[0], rtol=0, atol=1e-14 * np.max(np.abs(a[0])))


@pytest.mark.parametrize("storage,tol", [(M.F64, 1e-12), (M.F32, 1e-5)], ids=["f64", "f32"])
def test_eight_moment_correction_matches_the_oracle(emu, storage, tol):
    nodes, cells, mesh, W0 = _two_cavity(True)
    cfg = _cfg(storage, [(0.0, 0.0, 1.0)])
    cfg.compat_moments = 8
    g, h, _ = _run_emu(emu, cfg, nodes, cells, W0, 3)
    go, ho, _ = _run_oracle(mesh, W0, 3, nmom=8)
    np.testing.assert_allclose(g, go, rtol=0, atol=tol * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=tol * np.max(np.abs(ho)))
    g4, _, _ = _run_oracle(mesh, W0, 3, nmom=4)
    assert np.max(np.abs(g4 - go)) > 10 * tol * np.max(np.abs(go))


@pytest.mark.parametrize("shape", ["square", "triangle"])
def test_single_cell_closed_box_matches_the_oracle(emu, shape):
    """The degenerate mesh of one cell: every face a wall, the least-squares matrix from the
    reflected ghosts alone (all gradients zero), a gas off equilibrium relaxing in the box."""
    if shape == "square":
        nodes, cells = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]]), [(0, 1, 2, 3)]
    else:
        nodes, cells = np.array([[0.0, 0.0], [1.0, 0.0], [0.3, 0.8]]), [(0, 1, 2)]
    mesh = un.UMesh(nodes, cells)
    W0 = np.array([[1.2, 0.3, -0.2, 1.4]])
    g, h, _ = _run_emu(emu, _cfg(M.F64, [(0.0, 0.0, 1.0)]), nodes, cells, W0, 3)
    go, ho, _ = _run_oracle(mesh, W0, 3)
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-12 * np.max(np.abs(go)))
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-12 * np.max(np.abs(ho)))
