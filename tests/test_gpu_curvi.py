"""Structured curvilinear meshes (the O-grid of the cylinder configuration), through the
C ABI, against the oracle's curvilinear step.

* On a Cartesian node grid the curvilinear path reproduces the Cartesian path (the geometry
  reduces exactly; only the flux scaling dt/|V| |S| rounds differently).
* On small O-grids (wall inside, freestream outside) the library matches the oracle
  (FP64 1e-10, FP32 1e-5) and the wall carries no net mass flux.
* The cylinder configuration at full size (256 x 128 cells, 201^2 velocities) in FP32 and
  BF16: the flow stays mirror-symmetric about the x axis, and BF16 stays within 1e-3 of FP32.
* Two velocity spaces on a small O-grid against the oracle's curvilinear multi-level step, and
  adapted spaces on a closed annulus conserving mass.
"""
import numpy as np
import pytest

from tests.helpers import have_gpu, oracle_moments, oracle_run, oracle_setup
from paper_2609_35258_b300 import workloads

pytestmark = pytest.mark.gpu

if not have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_35258_b300 import mlvs as M  # noqa: E402
from paper_2609_35258_b300.solver import Solver  # noqa: E402


def _with_nodes(desc):
    d = dict(desc)
    nx, ny = d["nx"], d["ny"]
    X, Y = np.meshgrid(np.arange(nx + 1) * d["Lx"] / nx, np.arange(ny + 1) * d["Ly"] / ny)
    d["nodes"] = np.stack([X, Y], axis=-1)
    return d


@pytest.mark.parametrize("kind", ["periodic", "cavity", "channel"])
def test_cartesian_nodes_reproduce_cartesian_path(kind):
    if kind == "periodic":
        desc = workloads.periodic_random(20, 12, n_base=25, storage="f64")
    elif kind == "cavity":
        desc = workloads.cavity(16, n_base=25, storage="f64")
    else:
        desc = workloads.supersonic_channel(24, 8, n_base=25, umax=8.0, storage="f64", walls=True)
    a = Solver(desc)
    b = Solver(_with_nodes(desc))
    assert abs(a.dt - b.dt) < 1e-13 * a.dt
    a.step(6)
    b.step(6)
    ma, mb = a.moments(), b.moments()
    assert np.max(np.abs(ma - mb)) < 1e-12 * np.max(np.abs(ma))


def _kappa_pair(n_base):
    """Two masked spaces, fine near the origin and coarser towards +x (a) or +y (b)."""
    from oracle import vspace
    N1 = len(vspace.axis_groups(n_base, 1))
    yy, xx = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    r = np.hypot(xx - N1 // 2, yy - N1 // 2)
    a = np.where(r < N1 / 4, 0, np.where(xx > N1 // 2, 2, 1)).astype(np.uint8)
    b = np.where(r < N1 / 4, 0, np.where(yy > N1 // 2, 2, 1)).astype(np.uint8)
    return a, b


@pytest.mark.parametrize("kind", ["cavity", "channel"])
def test_cartesian_nodes_reproduce_cartesian_multilevel(kind):
    """Three spaces (uniform level 0 and two masked ones) on a checkerboard of 4x4 cell
    blocks: walls, freestream sides, cross-level faces and ghosts on the curvilinear path
    give the Cartesian multi-level result."""
    if kind == "cavity":
        desc = workloads.cavity(16, n_base=25, storage="f64")
    else:
        desc = workloads.supersonic_channel(24, 8, n_base=25, umax=8.0, storage="f64", walls=True)
    ka, kb = _kappa_pair(25)
    nx, ny = desc["nx"], desc["ny"]
    lev = np.array([((i // 4) + 2 * (j // 4)) % 3 for j in range(ny) for i in range(nx)], dtype=np.int32)
    runs = []
    for d in (desc, _with_nodes(desc)):
        s = Solver(d, levels=(0, ka, kb))
        M.mlvs_set_cell_levels(s.h, 0, lev)
        s.step(6)
        runs.append(s.moments())
        s.close()
    ma, mb = runs
    assert np.max(np.abs(ma - mb)) < 1e-12 * np.max(np.abs(ma))
    assert np.max(np.abs(ma[0] - 1.0)) > 1e-4                # the flow developed


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_ogrid_matches_oracle(storage, tol):
    desc = workloads.cylinder(24, 8, mach=2.0, Kn=0.1, n_base=25, umax=8.0, r_out=4.0, storage=storage)
    o = oracle_setup(desc)
    s = Solver(desc)
    assert abs(s.dt - o["dt"]) < 1e-14 * o["dt"]
    s.step(8)
    g, h = oracle_run(o, 8)
    gm, om = s.moments(), oracle_moments(o, g, h)
    rho, T = om[0], om[3]
    assert np.max(np.abs(gm[0] - rho) / rho) < tol
    assert np.max(np.abs(gm[1:3] - om[1:3])) < 10 * tol
    assert np.max(np.abs(gm[3] - T) / T) < tol
    assert np.max(np.abs(om[0] - 1.0)) > 1e-3          # the flow developed


def _mirror(f, ntheta):
    """Values of the cells mirrored about the x axis: cell i <-> cell ntheta-1-i."""
    return f.reshape(-1, ntheta)[:, ::-1].ravel()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_cylinder_full_size_symmetry(storage):
    desc = workloads.cylinder(storage=storage)           # 256 x 128 cells, 201^2, Ma 5, Kn 0.1
    s = Solver(desc)
    M.mlvs_set_graph(s.h, True)
    s.step(20)
    m = s.moments(M.RHO | M.U | M.V | M.T)
    nt = desc["nx"]
    tol = 1e-5 if storage == "f32" else 3e-3
    assert np.max(np.abs(m[0] - _mirror(m[0], nt)) / m[0]) < tol
    assert np.max(np.abs(m[1] - _mirror(m[1], nt))) < tol * 7
    assert np.max(np.abs(m[2] + _mirror(m[2], nt))) < tol * 7
    assert np.max(np.abs(m[3] - _mirror(m[3], nt)) / m[3]) < tol
    assert np.max(m[0]) > 1.05                             # a bow shock is forming


def test_selector_features_on_the_ogrid():
    from oracle import curvi, dugks, mlp as omlp
    desc = workloads.cylinder(24, 8, mach=2.0, Kn=0.1, n_base=25, umax=8.0, r_out=4.0, storage="f64")
    o = oracle_setup(desc)
    s = Solver(desc)
    s.step(4)
    g, h = oracle_run(o, 4)
    F = M.mlvs_features(s.h, 0, 24 * 8)
    st = dugks.cell_state(g, h, o["sp"].xi, o["sp"].w, o["gas"], o["dt"])
    G = curvi.geometry(o["mesh"])
    longest = np.maximum(np.maximum(G["li"][:, :-1], G["li"][:, 1:]), np.maximum(G["lj"][:-1, :], G["lj"][1:, :]))
    Fo = omlp.features_curvi(st["rho"], st["u"][..., 0], st["u"][..., 1], st["T"], st["q"][..., 0],
                             st["q"][..., 1], G["Jt"], G["area"] / longest, True, False, R=o["gas"].R,
                             T_ref=1.0, mu_ref=o["gas"].mu_ref, omega=o["gas"].omega)
    assert np.max(np.abs(F - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5
    assert np.max(Fo[:, 6]) > 1e-3            # gradients present


def test_ogrid_two_spaces_match_oracle():
    """Two spaces on a small O-grid (wall inside, freestream outside), cells switched from the
    fine space as the library does, three steps against the oracle's curvilinear multi-level
    step (FP64)."""
    from oracle import mlvs as omlvs, mlvs_curvi
    desc = workloads.cylinder(24, 8, mach=2.0, Kn=0.1, n_base=17, umax=8.0, r_out=4.0, storage="f64")
    n = 24 * 8
    lev = np.array([1 if 6 <= (c % 24) < 18 else 0 for c in range(n)], dtype=np.int32)
    o = oracle_setup(desc)
    book = omlvs.SpaceBook(o["base"])
    keys = [book.uniform(L) for L in (0, 1)]
    init = desc["init"]
    st = omlvs.MLVSState.from_primitives(o["mesh"], o["gas"], book, [keys[0]] * n, init[..., 0],
                                         init[..., 1:3], init[..., 3], o["dt"], o["opt"])
    for c in range(n):
        omlvs.remap(st, c, keys[lev[c]])
    s = Solver(desc, levels=(0, 1))
    M.mlvs_set_cell_levels(s.h, 0, lev)
    for _ in range(3):
        mlvs_curvi.step(st)
    s.step(3)
    for c in range(n):
        g, _ = s.read_cells(c, 1, 10000)
        gref = st.g[c]
        np.testing.assert_allclose(g[0], gref, rtol=0, atol=1e-9 * np.max(np.abs(gref)))
    s.close()


def test_multilevel_spaces_on_a_closed_annulus_conserve():
    """Walls inside and outside (a closed domain): adaptation to multi-level spaces and the
    steps after it keep the mass to FP64 rounding."""
    desc = workloads.cylinder(32, 10, mach=1.0, Kn=0.05, n_base=41, umax=8.0, r_out=4.0, storage="f64")
    desc["bc"] = ("periodic", "periodic", "wall", "wall")
    s = Solver(desc, adaptive=1)
    s.step(5)
    m0 = s.moments(M.RHO)[0]
    G = np.asarray(_areas(desc))
    tot0 = np.sum(m0 * G)
    st = M.mlvs_adapt(s.h, M.adapt_params(5e-3, 2.5e-3, 5e-5, 0.05, 3))
    assert st.updates_per_step < 320 * 41 * 41          # coarser spaces somewhere
    s.step(10)
    m1 = s.moments(M.RHO)[0]
    assert abs(np.sum(m1 * G) - tot0) < 1e-12 * tot0


def _areas(desc):
    from oracle import curvi
    xy = desc["nodes"]
    return curvi.geometry(curvi.CurviMesh(xy[..., 0], xy[..., 1], bc=desc["bc"]))["area"].ravel()
