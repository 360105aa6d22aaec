// Runs the library's Cartesian single-level step on the CPU: the tile kernels (k_faces: the
// face phi-bar into the face buffer and the face sums; k_update: the update from the face
// buffer) on emulated thread blocks (a block's threads as std::threads, a std::barrier for
// __syncthreads, per-warp exchanges for the shuffles, the dynamic shared memory as one buffer
// for the running block), with the initialisation, chunk-sum and finalisation kernels around
// them in the order the handle launches them for a level that holds every cell.  The level's
// space is the uniform base space, or a space cut from the base grid by a coarsening mask:
// then the finalisation takes the split path (state per thread, the velocity sums per warp
// from the space's row tables, the correction per thread), with the four- or eight-moment
// correction.  `split` sends the uniform space's finalisation down the split path as well
// (its velocity sums: one-axis sums over the lanes), as the handle does for small launches.  FP64 storage, or FP32 when compiled with EMU_FP32.  Test infrastructure.
#define EMU_SHARED_SPEC
#include "cta_shim.hpp"

namespace mlvs {
alignas(16) unsigned char smem[256 * 1024];   // the dynamic shared memory of the running block
alignas(16) unsigned char fsm[128 * 1024];    // that of the split finalisation's velocity sums
alignas(16) unsigned char fsm8[128 * 1024];   // (its eight-moment form)
}

#include "../../paper_2609_35258_b300/csrc/dugks_tile.cuh"
#include "../../paper_2609_35258_b300/csrc/finalize.cuh"
#include "../../paper_2609_35258_b300/csrc/mapping.cuh"
#include "../../paper_2609_35258_b300/csrc/vspace_host.hpp"

#include <algorithm>
#include <map>
#include <set>
#include <stdexcept>

using namespace mlvs;
#ifdef EMU_FP32
using T = float;
using S = float;
#else
using T = double;
using S = double;
#endif
constexpr int D = 2, TX = 16, TY = 16, VPC = 384, FIN_BLOCK = 64;

extern "C" int emu_tile_run(int nx, int ny, double Lx, double Ly, const int* bc, const double* wall,
                            const double* gas6, int n_base, double umin, double umax, int rule, double dt,
                            int compat_cell, int compat_face, int limiter, const double* far, const double* W0,
                            int steps, int vpc, const unsigned char* kappa /* [N1*N1] or null */,
                            int compat_moments, int split, double* fout /* [2][nv][ncell] */, int* nv_out) {
  const Base1D b = make_base_1d(n_base, umin, umax, rule);
  const int N1 = (int)groups_1d(n_base, 1).size();
  std::vector<int> keff(N1 * N1, 0), owner;
  if (kappa) {
    std::vector<int> kap(kappa, kappa + N1 * N1);
    keff = enforce_consistency(kap, n_base, D);
  }
  const VSpace vs = kappa_vspace(b, D, keff, owner);
  const bool cut = !std::all_of(keff.begin(), keff.end(), [](int x) { return x == 0; });
  const bool c8 = compat_moments == 8;
  const int nv = vs.nv();
  *nv_out = nv;
  std::vector<T> vt(4 * (size_t)nv), ax;
  for (int v = 0; v < nv; ++v) {
    vt[v] = vs.xix[v]; vt[nv + v] = vs.xiy[v]; vt[2 * nv + v] = vs.wx[v]; vt[3 * nv + v] = vs.wy[v];
  }
  if (!cut) {
    auto gr = groups_1d(n_base, 0);
    ax.resize(2 * gr.size());
    for (size_t g = 0; g < gr.size(); ++g) {
      double X, Wg;
      merged(b, gr[g].first, gr[g].second, X, Wg);
      ax[g] = T(X);
      ax[gr.size() + g] = T(Wg);
    }
  }
  // row tables of a cut space (entries: distinct (level, axis range) of the points, in
  // (level, range) order; a row per y entry, its x entries in segments of one level, as
  // positions in the per-level prefix sums, each level's block led by one zero slot)
  std::vector<T> e1;
  std::vector<int> lst(5, 0);
  std::vector<int4> rows;
  std::vector<int2> segs;
  int n1 = 0;
  if (cut) {
    std::map<std::pair<int, int>, int> level_of;
    for (int L = 3; L >= 0; --L)
      for (const auto& g : groups_1d(n_base, L)) level_of[g] = L;
    std::set<std::pair<int, std::pair<int, int>>> used;
    for (int v = 0; v < vs.nv(); ++v)
      for (int d = 0; d < 2; ++d) {
        const std::pair<int, int> r(vs.rect[4 * v + 2 * d], vs.rect[4 * v + 2 * d + 1]);
        used.insert({level_of.at(r), r});
      }
    std::map<std::pair<int, int>, int> ent;
    std::vector<int> lvl;
    std::vector<double> ex, ew;
    for (const auto& u : used) {
      ent[u.second] = (int)ex.size();
      lvl.push_back(u.first);
      double X, Wg;
      merged(b, u.second.first, u.second.second, X, Wg);
      ex.push_back(X);
      ew.push_back(Wg);
      for (int L = u.first + 1; L <= 4; ++L) lst[L] = (int)ex.size();
    }
    n1 = (int)ex.size();
    std::map<int, std::vector<int>> row_of;
    for (int v = 0; v < vs.nv(); ++v)
      row_of[ent.at({vs.rect[4 * v + 2], vs.rect[4 * v + 3]})].push_back(ent.at({vs.rect[4 * v], vs.rect[4 * v + 1]}));
    for (auto& r : row_of) {
      std::vector<int>& xs = r.second;
      std::sort(xs.begin(), xs.end());
      const int first = (int)segs.size();
      for (size_t i = 0; i < xs.size();) {
        size_t j = i + 1;
        while (j < xs.size() && xs[j] == xs[j - 1] + 1 && lvl[xs[j]] == lvl[xs[i]]) ++j;
        const int L = lvl[xs[i]];
        segs.push_back(make_int2(xs[i] + L, xs[j - 1] + 1 + L));
        i = j;
      }
      rows.push_back(make_int4(r.first, first, (int)segs.size() - first, 0));
    }
    e1.resize(2 * (size_t)n1);
    for (int e = 0; e < n1; ++e) { e1[e] = T(ex[e]); e1[n1 + e] = T(ew[e]); }
  }
  const int ncell = nx * ny;
  const int px = bc[0] == 0, py = bc[2] == 0;
  const int nfx = px ? nx : nx + 1, nfy = py ? ny : ny + 1, nface = nfx * ny + nx * nfy;
  StepConst k;
  std::memset(&k, 0, sizeof(k));
  k.nx = nx; k.ny = ny; k.px = px; k.py = py;
  for (int s = 0; s < 4; ++s) k.bc[s] = bc[s];
  k.nfx = nfx; k.nfy = nfy; k.ncell = ncell; k.nface = nface;
  k.nv = nv; k.nax = (int)ax.size() / 2;
  k.dx = Lx / nx; k.dy = Ly / ny; k.dt = dt;
  k.c0 = gas6[1] + 3.0 - D; k.twoK = 2.0 * gas6[1];
  k.vpc = vpc; k.nchunk = (nv + vpc - 1) / vpc;
  GasDev gas{gas6[0], gas6[1], gas6[2], gas6[3], gas6[4], gas6[5]};
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntiles = ntx * nty;
  std::vector<int> tiles(ntiles), ids(ncell), lvl(ncell, 0), slot(ncell), gho(ncell, -1), fslot(nface, -1);
  for (int i = 0; i < ntiles; ++i) tiles[i] = i;
  for (int c = 0; c < ncell; ++c) ids[c] = slot[c] = c;
  std::vector<unsigned char> frole(nface, FR_NORMAL);
  std::vector<T> f[2] = {std::vector<T>(2 * (size_t)nv * ncell), std::vector<T>(2 * (size_t)nv * ncell)};
  std::vector<T> prm[2] = {std::vector<T>((size_t)NP * ncell), std::vector<T>((size_t)NP * ncell)};
  std::vector<T> fprm((size_t)NP * nface, 0.0), ucell(2 * (size_t)ncell);
  std::vector<double> cpart((size_t)k.nchunk * NMOM * ncell), fpart((size_t)k.nchunk * NMOM * nface);
  std::vector<double> msum((size_t)NMOM * std::max(nface, ncell)), W(11 * (size_t)ncell);
  const int np = std::max(nface, ncell);
  std::vector<double> scr((size_t)(c8 ? FIN_SCR8 : FIN_SCR) * np);
  std::vector<int> need(np);
  std::vector<T> prm8[2] = {std::vector<T>(4 * (size_t)ncell, T(0)), std::vector<T>(4 * (size_t)ncell, T(0))};
  std::vector<T> fprm8(4 * (size_t)nface, T(0));
  int err_words[ERR_WORDS] = {0};
  int& err = err_words[0];
  unsigned stepctr = 0;
  auto pargs = [&](bool face) {
    PointArgs a;
    std::memset(&a, 0, sizeof(a));
    a.k = k; a.gas = gas; a.is_face = face; a.npt = face ? nface : ncell; a.pts = nullptr;
    a.nwork = a.npt; a.part = face ? fpart.data() : cpart.data(); a.vt = vt.data(); a.ax = ax.data();
    a.ids = ids.data(); a.frole = frole.data(); a.ucell = ucell.data();
    a.compat = face ? compat_face : compat_cell;
    for (int s = 0; s < 4; ++s)
      for (int j = 0; j < 3; ++j) a.wall[s][j] = wall[3 * s + j];
    for (int j = 0; j < 4; ++j) a.far[j] = far[j];
    a.err = err_words;
    if (cut) {
      a.e1 = e1.data(); a.n1 = n1; a.lst = lst.data(); a.rows = rows.data(); a.nrows = (int)rows.size();
      a.segs = segs.data();
    }
    return a;
  };
  auto fin_grid = [](int n) { return dim3(std::max(1, (n + FIN_BLOCK - 1) / FIN_BLOCK), 1, 1); };
  auto finalize = [&](PointArgs a) {
    const long nt = (long)NMOM * a.nwork;
    emu_launch(dim3((unsigned)((nt + 255) / 256), 1, 1), 256,
               [&] { k_sum_chunks(a.part, a.k.nchunk, a.npt, a.pts, a.nwork, msum.data()); });
    a.msum = msum.data();
    if (!cut && !split) {   // split: the split path on the tensor-product space too
      emu_launch(fin_grid(a.nwork), FIN_BLOCK, [&] { k_finalize<T, D>(a); });
      return;
    }
    a.scr = scr.data();
    a.need = need.data();
    emu_launch(fin_grid(a.nwork), FIN_BLOCK, [&] { k_fin_pre<T, D>(a); });
    const unsigned gs = (unsigned)std::max(1, (a.nwork * 32 + 127) / 128);
    if ((size_t)4 * row_smem_values(a.n1, c8 ? 10 : 8) * sizeof(T) > sizeof(fsm)) throw std::runtime_error("fsm");
    if (c8) {
      emu_launch(dim3(gs, 1, 1), 128, [&] { k_fin_sums<T, D, true>(a); });
      emu_launch(fin_grid(a.nwork), FIN_BLOCK, [&] { k_fin_post<T, D, true>(a); });
    } else {
      emu_launch(dim3(gs, 1, 1), 128, [&] { k_fin_sums<T, D>(a); });
      emu_launch(fin_grid(a.nwork), FIN_BLOCK, [&] { k_fin_post<T, D>(a); });
    }
  };
  // initial state (as the handle's init: parameters, phi~, velocities, chunk moments)
  int cur = 0, pcur = 0;
  {
    PointArgs a = pargs(false);
    a.prm_out = prm[0].data();
    emu_launch(fin_grid(ncell), FIN_BLOCK, [&] { k_init_params<T, D>(a, W0); });
    emu_launch(dim3((ncell + 127) / 128, std::min(nv, 1024), 1), 128,
               [&] { k_init_f<S, T, D>(k, ncell, prm[0].data(), vt.data(), f[0].data()); });
    emu_launch(dim3((ncell + 127) / 128, 1, 1), 128,
               [&] { k_scatter_velocity<T>(prm[0].data(), ncell, ids.data(), ucell.data(), ncell); });
    emu_launch(dim3((ncell + 127) / 128, 1, 1), 128,
               [&] { k_set_shift<T>(prm[0].data(), ncell, ids.data(), ucell.data(), ncell); });
    emu_launch(dim3((ncell + 127) / 128, k.nchunk, 1), 128,
               [&] { k_moments<S, T, D>(k, ncell, prm[0].data(), vt.data(), f[0].data(), cpart.data()); });
  }
  using L0 = TileSmem<T, TX, TY, D>;
  using L1 = UpdSmem<T, TX, TY, D, VPC>;
  if (L0::BYTES > sizeof(smem) || L1::BYTES > sizeof(smem) || vpc > VPC || vpc % 2) return 2;
  std::vector<T> fbar(2 * (size_t)((nv + 1) / 2) * 2 * nface, 0.0);
  for (int s = 0; s < steps; ++s) {
    {
      PointArgs a = pargs(false);
      a.cprm = prm[pcur].data();
      a.prm_out = prm[pcur ^ 1].data();
      a.W = W.data();
      if (c8) a.prm8_out = prm8[pcur ^ 1].data();
      finalize(a);
      emu_launch(dim3((ncell + 127) / 128, 1, 1), 128,
                 [&] { k_scatter_velocity<T>(prm[pcur ^ 1].data(), ncell, ids.data(), ucell.data(), ncell); });
      pcur ^= 1;
    }
    TileArgs t;
    std::memset(&t, 0, sizeof(t));
    t.k = k; t.f_in = f[cur].data(); t.f_out = f[cur ^ 1].data(); t.nslot = ncell;
    t.cparam = prm[pcur].data(); t.fparam = fprm.data(); t.vt = vt.data(); t.tiles = tiles.data();
    t.ntx = ntx; t.nty = nty; t.level = 0; t.lvl_of = lvl.data(); t.slot_of = slot.data();
    t.ghost_of = nullptr; t.ghost = nullptr; t.nghost = 0; t.frole = frole.data(); t.fslot = fslot.data();
    t.ucell = ucell.data(); t.step = &stepctr; t.fbar = fbar.data();
    t.part = fpart.data();
    t.cparam8 = prm8[pcur].data();
    t.fparam8 = fprm8.data();
    if (c8)
      emu_launch(dim3(ntiles, k.nchunk, 1), TX * TY,
                 [&] { k_faces<S, T, D, TX, TY, false, false, true>(t, nullptr, nullptr, limiter); });
    else
      emu_launch(dim3(ntiles, k.nchunk, 1), TX * TY,
                 [&] { k_faces<S, T, D, TX, TY, false, false>(t, nullptr, nullptr, limiter); });
    {
      PointArgs a = pargs(true);
      a.cprm = prm[pcur].data();
      a.prm_out = fprm.data();
      if (c8) a.prm8_out = fprm8.data();
      finalize(a);
    }
    t.part = cpart.data();
    if (c8)
      emu_launch(dim3(ntiles, k.nchunk, 1), TX * TY,
                 [&] { k_update<S, T, D, TX, TY, VPC, false, false, true>(t, nullptr, nullptr); });
    else
      emu_launch(dim3(ntiles, k.nchunk, 1), TX * TY,
                 [&] { k_update<S, T, D, TX, TY, VPC, false, false>(t, nullptr, nullptr); });
    cur ^= 1;
  }
  for (size_t i = 0; i < f[cur].size(); ++i) fout[i] = (double)f[cur][i];
  return err;
}

// The per-warp shared-memory layout of the finalisation's row sums, for the layout tests.
extern "C" int emu_row_smem_values(int n1, int NO) { return row_smem_values(n1, NO); }
extern "C" int emu_row_pd(int NO) { return row_pd(NO); }
