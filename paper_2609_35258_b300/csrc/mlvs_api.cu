// C ABI of the MLVS-DUGKS library: handle, velocity spaces, levels and the step sequence.
//
// Every cell carries its distributions on the space of its level (Sec. 3.1-3.2).  A face is
// evaluated on the common refinement of its two cells' spaces (V^int, Sec. 3.4): on a level
// that has cells, or on a cell-less face level.  Stencil cells of another level enter a
// level's kernels as ghosts: their phi-bar-plus mapped to the level's space with the
// four-moment correction (Eq. interface_state_moment_matching).  The microflux of a
// cross-level face is mapped back to the native space of each side and corrected so that its
// mass, momentum and energy fluxes are those of the face (Eq. native_flux_moment_matching).
//
// One step (Sec. 2.2) per instance, on the handle's stream:
//   1. finalisation of the cells per level (chunk sums, then k_finalize, or k_fin_pre /
//      k_fin_sums / k_fin_post on spaces that are not tensor products): W, tau, q, model
//      parameters + compatibility correction
//   2. k_map_multi (SRC_BARP): the ghosts of every (source level, level) route in one launch
//   3. k_faces per level: face phi-bar (stored to the level's face buffer), face moment partials
//   4. finalisation of the faces each level evaluates: Eq. W_from_bar, Eq. recover_phi
//      weights, wall densities
//   5. per level, finest space first: k_update (microfluxes from the face buffer,
//      Eq. explicit_update), then
//      k_map_multi (SRC_FLUX) of its cross-level fluxes to the levels that receive them
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "../../include/mlvs.h"
#include "mlvs_internal.h"
#include "dugks_tile.cuh"
#include "finalize.cuh"
#include "mapping.cuh"
#include "criterion.cuh"
#include "map9.cuh"
#include "features.cuh"
#include "cluster_host.hpp"
#include "vspace_host.hpp"
#include "umesh_host.hpp"
#include "gas_host.hpp"

using namespace mlvs;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
  cudaError_t alloc(size_t bytes) {
    release();
    n = bytes;
    return cudaMalloc(&p, bytes ? bytes : 16);
  }
  template <class X> X* as() const { return reinterpret_cast<X*>(p); }
};

// Host vector -> new device buffer.  A copy from pageable memory returns once the source
// has been staged, so v may go out of scope right after the call.
template <class X> cudaError_t upload(DevBuf& d, const std::vector<X>& v, cudaStream_t s) {
  cudaError_t e = d.alloc(v.size() * sizeof(X));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, s);
}

// A velocity space on the base grid.
struct SpaceRt {
  std::vector<int> keff;     // consistent coarsening index per 2x2 block
  VSpace vs;
  std::vector<int> owner;    // base node -> point
  int nax = 0;               // > 0: tensor product of one axis of nax points
  DevBuf vt, ax, ainv;
  DevBuf owner_d, xid, kp_d; // criterion tables: owner, FP64 coordinates, keff (bytes)
  DevBuf geo;                // [5][nv] geometric sums of every point's rectangle
  // 2-D spaces that are not tensor products: the row tables of the finalisation's velocity
  // sums (entries [2][n1] X, W; level blocks [5]; rows; segments)
  DevBuf e1, lst, rows, segs;
  int n1 = 0, nrows = 0;
};

struct CSR {
  DevBuf off, idx, wgt;
};

// A level: the cells that carry their distributions on one space, or (real = false) a
// cell-less face level for cross-level faces whose common refinement is no cell level.
struct LevelRt {
  int space = 0;
  bool real = true;
  std::vector<int> cells;    // global cell id of every slot
  StepConst k;
  DevBuf f[2], prm[2], fprm, cpart, fpart, ids, frole, fslot, ghost_of, ghost, X, Y, tiles;
  DevBuf prm8[2], fprm8;     // eight-moment correction: b4..b7 of the cells and the faces
  DevBuf fbar;               // [2][nv][nface] face phi-bar of the faces the level evaluates
  DevBuf fscr, fneed;        // split finalisation scratch (spaces that are not tensor products)
  DevBuf wden;               // curvilinear walls: [nface] wall-Maxwellian normalisation
  DevBuf msum;               // [NMOM][max(cells, faces)] chunk sums for the finalisation
  DevBuf flist;              // faces the level evaluates (normal and cross), when not all
  DevBuf xfid;               // [nX] face id of every column of X
  std::vector<int> tiles_h;  // the tile list (host copy)
  int nflist = 0;
  int nghost = 0, nX = 0, nY = 0, ntiles = 0;
  int cur = 0, pcur = 0;
  bool fresh = false;
  std::vector<int> ghost_cells;
};

struct Route {               // mapped items from level src to level dst
  int src, dst;
  std::vector<MapItem> items;
  DevBuf items_d;
};

// Every ghost route of an instance in one launch: route arguments for each of the four
// (f, parameter) buffer parities of the source levels, and the item groups.
struct MapBatch {
  DevBuf routes[4], work;
  int nwork = 0, G = 1;
  bool ok = false;
};

struct Inst {
  std::vector<LevelRt> lv;   // cell levels first (ids 0..n_levels-1), face levels after
  std::vector<int> lvl_of, slot_of;
  DevBuf lvl_of_d, slot_of_d, ucell, W, err, stepctr;
  std::vector<Route> ghosts, fluxes;
  MapBatch gb;
  MapBatch fb;               // every flux route in one launch (only routes[0] is used)
  // multi-level instances: tile arguments [pass][buffer parity 2 cur + pcur][level]; work
  // items (level, tile list index, velocity chunk, 0) of the faces pass (every level with
  // tiles) and of the update (tiles with a cell of a cell level); cross-flux items (level,
  // first X column, first velocity pair, 0)
  DevBuf tab, wf, wu, wx;
  int nwf = 0, nwu = 0, nwx = 0;
  int n_int = 0, n_cross = 0;  // interior faces, and those between two levels (Sec. 3.5)
};

// Event pairs recorded around launches when a step is profiled.
struct Prof {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> marks;  // (phase, first event index)
  size_t used = 0;
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct mlvs_handle {
  mlvs_config cfg;
  int exp_corrected = 0, exp_failed = 0;   // positivity fallback of the last remap
  int map9_singular = 0;                    // nine-moment level switches with a singular block
  Prof prof;
  bool profiling = false;
  int launches = 0;
  std::vector<double> initW;
  cudaStream_t stream = nullptr;
  int D = 2;
  int nx = 1, ny = 1;
  double dx = 1, dy = 1, dt = 0;
  GasDev gas{};
  int tsize = 8;    // sizeof compute type
  int ssize = 4;    // sizeof storage type
  Base1D base;
  int n_base = 0;
  std::vector<SpaceRt> spaces;
  std::map<std::vector<int>, int> space_of_key;
  std::map<std::pair<int, int>, CSR> csr;
  int n_levels = 0;
  std::vector<int> level_space;   // space of every cell level
  std::vector<Inst> inst;
  // criterion tables of the base grid (2-D)
  int N1 = 0;
  int ng[4] = {0, 0, 0, 0};
  DevBuf bx_d, bw_d, g1_d, pstart_d, cstart_d, w1_d, x1_d, xx1_d, kbuf, sel_d, feat_d, prob_d;
  DevBuf crit_tb;                       // criterion: per-block transport sums, one slice per CTA
  unsigned char* kbuf_host = nullptr;   // pinned copy of the masks
  size_t kbuf_host_n = 0;
  mlvs_adapt_params adapt{};
  int adaptive = 0;          // 1: mlvs_adapt groups the masks; 0: fixed level set
  int adapt_interval = 0;
  long long steps_done = 0;
  bool ready = false;
  int sticky = MLVS_OK;
  std::string err;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ea0 = nullptr, ea1 = nullptr;
  // CUDA graphs and chunking
  unsigned long long uid = 0;     // unique per handle (graph keys)
  bool use_graph = false;
  long long epoch = 0;            // bumped whenever the level structure or chunking changes
  long long warm_epoch = -1;      // epoch of the last regular step (maps and tables exist)
  int cta_target = 148 * 4;       // CTAs per tile launch the chunking aims at (autotuned)
  // curvilinear mesh (mesh_kind 1): host geometry in FP64, device copies in the compute type
  bool curvi = false;
  std::vector<double> cgeo;       // [5][ncell]: J^{-T} (4), |V|
  std::vector<double> fgeo;       // [7][nface]: normal (2), |S|, x_b - x_L (2), x_b - x_R (2)
  double lmin = 0.0;              // smallest cell width |V| / max |S|
  DevBuf cgeo_d, fgeo_d, featgeo_d;
  std::vector<double> width;      // |V| / max |S| per cell
  std::map<std::vector<long long>, std::pair<cudaGraphExec_t, std::vector<int>>> graphs;
  // graphs of a group whose tile passes run as one launch over every handle's levels: their
  // tile-argument tables (pinned host copy and device table per step) and work lists
  struct GroupBufs {
    TileArgs* host = nullptr;   // [2 steps][2 passes][levels] (pinned; read by the graph's copies)
    DevBuf tab, wf, wu, wx;
    int nwf = 0, nwu = 0, nwx = 0;
  };
  std::map<std::vector<long long>, GroupBufs> gbufs;
  cudaStream_t cap = nullptr;     // capture stream
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> bev;   // join events, one per branch
  cudaEvent_t ev_fork = nullptr, ev_post = nullptr;
  std::vector<cudaEvent_t> ev_pre;
};

static mlvs_status fail(mlvs_handle* h, mlvs_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

#define CK_H(hh, call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(hh, MLVS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, MLVS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

unsigned hash_host(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

constexpr int kTX2 = 16, kTY2 = 16, kTX1 = 128;
constexpr int kMaxVpc = kVpcMax;   // largest velocity chunk of a tile launch
int tile_w(int D) { return D == 2 ? kTX2 : kTX1; }
int tile_h(int D) { return D == 2 ? kTY2 : 1; }


}  // namespace

// ---------------------------------------------------------------------------------------
// spaces and projection tables

// Row tables of a 2-D space that is not a tensor product (the split finalisation's velocity
// sums): entries = the distinct axis ranges of its points, each at the lowest level whose
// groups contain it, ordered by (level, first base node); rows = the points sharing a y
// entry; a row's segments = its runs of consecutive x entries of one level.  Every point lies
// in exactly one segment of its row.
static cudaError_t row_tables(mlvs_handle* h, SpaceRt& S) {
  const int n = h->n_base, nv = S.vs.nv();
  std::map<std::pair<int, int>, int> level_of;
  for (int L = 3; L >= 0; --L)
    for (const auto& g : groups_1d(n, L)) level_of[g] = L;
  std::set<std::pair<int, std::pair<int, int>>> used;   // (level, range)
  for (int v = 0; v < nv; ++v)
    for (int d = 0; d < 2; ++d) {
      const std::pair<int, int> r(S.vs.rect[4 * v + 2 * d], S.vs.rect[4 * v + 2 * d + 1]);
      auto it = level_of.find(r);
      if (it == level_of.end()) return cudaSuccess;   // not a union of level groups: direct sums
      used.insert({it->second, r});
    }
  std::map<std::pair<int, int>, int> ent;
  std::vector<int> lvl;
  std::vector<double> ex, ew;
  std::vector<int> lst(5, 0);
  for (const auto& u : used) {
    ent[u.second] = (int)ex.size();
    lvl.push_back(u.first);
    double X, W;
    merged(h->base, u.second.first, u.second.second, X, W);
    ex.push_back(X);
    ew.push_back(W);
    for (int L = u.first + 1; L <= 4; ++L) lst[L] = (int)ex.size();
  }
  const int n1 = (int)ex.size();
  std::map<int, std::vector<int>> row_of;   // y entry -> x entries
  for (int v = 0; v < nv; ++v)
    row_of[ent.at({S.vs.rect[4 * v + 2], S.vs.rect[4 * v + 3]})].push_back(
        ent.at({S.vs.rect[4 * v], S.vs.rect[4 * v + 1]}));
  std::vector<int4> rows;
  std::vector<int2> segs;
  long covered = 0;
  for (auto& r : row_of) {
    std::vector<int>& xs = r.second;
    std::sort(xs.begin(), xs.end());
    const int first = (int)segs.size();
    for (size_t i = 0; i < xs.size();) {
      size_t j = i + 1;
      while (j < xs.size() && xs[j] == xs[j - 1] + 1 && lvl[xs[j]] == lvl[xs[i]]) ++j;
      const int L = lvl[xs[i]];
      segs.push_back(make_int2(xs[i] + L, xs[j - 1] + 1 + L));
      covered += (long)(j - i);
      i = j;
    }
    rows.push_back(make_int4(r.first, first, (int)segs.size() - first, 0));
  }
  if (covered != nv) return cudaSuccess;
  std::vector<double> e1(2 * (size_t)n1);
  for (int e = 0; e < n1; ++e) { e1[e] = ex[e]; e1[n1 + e] = ew[e]; }
  cudaError_t err;
  if (h->tsize == 8) err = upload(S.e1, e1, h->stream);
  else err = upload(S.e1, std::vector<float>(e1.begin(), e1.end()), h->stream);
  if (err != cudaSuccess) return err;
  if ((err = upload(S.lst, lst, h->stream)) != cudaSuccess) return err;
  if ((err = upload(S.rows, rows, h->stream)) != cudaSuccess) return err;
  if ((err = upload(S.segs, segs, h->stream)) != cudaSuccess) return err;
  S.n1 = n1;
  S.nrows = (int)rows.size();
  return cudaSuccess;
}

static mlvs_status get_space(mlvs_handle* h, const std::vector<int>& kappa, int* out) {
  std::vector<int> keff = enforce_consistency(kappa, h->n_base, h->D);
  auto it = h->space_of_key.find(keff);
  if (it != h->space_of_key.end()) { *out = it->second; return MLVS_OK; }
  SpaceRt S;
  S.keff = keff;
  S.vs = kappa_vspace(h->base, h->D, keff, S.owner);
  bool uni = true;
  for (int x : keff) uni = uni && (x == keff[0]);
  std::vector<double> axd;
  if (uni) {
    auto gr = groups_1d(h->n_base, keff[0]);
    S.nax = (int)gr.size();
    axd.resize(2 * gr.size());
    for (size_t g = 0; g < gr.size(); ++g) merged(h->base, gr[g].first, gr[g].second, axd[g], axd[gr.size() + g]);
  }
  const int nv = S.vs.nv();
  std::vector<double> vt(4 * (size_t)nv);
  for (int v = 0; v < nv; ++v) {
    vt[v] = S.vs.xix[v];
    vt[nv + v] = S.vs.xiy[v];
    vt[2 * nv + v] = S.vs.wx[v];
    vt[3 * nv + v] = S.vs.wy[v];
  }
  std::vector<double> inv(16);
  if (!mapping_inverse(S.vs, h->D, inv.data())) return fail(h, MLVS_ERR_SINGULAR, "singular mapping matrix");
  if (h->tsize == 8) {
    CK(upload(S.vt, vt, h->stream));
    CK(upload(S.ax, axd, h->stream));
  } else {
    CK(upload(S.vt, std::vector<float>(vt.begin(), vt.end()), h->stream));
    CK(upload(S.ax, std::vector<float>(axd.begin(), axd.end()), h->stream));
  }
  CK(upload(S.ainv, inv, h->stream));
  {
    std::vector<double> xid(2 * (size_t)nv);
    for (int v = 0; v < nv; ++v) { xid[v] = S.vs.xix[v]; xid[nv + v] = S.vs.xiy[v]; }
    CK(upload(S.xid, xid, h->stream));
    CK(upload(S.owner_d, S.owner, h->stream));
    CK(upload(S.kp_d, std::vector<unsigned char>(keff.begin(), keff.end()), h->stream));
    // per point: sum w|x|, sum w|y|, sum w x^2, sum w y^2, sum w|x||y| over its rectangle
    std::vector<double> geo(5 * (size_t)nv, 0.0);
    if (h->D == 2) {
      const auto& bx = h->base.x;
      const auto& bw = h->base.w;
      for (int v = 0; v < nv; ++v) {
        double w0x = 0, w1x = 0, w2x = 0, w0y = 0, w1y = 0, w2y = 0;
        for (int i = S.vs.rect[4 * v]; i < S.vs.rect[4 * v + 1]; ++i) {
          w0x += bw[i]; w1x += bw[i] * std::fabs(bx[i]); w2x += bw[i] * bx[i] * bx[i];
        }
        for (int i = S.vs.rect[4 * v + 2]; i < S.vs.rect[4 * v + 3]; ++i) {
          w0y += bw[i]; w1y += bw[i] * std::fabs(bx[i]); w2y += bw[i] * bx[i] * bx[i];
        }
        geo[v] = w1x * w0y;
        geo[nv + v] = w0x * w1y;
        geo[2 * (size_t)nv + v] = w2x * w0y;
        geo[3 * (size_t)nv + v] = w0x * w2y;
        geo[4 * (size_t)nv + v] = w1x * w1y;
      }
    }
    CK(upload(S.geo, geo, h->stream));
  }
  if (!uni && h->D == 2) CK(row_tables(h, S));
  h->spaces.push_back(std::move(S));
  *out = (int)h->spaces.size() - 1;
  h->space_of_key[keff] = *out;
  return MLVS_OK;
}

// Projection table P_{s->t} (Sec. 3.3.2): every target point inherits from the one source
// point containing it (refinement) or averages the source points it is made of (coarsening).
static mlvs_status get_csr(mlvs_handle* h, int s, int t, CSR** out) {
  auto key = std::make_pair(s, t);
  auto it = h->csr.find(key);
  if (it != h->csr.end()) { *out = &it->second; return MLVS_OK; }
  const SpaceRt& S = h->spaces[s];
  const SpaceRt& Tt = h->spaces[t];
  const int n = h->n_base;
  std::vector<int> off(1, 0), idx;
  std::vector<double> wgt;
  for (int i = 0; i < Tt.vs.nv(); ++i) {
    const int xa = Tt.vs.rect[4 * i], xb = Tt.vs.rect[4 * i + 1];
    const int ya = Tt.vs.rect[4 * i + 2], yb = Tt.vs.rect[4 * i + 3];
    std::vector<int> own;
    for (int iy = ya; iy < yb; ++iy)
      for (int ix = xa; ix < xb; ++ix) own.push_back(S.owner[(h->D == 2 ? iy * n : 0) + ix]);
    std::sort(own.begin(), own.end());
    own.erase(std::unique(own.begin(), own.end()), own.end());
    if (own.size() == 1) {
      idx.push_back(own[0]);
      wgt.push_back(1.0);
    } else {
      double area = 0.0;
      for (int o : own) area += S.vs.w[o];
      if (std::fabs(area - Tt.vs.w[i]) > 1e-10 * Tt.vs.w[i])
        return fail(h, MLVS_ERR_ARG, "velocity spaces are not nested");
      for (int o : own) { idx.push_back(o); wgt.push_back(S.vs.w[o] / area); }
    }
    off.push_back((int)idx.size());
  }
  CSR c;
  CK(upload(c.off, off, h->stream));
  CK(upload(c.idx, idx, h->stream));
  if (h->tsize == 8) { CK(upload(c.wgt, wgt, h->stream)); }
  else { CK(upload(c.wgt, std::vector<float>(wgt.begin(), wgt.end()), h->stream)); }
  auto res = h->csr.emplace(key, std::move(c));
  *out = &res.first->second;
  return MLVS_OK;
}

// ---------------------------------------------------------------------------------------
// typed launchers

namespace {

template <class S, class T, int D> struct Runner {
  static constexpr int TX = (D == 2) ? kTX2 : kTX1;
  static constexpr int TY = (D == 2) ? kTY2 : 1;
  static constexpr int VPC = kMaxVpc;
  static constexpr size_t SM0 = TileSmem<T, TX, TY, D>::BYTES;
  static constexpr size_t SM0C = TileSmem<T, TX, TY, D, true>::BYTES;
  static constexpr size_t SMU = UpdSmem<T, TX, TY, D, VPC>::BYTES;
  static constexpr int FIN_BLOCK = 32;   // small launches spread over more SMs (FP64 latency)
  static int fin_grid(int npt) { return std::max(1, (npt + FIN_BLOCK - 1) / FIN_BLOCK); }
  // Tensor-product spaces with many points: one thread per point (one-axis sums in the
  // thread).  Otherwise the split path: state per thread, velocity sums per warp (on tensor-
  // product spaces the one-axis sums over the warp's lanes), correction per thread, which
  // spreads a small launch's sums over more of the GPU.
  static constexpr int kFinThreadMin = 4096;
  static void launch_finalize(mlvs_handle* h, PointArgs a, LevelRt& L) {
    // chunk sums first (many threads), then the finalisation reads them
    if (a.nwork <= 0) return;
    if (L.msum.p) {
      ++h->launches;
      const long nt = (long)NMOM * a.nwork;
      k_sum_chunks<<<(unsigned)((nt + 255) / 256), 256, 0, h->stream>>>(a.part, a.k.nchunk, a.npt, a.pts, a.nwork,
                                                                         L.msum.as<double>());
      a.msum = L.msum.as<double>();
    }
    if (a.k.nax > 0 && (a.nwork >= kFinThreadMin || a.prm8_out)) {   // the eight-moment solve per thread
      k_finalize<T, D><<<fin_grid(a.nwork), FIN_BLOCK, 0, h->stream>>>(a);
      return;
    }
    a.scr = L.fscr.as<double>();
    a.need = L.fneed.as<int>();
    h->launches += 2;
    k_fin_pre<T, D><<<fin_grid(a.nwork), FIN_BLOCK, 0, h->stream>>>(a);
    // the eight-moment correction on a space that is not a tensor product: its sums from the
    // row tables (orders up to 9) and its solve per thread
    const bool c8 = D == 2 && a.prm8_out;
    size_t sm = 0;
    if (a.rows) {   // the row tables' prefix sums: shared memory per warp (4 warps per CTA)
      sm = (size_t)4 * row_smem_values(a.n1, c8 ? 10 : 8) * sizeof(T);
      if (sm > (size_t)smem_optin()) {
        a.rows = nullptr;   // the direct sums need none (the eight-moment sums report an error)
        sm = 0;
      }
    }
    const unsigned gs = (unsigned)std::max(1, (a.nwork * 32 + 127) / 128);
    if (c8) {
      k_fin_sums<T, D, true><<<gs, 128, sm, h->stream>>>(a);
      k_fin_post<T, D, true><<<fin_grid(a.nwork), FIN_BLOCK, 0, h->stream>>>(a);
    } else {
      k_fin_sums<T, D><<<gs, 128, sm, h->stream>>>(a);
      k_fin_post<T, D><<<fin_grid(a.nwork), FIN_BLOCK, 0, h->stream>>>(a);
    }
  }

  // largest dynamic shared memory a CTA may opt in to on the current device
  static int smem_optin() {
    int dev = 0, v = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
  }

  static cudaError_t set_smem_limits() {
    {
      cudaError_t e = cudaFuncSetAttribute(k_fin_sums<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fin_sums<T, D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
      if (e != cudaSuccess) return e;
    }
    const void* fn[4] = {(const void*)k_faces<S, T, D, TX, TY, false, false>,
                         (const void*)k_faces<S, T, D, TX, TY, true, false>,
                         (const void*)k_update<S, T, D, TX, TY, VPC, false, false>,
                         (const void*)k_update<S, T, D, TX, TY, VPC, true, false>};
    for (int i = 0; i < 4; ++i) {
      cudaError_t e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(i < 2 ? SM0 : SMU));
      if (e != cudaSuccess) return e;
    }
    if constexpr (D == 2) {
      const void* fc[4] = {(const void*)k_faces<S, T, D, TX, TY, false, true>,
                           (const void*)k_faces<S, T, D, TX, TY, true, true>,
                           (const void*)k_update<S, T, D, TX, TY, VPC, false, true>,
                           (const void*)k_update<S, T, D, TX, TY, VPC, true, true>};
      for (int i = 0; i < 4; ++i) {
        cudaError_t e = cudaFuncSetAttribute(fc[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(i < 2 ? SM0C : SMU));
        if (e != cudaSuccess) return e;
      }
      const void* f8[4] = {(const void*)k_faces<S, T, D, TX, TY, false, false, true>,
                           (const void*)k_faces<S, T, D, TX, TY, false, true, true>,
                           (const void*)k_update<S, T, D, TX, TY, VPC, false, false, true>,
                           (const void*)k_update<S, T, D, TX, TY, VPC, false, true, true>};
      for (int i = 0; i < 4; ++i) {
        cudaError_t e = cudaFuncSetAttribute(f8[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(i == 0 ? SM0 : (i == 1 ? SM0C : SMU)));
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }

  // one tile pass (MODE 0: k_faces, MODE 1: k_update) of a level that holds every cell,
  // Cartesian or curvilinear
  template <int MODE>
  static void launch_tile(mlvs_handle* h, dim3 grid, const TileArgs& t, int limiter) {
    if constexpr (D == 2) {
      if (h->cfg.compat_moments == 8) {   // the eight-moment correction's model
        if (h->curvi) {
          if constexpr (MODE == 0)
            k_faces<S, T, D, TX, TY, false, true, true><<<grid, TX * TY, SM0C, h->stream>>>(t, nullptr, nullptr, limiter);
          else k_update<S, T, D, TX, TY, VPC, false, true, true><<<grid, TX * TY, SMU, h->stream>>>(t, nullptr, nullptr);
        } else {
          if constexpr (MODE == 0)
            k_faces<S, T, D, TX, TY, false, false, true><<<grid, TX * TY, SM0, h->stream>>>(t, nullptr, nullptr, limiter);
          else k_update<S, T, D, TX, TY, VPC, false, false, true><<<grid, TX * TY, SMU, h->stream>>>(t, nullptr, nullptr);
        }
        return;
      }
      if (h->curvi) {
        if constexpr (MODE == 0)
          k_faces<S, T, D, TX, TY, false, true><<<grid, TX * TY, SM0C, h->stream>>>(t, nullptr, nullptr, limiter);
        else k_update<S, T, D, TX, TY, VPC, false, true><<<grid, TX * TY, SMU, h->stream>>>(t, nullptr, nullptr);
        return;
      }
    }
    if constexpr (MODE == 0)
      k_faces<S, T, D, TX, TY, false, false><<<grid, TX * TY, SM0, h->stream>>>(t, nullptr, nullptr, limiter);
    else k_update<S, T, D, TX, TY, VPC, false, false><<<grid, TX * TY, SMU, h->stream>>>(t, nullptr, nullptr);
  }

  // one tile pass over every level of a multi-level instance: n work items, argument table tab
  template <int MODE>
  static void launch_lv(mlvs_handle* h, int n, const TileArgs* tab, const int4* w, int limiter) {
    const TileArgs none{};
    if constexpr (D == 2) {
      if (h->curvi) {
        if constexpr (MODE == 0) k_faces<S, T, D, TX, TY, true, true><<<n, TX * TY, SM0C, h->stream>>>(none, tab, w, limiter);
        else k_update<S, T, D, TX, TY, VPC, true, true><<<n, TX * TY, SMU, h->stream>>>(none, tab, w);
        return;
      }
    }
    if constexpr (MODE == 0) k_faces<S, T, D, TX, TY, true, false><<<n, TX * TY, SM0, h->stream>>>(none, tab, w, limiter);
    else k_update<S, T, D, TX, TY, VPC, true, false><<<n, TX * TY, SMU, h->stream>>>(none, tab, w);
  }

  // a level that holds every cell runs the tile kernels without level tables
  static bool single(const mlvs_handle* h, const LevelRt& L) {
    return L.cells.size() == (size_t)h->nx * h->ny && L.nghost == 0 && L.nX == 0 && L.nY == 0;
  }
  // every other instance steps through the level-batched launches
  static bool batched(const mlvs_handle* h, const Inst& I) { return I.lv.size() > 1 || !single(h, I.lv[0]); }

  static void mark_begin(mlvs_handle* h, int ph) {
    ++h->launches;
    if (!h->profiling) return;
    h->prof.marks.push_back({ph, (int)h->prof.used});
    cudaEventRecord(h->prof.next(), h->stream);
  }
  static void mark_end(mlvs_handle* h) {
    if (!h->profiling) return;
    cudaEventRecord(h->prof.next(), h->stream);
  }

  static PointArgs pargs(mlvs_handle* h, Inst& I, LevelRt& L, bool face) {
    PointArgs a;
    a.k = L.k;
    a.gas = h->gas;
    a.is_face = face ? 1 : 0;
    a.npt = face ? L.k.nface : (int)L.cells.size();
    a.pts = (face && L.nflist < L.k.nface) ? L.flist.as<int>() : nullptr;
    a.nwork = face ? L.nflist : a.npt;
    a.part = face ? L.fpart.as<double>() : L.cpart.as<double>();
    const SpaceRt& sp = h->spaces[L.space];
    a.vt = sp.vt.p;
    a.ax = sp.ax.p;
    a.ids = L.ids.as<int>();
    a.frole = L.frole.as<unsigned char>();
    a.ucell = I.ucell.p;
    a.compat = face ? h->cfg.compat_face : h->cfg.compat_cell;
    for (int s = 0; s < 4; ++s)
      for (int j = 0; j < 3; ++j) a.wall[s][j] = h->cfg.wall[s][j];
    for (int j = 0; j < 4; ++j) a.far[j] = h->cfg.far[j];
    a.err = I.err.as<int>();
    a.W = nullptr;
    a.cprm = nullptr;
    a.prm_out = nullptr;
    a.scr = nullptr;
    a.need = nullptr;
    a.msum = nullptr;
    a.wden = h->curvi ? L.wden.as<double>() : nullptr;
    a.e1 = sp.nrows > 0 ? sp.e1.p : nullptr;
    a.n1 = sp.n1;
    a.lst = sp.lst.as<int>();
    a.rows = sp.nrows > 0 ? sp.rows.as<int4>() : nullptr;
    a.nrows = sp.nrows;
    a.segs = sp.segs.as<int2>();
    a.prm8_out = nullptr;
    return a;
  }

  static TileArgs targs(mlvs_handle* h, Inst& I, LevelRt& L, int lid) {
    TileArgs t;
    t.k = L.k;
    const int nc = (int)L.cells.size();
    t.f_in = L.f[L.cur].p;
    t.f_out = L.f[L.cur ^ 1].p;
    t.nslot = nc;
    t.cparam = L.prm[L.pcur].p;
    t.fparam = L.fprm.p;
    t.vt = h->spaces[L.space].vt.p;
    t.part = nullptr;
    t.tiles = L.tiles.as<int>();
    t.ntx = (h->nx + TX - 1) / TX;
    t.nty = (D == 2) ? (h->ny + TY - 1) / TY : 1;
    t.level = lid;
    t.lvl_of = I.lvl_of_d.as<int>();
    t.slot_of = I.slot_of_d.as<int>();
    t.ghost_of = L.nghost ? L.ghost_of.as<int>() : nullptr;
    t.ghost = L.ghost.p;
    t.nghost = L.nghost;
    t.frole = L.frole.as<unsigned char>();
    t.fslot = L.fslot.as<int>();
    t.X = L.X.p;
    t.nX = L.nX;
    t.xfid = L.xfid.as<int>();
    t.cparam8 = L.prm8[L.pcur].p;
    t.fparam8 = L.fprm8.p;
    t.Y = L.Y.p;
    t.nY = L.nY;
    t.fbar = L.fbar.p;
    t.ucell = I.ucell.p;
    t.cgeo = h->curvi ? h->cgeo_d.p : nullptr;
    t.fgeo = h->curvi ? h->fgeo_d.p : nullptr;
    t.step = I.stepctr.as<unsigned>();
    t.salt = hash_host((unsigned)lid * 0x9e3779b9u + (unsigned)(&I - h->inst.data()) * 0x85ebca77u);
    return t;
  }

  // cells of one level: params into prm[pcur^1], W and the cell velocities
  static cudaError_t finalize_cells(mlvs_handle* h, Inst& I, LevelRt& L) {
    const int n = (int)L.cells.size();
    if (n == 0) { L.fresh = true; return cudaSuccess; }
    PointArgs a = pargs(h, I, L, false);
    a.cprm = L.prm[L.pcur].p;
    a.prm_out = L.prm[L.pcur ^ 1].p;
    a.prm8_out = L.prm8[L.pcur ^ 1].p;   // null without the eight-moment correction
    a.W = I.W.as<double>();
    mark_begin(h, 0);
    ++h->launches;
    launch_finalize(h, a, L);
    k_scatter_velocity<T><<<(n + 127) / 128, 128, 0, h->stream>>>(L.prm[L.pcur ^ 1].as<T>(), n, L.ids.as<int>(),
                                                                 I.ucell.as<T>(), h->nx * h->ny);
    mark_end(h);
    L.pcur ^= 1;
    L.fresh = true;
    return cudaGetLastError();
  }

  static MapArgs margs(mlvs_handle* h, int s, int t, CSR* c) {
    MapArgs m;
    const SpaceRt& Ss = h->spaces[s];
    const SpaceRt& St = h->spaces[t];
    m.s.nv = Ss.vs.nv(); m.s.vt = Ss.vt.p; m.s.ainv = Ss.ainv.as<double>();
    m.t.nv = St.vs.nv(); m.t.vt = St.vt.p; m.t.ainv = St.ainv.as<double>();
    m.off = c->off.as<int>();
    m.idx = c->idx.as<int>();
    m.wgt = c->wgt.p;
    m.R = h->gas.R;
    m.c0 = h->gas.K + 3.0 - D;
    m.cv = 0.5 * (3.0 + h->gas.K) * h->gas.R;
    m.twoK = 2.0 * h->gas.K;
    m.correct = 1;
    return m;
  }

  static int map_grid(int n) { return std::max(1, std::min(n, 148 * 8)); }

  // mapping launch with the items-per-CTA choice of the route size
  template <class SrcT, class DstT, int KIND>
  static void launch_map(mlvs_handle* h, const MapArgs& m) {
    const int g = map_items_per_cta(m.nitems);
    const int nb = map_grid((m.nitems + g - 1) / g);
    switch (g) {
      case 8: k_map<SrcT, DstT, T, D, KIND, 8><<<nb, 256, 0, h->stream>>>(m); break;
      case 4: k_map<SrcT, DstT, T, D, KIND, 4><<<nb, 256, 0, h->stream>>>(m); break;
      case 2: k_map<SrcT, DstT, T, D, KIND, 2><<<nb, 256, 0, h->stream>>>(m); break;
      default: k_map<SrcT, DstT, T, D, KIND, 1><<<nb, 256, 0, h->stream>>>(m); break;
    }
  }

  // route arguments and item groups of the batched ghost launch (after the routes' items are
  // on the device)
  static cudaError_t ghost_batch(mlvs_handle* h, Inst& I) {
    MapBatch& B = I.gb;
    B.ok = false;
    B.nwork = 0;
    std::vector<int> rs;
    std::vector<const Route*> rp;
    for (int r = 0; r < (int)I.ghosts.size(); ++r)
      if (!I.ghosts[r].items.empty()) { rs.push_back(r); rp.push_back(&I.ghosts[r]); }
    if (rs.empty()) return cudaSuccess;
    std::vector<MapWork> work;
    const int G = group_items(rp, work);
    for (int par = 0; par < 4; ++par) {
      std::vector<MapArgs> tab;
      for (int r : rs) {
        Route& rt = I.ghosts[r];
        LevelRt& Ls = I.lv[rt.src];
        LevelRt& Ld = I.lv[rt.dst];
        CSR* c = nullptr;
        if (get_csr(h, Ls.space, Ld.space, &c) != MLVS_OK) return cudaErrorInvalidValue;
        MapArgs m = margs(h, Ls.space, Ld.space, c);
        m.src = Ls.f[par >> 1].p;
        m.src_ld = (int)Ls.cells.size();
        m.dst = Ld.ghost.p;
        m.dst_ld = Ld.nghost;
        m.prm = Ls.prm[par & 1].p;
        m.prm_ld = (int)Ls.cells.size();
        m.items = rt.items_d.as<MapItem>();
        m.nitems = (int)rt.items.size();
        tab.push_back(m);
      }
      cudaError_t e = upload(B.routes[par], tab, h->stream);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = upload(B.work, work, h->stream);
    if (e != cudaSuccess) return e;
    B.nwork = (int)work.size();
    B.G = G;
    B.ok = true;
    return cudaSuccess;
  }

  // item groups of a set of routes: the largest G whose group count still fills the GPU
  static int group_items(const std::vector<const Route*>& rs, std::vector<MapWork>& work) {
    auto groups = [&](int g) {
      long n = 0;
      for (const Route* r : rs) n += ((long)r->items.size() + g - 1) / g;
      return n;
    };
    int G = 1;
    for (int g : {8, 4, 2})
      if (groups(g) >= 148 * 4) { G = g; break; }
    work.clear();
    for (int q = 0; q < (int)rs.size(); ++q) {
      const int n = (int)rs[q]->items.size();
      for (int b = 0; b < n; b += G) work.push_back({q, b, std::min(G, n - b)});
    }
    return G;
  }

  // route arguments and item groups of the batched flux launch (every route)
  static cudaError_t flux_batch(mlvs_handle* h, Inst& I) {
    MapBatch& B = I.fb;
    B.ok = false;
    B.nwork = 0;
    std::vector<const Route*> rs;
    for (auto& r : I.fluxes)
      if (!r.items.empty()) rs.push_back(&r);
    if (rs.empty()) return cudaSuccess;
    std::vector<MapWork> work;
    B.G = group_items(rs, work);
    std::vector<MapArgs> tab;
    for (const Route* r : rs) {
      LevelRt& Ls = I.lv[r->src];
      LevelRt& Ld = I.lv[r->dst];
      CSR* c = nullptr;
      if (get_csr(h, Ls.space, Ld.space, &c) != MLVS_OK) return cudaErrorInvalidValue;
      MapArgs m = margs(h, Ls.space, Ld.space, c);
      m.src = Ls.X.p;
      m.src_ld = Ls.nX;
      m.dst = Ld.Y.p;
      m.dst_ld = Ld.nY;
      m.prm = Ls.fprm.p;
      m.prm_ld = Ls.k.nface;
      m.items = r->items_d.as<MapItem>();
      m.nitems = (int)r->items.size();
      tab.push_back(m);
    }
    cudaError_t e = upload(B.routes[0], tab, h->stream);
    if (e != cudaSuccess) return e;
    if ((e = upload(B.work, work, h->stream)) != cudaSuccess) return e;
    B.nwork = (int)work.size();
    B.ok = true;
    return cudaSuccess;
  }

  // argument table and work items of the level-batched tile launches (multi-level
  // instances).  Items go in decreasing order of their velocity count, so that the longest
  // start first.  The instance must be in h->inst with all its buffers allocated (the table
  // holds their addresses and the instance's random-bit salt).
  static cudaError_t tile_batch(mlvs_handle* h, Inst& I) {
    I.nwf = I.nwu = I.nwx = 0;
    const int nl = (int)I.lv.size();
    if (!batched(h, I)) return cudaSuccess;
    std::vector<TileArgs> tab((size_t)2 * 4 * nl);
    for (int mode = 0; mode < 2; ++mode)
      for (int par = 0; par < 4; ++par)
        for (int l = 0; l < nl; ++l) {
          LevelRt& L = I.lv[l];
          const int cur = L.cur, pcur = L.pcur;
          L.cur = par >> 1;
          L.pcur = par & 1;
          TileArgs t = targs(h, I, L, l);
          L.cur = cur;
          L.pcur = pcur;
          t.part = mode == 0 ? L.fpart.as<double>() : L.cpart.as<double>();
          // every address a kernel of the work lists dereferences must exist
          const bool cells = !L.cells.empty(), tiles = L.ntiles > 0;
          if ((tiles && (!t.tiles || !t.lvl_of || !t.slot_of || !t.frole || !t.fslot || !t.vt || !t.part ||
                         !t.fparam || !t.fbar || !t.ucell || !t.step)) ||
              (tiles && h->curvi && (!t.cgeo || !t.fgeo)) ||
              (cells && (!t.f_in || !t.f_out || !t.cparam)) || (L.nghost > 0 && (!t.ghost || !t.ghost_of)) ||
              (L.nX > 0 && (!t.X || !t.xfid)) || (L.nY > 0 && !t.Y))
            return cudaErrorInvalidValue;
          tab[((size_t)mode * 4 + par) * nl + l] = t;
        }
    std::vector<int> ord(nl);
    for (int l = 0; l < nl; ++l) ord[l] = l;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return I.lv[a].k.vpc > I.lv[b].k.vpc; });
    std::vector<int4> wf, wu, wx;
    for (int l : ord) {
      const LevelRt& L = I.lv[l];
      std::set<int> with_cells;
      for (int c : L.cells) with_cells.insert(((c / h->nx) / TY) * ((h->nx + TX - 1) / TX) + (c % h->nx) / TX);
      for (int c = 0; c < L.k.nchunk; ++c)
        for (int ti = 0; ti < L.ntiles; ++ti) {
          wf.push_back(make_int4(l, ti, c, 0));
          if (with_cells.count(L.tiles_h[ti])) wu.push_back(make_int4(l, ti, c, 0));
        }
      const int npair = (L.k.nv + 1) / 2;
      for (int c0 = 0; c0 < L.nX; c0 += 128)
        for (int p0 = 0; p0 < npair; p0 += kXPairs) wx.push_back(make_int4(l, c0, p0, 0));
    }
    cudaError_t e;
    if ((e = upload(I.tab, tab, h->stream)) != cudaSuccess) return e;
    if ((e = upload(I.wf, wf, h->stream)) != cudaSuccess) return e;
    if ((e = upload(I.wu, wu, h->stream)) != cudaSuccess) return e;
    if ((e = upload(I.wx, wx, h->stream)) != cudaSuccess) return e;
    I.nwf = (int)wf.size();
    I.nwu = (int)wu.size();
    I.nwx = (int)wx.size();
    return cudaSuccess;
  }

  static cudaError_t run_ghosts(mlvs_handle* h, Inst& I) {
    const bool nine = D == 2 && h->cfg.map_moments == 9;
    const bool positive = D == 2 && h->cfg.positive_mapping && !nine;
    // one launch for every route when all source levels are on the same buffer parity
    if (I.gb.ok && !nine && !positive) {
      int par = -1;
      bool same = true;
      for (auto& r : I.ghosts) {
        if (r.items.empty()) continue;
        const LevelRt& Ls = I.lv[r.src];
        const int p = 2 * Ls.cur + Ls.pcur;
        if (par < 0) par = p;
        else if (p != par) same = false;
      }
      if (same && par >= 0) {
        const MapArgs* rt = I.gb.routes[par].as<MapArgs>();
        const MapWork* wk = I.gb.work.as<MapWork>();
        const int nb = std::max(1, std::min(I.gb.nwork, 148 * 16));
        mark_begin(h, 4);
        switch (I.gb.G) {
          case 8: k_map_multi<S, T, T, D, SRC_BARP, 8><<<nb, 256, 0, h->stream>>>(rt, wk, I.gb.nwork); break;
          case 4: k_map_multi<S, T, T, D, SRC_BARP, 4><<<nb, 256, 0, h->stream>>>(rt, wk, I.gb.nwork); break;
          case 2: k_map_multi<S, T, T, D, SRC_BARP, 2><<<nb, 256, 0, h->stream>>>(rt, wk, I.gb.nwork); break;
          default: k_map_multi<S, T, T, D, SRC_BARP, 1><<<nb, 256, 0, h->stream>>>(rt, wk, I.gb.nwork); break;
        }
        mark_end(h);
        return cudaGetLastError();
      }
    }
    for (auto& r : I.ghosts) {
      if (r.items.empty()) continue;
      LevelRt& Ls = I.lv[r.src];
      LevelRt& Ld = I.lv[r.dst];
      CSR* c = nullptr;
      if (get_csr(h, Ls.space, Ld.space, &c) != MLVS_OK) return cudaErrorInvalidValue;
      MapArgs m = margs(h, Ls.space, Ld.space, c);
      m.src = Ls.f[Ls.cur].p;
      m.src_ld = (int)Ls.cells.size();
      m.dst = Ld.ghost.p;
      m.dst_ld = Ld.nghost;
      m.prm = Ls.prm[Ls.pcur].p;
      m.prm_ld = (int)Ls.cells.size();
      m.items = r.items_d.as<MapItem>();
      m.nitems = (int)r.items.size();
      mark_begin(h, 4);
      if (nine) k_map9<S, T, T, SRC_BARP><<<(m.nitems + 127) / 128, 128, 0, h->stream>>>(m, I.err.as<int>());
      else launch_map<S, T, SRC_BARP>(h, m);
      mark_end(h);
      if (positive) {
        // ghost states whose additive mapping went negative: the exponential correction
        mark_begin(h, 4);
        k_expmap<S, T, T, SRC_BARP><<<(m.nitems + 127) / 128, 128, 0, h->stream>>>(m, nullptr);
        mark_end(h);
      }
    }
    return cudaGetLastError();
  }

  // the cross-level microfluxes X of every level mapped to the receiving levels' Y
  static cudaError_t run_fluxes(mlvs_handle* h, Inst& I) {
    const bool nine = D == 2 && h->cfg.map_moments == 9;
    if (I.fb.ok && !nine) {
      const MapBatch& B = I.fb;
      const MapArgs* rt = B.routes[0].as<MapArgs>();
      const MapWork* wk = B.work.as<MapWork>();
      const int nb = std::max(1, std::min(B.nwork, 148 * 16));
      mark_begin(h, 5);
      switch (B.G) {
        case 8: k_map_multi<T, T, T, D, SRC_FLUX, 8><<<nb, 256, 0, h->stream>>>(rt, wk, B.nwork); break;
        case 4: k_map_multi<T, T, T, D, SRC_FLUX, 4><<<nb, 256, 0, h->stream>>>(rt, wk, B.nwork); break;
        case 2: k_map_multi<T, T, T, D, SRC_FLUX, 2><<<nb, 256, 0, h->stream>>>(rt, wk, B.nwork); break;
        default: k_map_multi<T, T, T, D, SRC_FLUX, 1><<<nb, 256, 0, h->stream>>>(rt, wk, B.nwork); break;
      }
      mark_end(h);
      return cudaGetLastError();
    }
    for (auto& r : I.fluxes) {
      if (r.items.empty()) continue;
      LevelRt& Ls = I.lv[r.src];
      LevelRt& Ld = I.lv[r.dst];
      CSR* c = nullptr;
      if (get_csr(h, Ls.space, Ld.space, &c) != MLVS_OK) return cudaErrorInvalidValue;
      MapArgs m = margs(h, Ls.space, Ld.space, c);
      m.src = Ls.X.p;
      m.src_ld = Ls.nX;
      m.dst = Ld.Y.p;
      m.dst_ld = Ld.nY;
      m.prm = Ls.fprm.p;
      m.prm_ld = Ls.k.nface;
      m.items = r.items_d.as<MapItem>();
      m.nitems = (int)r.items.size();
      mark_begin(h, 5);
      if (nine) k_map9<T, T, T, SRC_FLUX><<<(m.nitems + 127) / 128, 128, 0, h->stream>>>(m, I.err.as<int>());
      else launch_map<T, T, SRC_FLUX>(h, m);
      mark_end(h);
    }
    return cudaGetLastError();
  }

  // Two steps of a group of handles (same storage and mesh kind), captured on hs[0]->cap: per
  // instance (one graph branch each) the step counter, cell finalisation and ghost states; one
  // faces launch over the work items of every level of every instance; per instance the face
  // finalisations; one cross-flux launch; per instance the flux mapping; one update launch.
  // The tile arguments of every level at each step's buffer parity go to a pinned table that
  // the graph copies to the device before the step's tile passes.  kernels[j]: the kernels of
  // handle j per two steps (the group launches counted on handle 0).
  static cudaError_t group_capture(mlvs_handle* const* hs, int nh, mlvs_handle::GroupBufs& B,
                                   std::vector<int>& kernels, cudaGraphExec_t* exec_out) {
    mlvs_handle* h0 = hs[0];
    struct Ref { mlvs_handle* h; Inst* I; int lvl0; };
    std::vector<Ref> refs;
    int nlt = 0;
    for (int j = 0; j < nh; ++j)
      for (auto& I : hs[j]->inst) {
        refs.push_back({hs[j], &I, nlt});
        nlt += (int)I.lv.size();
      }
    // work lists (the same for both steps), longest items first
    std::vector<std::pair<int, int4>> wf, wu, wx;   // (velocities per chunk, item)
    for (const Ref& r : refs)
      for (int l = 0; l < (int)r.I->lv.size(); ++l) {
        const LevelRt& L = r.I->lv[l];
        const int g = r.lvl0 + l;
        std::set<int> with_cells;
        const int ntx = (r.h->nx + TX - 1) / TX;
        for (int c : L.cells) with_cells.insert(((c / r.h->nx) / TY) * ntx + (c % r.h->nx) / TX);
        for (int c = 0; c < L.k.nchunk; ++c)
          for (int ti = 0; ti < L.ntiles; ++ti) {
            wf.push_back({L.k.vpc, make_int4(g, ti, c, 0)});
            if (with_cells.count(L.tiles_h[ti])) wu.push_back({L.k.vpc, make_int4(g, ti, c, 0)});
          }
        const int npair = (L.k.nv + 1) / 2;
        for (int c0 = 0; c0 < L.nX; c0 += 128)
          for (int p0 = 0; p0 < npair; p0 += kXPairs) wx.push_back({0, make_int4(g, c0, p0, 0)});
      }
    auto order = [](std::vector<std::pair<int, int4>>& v) {
      std::stable_sort(v.begin(), v.end(), [](const std::pair<int, int4>& a, const std::pair<int, int4>& b) {
        return a.first > b.first;
      });
      std::vector<int4> out(v.size());
      for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].second;
      return out;
    };
    cudaError_t e;
    if ((e = upload(B.wf, order(wf), h0->stream)) != cudaSuccess) return e;
    if ((e = upload(B.wu, order(wu), h0->stream)) != cudaSuccess) return e;
    if ((e = upload(B.wx, order(wx), h0->stream)) != cudaSuccess) return e;
    B.nwf = (int)wf.size();
    B.nwu = (int)wu.size();
    B.nwx = (int)wx.size();
    const size_t per_step = (size_t)2 * nlt;
    if ((e = cudaMallocHost(&B.host, 2 * per_step * sizeof(TileArgs))) != cudaSuccess) return e;
    if ((e = B.tab.alloc(2 * per_step * sizeof(TileArgs))) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(h0->stream)) != cudaSuccess) return e;   // uploads before the capture
    std::vector<int> l0(nh);
    for (int j = 0; j < nh; ++j) l0[j] = hs[j]->launches;
    std::vector<cudaStream_t> saved(nh);
    for (int j = 0; j < nh; ++j) saved[j] = hs[j]->stream;
    // run f(h, I) for every instance on a branch of its own, joined into the capture stream
    auto branches = [&](auto&& f) -> cudaError_t {
      cudaError_t ee = cudaEventRecord(h0->ev_fork, h0->cap);
      for (size_t b = 0; b < refs.size() && ee == cudaSuccess; ++b) {
        cudaStream_t st = h0->branch[b];
        if ((ee = cudaStreamWaitEvent(st, h0->ev_fork, 0)) != cudaSuccess) break;
        refs[b].h->stream = st;
        if ((ee = f(refs[b].h, *refs[b].I)) != cudaSuccess) break;
        if ((ee = cudaEventRecord(h0->bev[b], st)) != cudaSuccess) break;
        ee = cudaStreamWaitEvent(h0->cap, h0->bev[b], 0);
      }
      return ee;
    };
    if ((e = cudaStreamBeginCapture(h0->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t ce = cudaSuccess;
    const int limiter = h0->cfg.limiter;
    for (int step = 0; step < 2 && ce == cudaSuccess; ++step) {
      ce = branches([&](mlvs_handle* h, Inst& I) -> cudaError_t {
        if constexpr (sizeof(S) <= 4) {
          ++h->launches;
          k_step_counter<<<1, 1, 0, h->stream>>>(I.stepctr.as<unsigned>());
        }
        for (int l = 0; l < h->n_levels; ++l) {
          cudaError_t e2;
          if (!I.lv[l].fresh && (e2 = finalize_cells(h, I, I.lv[l])) != cudaSuccess) return e2;
        }
        return run_ghosts(h, I);
      });
      if (ce != cudaSuccess) break;
      // the levels' arguments at this step's parity: pass 0 (face partials), pass 1 (cell partials)
      TileArgs* ht = B.host + step * per_step;
      for (const Ref& r : refs)
        for (int l = 0; l < (int)r.I->lv.size(); ++l) {
          LevelRt& L = r.I->lv[l];
          TileArgs t = targs(r.h, *r.I, L, l);
          t.part = L.fpart.as<double>();
          ht[r.lvl0 + l] = t;
          t.part = L.cpart.as<double>();
          ht[nlt + r.lvl0 + l] = t;
        }
      TileArgs* dt = B.tab.as<TileArgs>() + step * per_step;
      h0->stream = h0->cap;
      if ((ce = cudaMemcpyAsync(dt, ht, per_step * sizeof(TileArgs), cudaMemcpyHostToDevice, h0->cap)) != cudaSuccess)
        break;
      if (B.nwf > 0) {
        ++h0->launches;
        launch_lv<0>(h0, B.nwf, dt, B.wf.as<int4>(), limiter);
      }
      ce = branches([&](mlvs_handle* h, Inst& I) -> cudaError_t {
        for (LevelRt& L : I.lv) {
          if (L.ntiles == 0) continue;
          PointArgs a = pargs(h, I, L, true);
          a.cprm = L.prm[L.pcur].p;
          a.prm_out = L.fprm.p;
          mark_begin(h, 2);
          launch_finalize(h, a, L);
          mark_end(h);
        }
        return cudaGetLastError();
      });
      if (ce != cudaSuccess) break;
      h0->stream = h0->cap;
      if (B.nwx > 0) {
        ++h0->launches;
        if (D == 2 && h0->curvi) k_cross_flux<T, D, true><<<B.nwx, 128, 0, h0->cap>>>(dt + nlt, B.wx.as<int4>());
        else k_cross_flux<T, D, false><<<B.nwx, 128, 0, h0->cap>>>(dt + nlt, B.wx.as<int4>());
      }
      ce = branches([&](mlvs_handle* h, Inst& I) -> cudaError_t { return run_fluxes(h, I); });
      if (ce != cudaSuccess) break;
      h0->stream = h0->cap;
      if (B.nwu > 0) {
        ++h0->launches;
        launch_lv<1>(h0, B.nwu, dt + nlt, B.wu.as<int4>(), limiter);
      }
      if ((ce = cudaGetLastError()) != cudaSuccess) break;
      for (const Ref& r : refs)
        for (int l = 0; l < r.h->n_levels; ++l) {
          LevelRt& L = r.I->lv[l];
          if (L.cells.empty()) continue;
          L.cur ^= 1;
          L.fresh = false;
        }
    }
    for (int j = 0; j < nh; ++j) hs[j]->stream = saved[j];
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h0->cap, &graph);
    if (ce == cudaSuccess) ce = ee;
    cudaGraphExec_t exec = nullptr;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    kernels.assign(nh, 0);
    for (int j = 0; j < nh; ++j) {
      kernels[j] = hs[j]->launches - l0[j];
      hs[j]->launches = l0[j];
    }
    if (ce != cudaSuccess) return ce;
    *exec_out = exec;
    return cudaSuccess;
  }

  // faces of every level, face finalisation, cross-level microfluxes and their mapping, then
  // the update of every cell level: one launch per tile pass over all levels' work items.
  // The cell levels' buffers advance together, so one parity selects the argument table.
  static cudaError_t step_levels(mlvs_handle* h, Inst& I, int limiter) {
    int par = -1;
    for (const LevelRt& L : I.lv) {
      if (L.cells.empty()) continue;
      const int p = 2 * L.cur + L.pcur;
      if (par < 0) par = p;
      else if (p != par) return cudaErrorInvalidValue;
    }
    par = std::max(par, 0);
    const size_t nl = I.lv.size();
    const TileArgs* tab = I.tab.as<TileArgs>();
    if (I.nwf > 0) {
      mark_begin(h, 1);
      launch_lv<0>(h, I.nwf, tab + (size_t)par * nl, I.wf.as<int4>(), limiter);
      mark_end(h);
    }
    for (LevelRt& L : I.lv) {
      if (L.ntiles == 0) continue;
      PointArgs a = pargs(h, I, L, true);
      a.cprm = L.prm[L.pcur].p;
      a.prm_out = L.fprm.p;
      mark_begin(h, 2);
      launch_finalize(h, a, L);
      mark_end(h);
    }
    if (I.nwx > 0) {
      mark_begin(h, 5);
      const TileArgs* t1 = tab + (size_t)(4 + par) * nl;
      if (D == 2 && h->curvi) k_cross_flux<T, D, true><<<I.nwx, 128, 0, h->stream>>>(t1, I.wx.as<int4>());
      else k_cross_flux<T, D, false><<<I.nwx, 128, 0, h->stream>>>(t1, I.wx.as<int4>());
      mark_end(h);
    }
    cudaError_t e = run_fluxes(h, I);
    if (e != cudaSuccess) return e;
    if (I.nwu > 0) {
      mark_begin(h, 3);
      launch_lv<1>(h, I.nwu, tab + (size_t)(4 + par) * nl, I.wu.as<int4>(), limiter);
      mark_end(h);
    }
    return cudaGetLastError();
  }

  static cudaError_t step(mlvs_handle* h, Inst& I) {
    cudaError_t e;
    if constexpr (sizeof(S) <= 4) {   // random bits of the stochastic rounding (BF16, FP32)
      ++h->launches;
      k_step_counter<<<1, 1, 0, h->stream>>>(I.stepctr.as<unsigned>());
    }
    for (int l = 0; l < h->n_levels; ++l)
      if (!I.lv[l].fresh && (e = finalize_cells(h, I, I.lv[l])) != cudaSuccess) return e;
    if ((e = run_ghosts(h, I)) != cudaSuccess) return e;
    const int limiter = h->cfg.limiter;
    if (batched(h, I)) {
      if ((e = step_levels(h, I, limiter)) != cudaSuccess) return e;
    } else if (I.lv[0].ntiles > 0) {
      // one level holding every cell: the tile kernels without level tables
      LevelRt& L = I.lv[0];
      TileArgs t = targs(h, I, L, 0);
      t.part = L.fpart.as<double>();
      const dim3 grid(L.ntiles, L.k.nchunk);
      mark_begin(h, 1);
      launch_tile<0>(h, grid, t, limiter);
      mark_end(h);
      PointArgs a = pargs(h, I, L, true);
      a.cprm = L.prm[L.pcur].p;
      a.prm_out = L.fprm.p;
      a.prm8_out = L.fprm8.p;
      mark_begin(h, 2);
      launch_finalize(h, a, L);
      mark_end(h);
      t.part = L.cpart.as<double>();
      mark_begin(h, 3);
      launch_tile<1>(h, grid, t, limiter);
      mark_end(h);
    }
    for (int l = 0; l < h->n_levels; ++l) {
      LevelRt& L = I.lv[l];
      if (L.cells.empty()) continue;
      L.cur ^= 1;
      L.fresh = false;
    }
    return cudaGetLastError();
  }

  // parameters from (rho, u, v, T) with q = 0 and phi~ = the corrected Maxwellian (level 0)
  static cudaError_t init_state(mlvs_handle* h, Inst& I, const double* dW0) {
    cudaError_t e = set_smem_limits();
    if (e != cudaSuccess) return e;
    LevelRt& L = I.lv[0];
    const int n = (int)L.cells.size();
    PointArgs a = pargs(h, I, L, false);
    a.prm_out = L.prm[0].p;
    k_init_params<T, D><<<fin_grid(n), FIN_BLOCK, 0, h->stream>>>(a, dW0);
    dim3 g((n + 127) / 128, std::min(L.k.nv, 1024));
    k_init_f<S, T, D><<<g, 128, 0, h->stream>>>(L.k, n, L.prm[0].as<T>(), h->spaces[L.space].vt.as<T>(),
                                                 L.f[0].as<S>());
    k_scatter_velocity<T><<<(n + 127) / 128, 128, 0, h->stream>>>(L.prm[0].as<T>(), n, L.ids.as<int>(),
                                                                 I.ucell.as<T>(), h->nx * h->ny);
    L.cur = 0;
    L.pcur = 0;
    return moments_of_levels(h, I);
  }

  // chunk partials of every cell level from f[cur] in the frame of the cell velocities
  static cudaError_t moments_of_levels(mlvs_handle* h, Inst& I) {
    for (int l = 0; l < h->n_levels; ++l) {
      LevelRt& L = I.lv[l];
      const int n = (int)L.cells.size();
      if (n == 0) continue;
      h->launches += 2;
      k_set_shift<T><<<(n + 127) / 128, 128, 0, h->stream>>>(L.prm[L.pcur].as<T>(), n, L.ids.as<int>(),
                                                            I.ucell.as<T>(), h->nx * h->ny);
      dim3 gm((n + 127) / 128, L.k.nchunk);
      k_moments<S, T, D><<<gm, 128, 0, h->stream>>>(L.k, n, L.prm[L.pcur].as<T>(), h->spaces[L.space].vt.as<T>(),
                                                     L.f[L.cur].as<S>(), L.cpart.as<double>());
      L.fresh = false;
    }
    return cudaGetLastError();
  }

  // move every cell's phi~ from the old levels to the new ones (copy or level switch)
  static cudaError_t transfer(mlvs_handle* h, Inst& Old, Inst& New) {
    const int ncell = h->nx * h->ny;
    cudaError_t e = cudaSuccess;
    std::map<std::pair<int, int>, std::vector<MapItem>> groups;
    for (int c = 0; c < ncell; ++c) {
      const int lo = Old.lvl_of[c], ln = New.lvl_of[c];
      groups[{lo, ln}].push_back({Old.slot_of[c], New.slot_of[c], Old.slot_of[c]});
    }
    for (auto& g : groups) {
      LevelRt& Lo = Old.lv[g.first.first];
      LevelRt& Ln = New.lv[g.first.second];
      DevBuf items;
      e = upload(items, g.second, h->stream);
      if (e != cudaSuccess) return e;
      const int ni = (int)g.second.size();
      if (Lo.space == Ln.space) {
        ++h->launches;
        k_copy_cols<S><<<map_grid(ni), 256, 0, h->stream>>>(Lo.f[Lo.cur].as<S>(), (int)Lo.cells.size(),
                                                          Ln.f[0].as<S>(), (int)Ln.cells.size(), 2 * Ln.k.nv,
                                                          items.as<MapItem>(), ni);
      } else {
        CSR* c = nullptr;
        if (get_csr(h, Lo.space, Ln.space, &c) != MLVS_OK) return cudaErrorInvalidValue;
        MapArgs m = margs(h, Lo.space, Ln.space, c);
        m.src = Lo.f[Lo.cur].p;
        m.src_ld = (int)Lo.cells.size();
        m.dst = Ln.f[0].p;
        m.dst_ld = (int)Ln.cells.size();
        m.prm = nullptr;
        m.prm_ld = 0;
        m.items = items.as<MapItem>();
        m.nitems = ni;
        if (D == 2 && h->cfg.map_moments == 9) {
          // the nine-moment level switch (Sec. 3.3.2): projection plus the block correction
          DevBuf cnt;
          if ((e = cnt.alloc(sizeof(int))) != cudaSuccess) return e;
          if ((e = cudaMemsetAsync(cnt.p, 0, sizeof(int), h->stream)) != cudaSuccess) return e;
          ++h->launches;
          k_map9<S, S, T, SRC_TILDE><<<(ni + 127) / 128, 128, 0, h->stream>>>(m, cnt.as<int>());
          int hc = 0;
          if ((e = cudaMemcpyAsync(&hc, cnt.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
            return e;
          if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return e;
          if (hc) ++h->map9_singular;
          continue;
        }
        ++h->launches;
        launch_map<S, S, SRC_TILDE>(h, m);
        if (D == 2 && h->cfg.positive_mapping) {
          // the exponential correction where the additive result went negative (Sec. 3.3.2)
          DevBuf cnt;
          if ((e = cnt.alloc(2 * sizeof(int))) != cudaSuccess) return e;
          if ((e = cudaMemsetAsync(cnt.p, 0, 2 * sizeof(int), h->stream)) != cudaSuccess) return e;
          ++h->launches;
          k_expmap<S, S, T, SRC_TILDE><<<(ni + 127) / 128, 128, 0, h->stream>>>(m, cnt.as<int>());
          int hc[2] = {0, 0};
          if ((e = cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
            return e;
          if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return e;
          h->exp_corrected += hc[0];
          h->exp_failed += hc[1];
        }
      }
      e = cudaStreamSynchronize(h->stream);   // items freed at scope end
      if (e != cudaSuccess) return e;
    }
    for (auto& L : New.lv) { L.cur = 0; L.pcur = 0; }
    return cudaGetLastError();
  }

  // curvilinear walls: the wall-Maxwellian normalisation of every face of a level (once)
  static cudaError_t wall_table(mlvs_handle* h, LevelRt& L) {
    if constexpr (D == 2) {
      cudaError_t e = L.wden.alloc((size_t)L.k.nface * sizeof(double));
      if (e != cudaSuccess) return e;
      std::vector<double> wv(12);
      for (int s = 0; s < 4; ++s)
        for (int j = 0; j < 3; ++j) wv[3 * s + j] = h->cfg.wall[s][j];
      DevBuf wd;
      if ((e = upload(wd, wv, h->stream)) != cudaSuccess) return e;
      ++h->launches;
      k_wall_den_table<T, D><<<(L.k.nface * 32 + 127) / 128, 128, 0, h->stream>>>(
          L.k, h->gas, h->spaces[L.space].vt.as<T>(), h->fgeo_d.as<T>(), wd.as<double>(), L.wden.as<double>());
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      return cudaStreamSynchronize(h->stream);
    }
    return cudaSuccess;
  }

  // masks of the criterion (Sec. 3.2) of every cell of an instance into kout[ncell][N1*N1]
  // sel: the global ids of the cells to evaluate (null: every cell)
  static cudaError_t criterion(mlvs_handle* h, Inst& I, const mlvs_adapt_params& p, unsigned char* kout,
                               const std::vector<int>* sel) {
    const int nb = h->N1 * h->N1;
    // slots of the selected cells, level by level
    std::vector<int> slots, off(h->n_levels + 1, 0);
    if (sel) {
      std::vector<std::vector<int>> per(h->n_levels);
      for (int c : *sel) per[I.lvl_of[c]].push_back(I.slot_of[c]);
      for (int l = 0; l < h->n_levels; ++l) {
        off[l] = (int)slots.size();
        slots.insert(slots.end(), per[l].begin(), per[l].end());
      }
      off[h->n_levels] = (int)slots.size();
      cudaError_t e = upload(h->sel_d, slots, h->stream);
      if (e != cudaSuccess) return e;
    }
    // per-block transport sums in shared memory when they fit, else in a global scratch slice
    // per CTA, the cells then launched in batches of kCritBatch
    int tblk = 0;
    if (p.eps_merge > 0.0) tblk = (2ull + CB_N) * nb * sizeof(double) <= 220ull * 1024 ? 1 : 2;
    const size_t smem = (2ull + (tblk == 1 ? CB_N : 0)) * nb * sizeof(double);
    constexpr int kCritBatch = 2048;
    const size_t tb_bytes = (size_t)kCritBatch * CB_N * nb * sizeof(double);
    if (tblk == 2 && h->crit_tb.n < tb_bytes && h->crit_tb.alloc(tb_bytes) != cudaSuccess)
      return cudaErrorMemoryAllocation;
    cudaError_t e = cudaFuncSetAttribute(k_criterion<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int l = 0; l < h->n_levels; ++l) {
      LevelRt& L = I.lv[l];
      const int nsel = sel ? off[l + 1] - off[l] : (int)L.cells.size();
      if (nsel == 0) continue;
      const SpaceRt& sp = h->spaces[L.space];
      CritArgs a;
      a.sel = sel ? h->sel_d.as<int>() + off[l] : nullptr;
      a.f = L.f[L.cur].p;
      a.ns = (int)L.cells.size();
      a.nv = L.k.nv;
      a.ids = L.ids.as<int>();
      a.owner = sp.owner_d.as<int>();
      a.xi = sp.xid.as<double>();
      a.bx = h->bx_d.as<double>();
      a.bw = h->bw_d.as<double>();
      a.n = h->n_base;
      a.N1 = h->N1;
      a.g1 = h->g1_d.as<int>();
      a.pstart = h->pstart_d.as<int>();
      a.cstart = h->cstart_d.as<int>();
      for (int q = 0; q < 4; ++q) a.ng[q] = h->ng[q];
      a.kprev = sp.kp_d.as<unsigned char>();
      a.W1 = h->w1_d.as<double>();
      a.X1 = h->x1_d.as<double>();
      a.XX1 = h->xx1_d.as<double>();
      a.geo = sp.geo.as<double>();
      a.tblk = tblk;
      a.TBg = tblk == 2 ? h->crit_tb.as<double>() : nullptr;
      a.C_split = p.C_split;
      a.C_merge = p.C_merge;
      a.eps = p.eps_merge;
      a.max_level = p.max_level;
      a.kout = kout;
      const int batch = tblk == 2 ? kCritBatch : nsel;
      for (int b0 = 0; b0 < nsel; b0 += batch) {
        a.sel0 = b0;
        ++h->launches;
        k_criterion<S><<<std::min(batch, nsel - b0), CRIT_THREADS, smem, h->stream>>>(a);
      }
    }
    return cudaGetLastError();
  }
};

struct Ops {
  cudaError_t (*init_state)(mlvs_handle*, Inst&, const double*);
  cudaError_t (*finalize_cells)(mlvs_handle*, Inst&, LevelRt&);
  cudaError_t (*step)(mlvs_handle*, Inst&);
  cudaError_t (*transfer)(mlvs_handle*, Inst&, Inst&);
  cudaError_t (*moments_of_levels)(mlvs_handle*, Inst&);
  cudaError_t (*criterion)(mlvs_handle*, Inst&, const mlvs_adapt_params&, unsigned char*, const std::vector<int>*);
  cudaError_t (*wall_table)(mlvs_handle*, LevelRt&);
  cudaError_t (*ghost_batch)(mlvs_handle*, Inst&);
  cudaError_t (*flux_batch)(mlvs_handle*, Inst&);
  cudaError_t (*tile_batch)(mlvs_handle*, Inst&);
  cudaError_t (*group_capture)(mlvs_handle* const*, int, mlvs_handle::GroupBufs&, std::vector<int>&,
                               cudaGraphExec_t*);
};

template <class S, class T, int D> Ops make_ops() {
  using R = Runner<S, T, D>;
  return Ops{&R::init_state, &R::finalize_cells, &R::step, &R::transfer, &R::moments_of_levels, &R::criterion,
             &R::wall_table, &R::ghost_batch, &R::flux_batch, &R::tile_batch, &R::group_capture};
}

Ops ops_for(int storage, int D) {
  if (storage == MLVS_F64) return D == 2 ? make_ops<double, double, 2>() : make_ops<double, double, 1>();
  if (storage == MLVS_F32) return D == 2 ? make_ops<float, float, 2>() : make_ops<float, float, 1>();
  return D == 2 ? make_ops<__nv_bfloat16, float, 2>() : make_ops<__nv_bfloat16, float, 1>();
}

int choose_vpc(int tile_ctas, int nv, int target) {
  // about `target` CTAs (default four per SM of the 148), at most 384 velocities per chunk
  int nchunk = std::max(1, (target + std::max(tile_ctas, 1) - 1) / std::max(tile_ctas, 1));
  nchunk = std::min(nchunk, nv);
  int vpc = (nv + nchunk - 1) / nchunk;
  vpc = (vpc + 1) & ~1;   // even: the tile kernels take the velocities in pairs
  return std::max(2, std::min(vpc, kMaxVpc));
}

}  // namespace

// ---------------------------------------------------------------------------------------
// level structure of one instance

static int wrapc(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Build the level structure of an instance for a cell -> level assignment (host only).
// a side whose faces carry a boundary distribution (wall or freestream)
static bool bnd(int bc) { return bc == MLVS_BC_WALL || bc == MLVS_BC_FREESTREAM; }

static mlvs_status build_levels(mlvs_handle* h, const std::vector<int>& lvl_of, Inst& I) {
  ++h->epoch;
  const int D = h->D, nx = h->nx, ny = h->ny, ncell = nx * ny;
  const int px = h->cfg.bc[0] == MLVS_BC_PERIODIC;
  const int py = D == 2 ? (h->cfg.bc[2] == MLVS_BC_PERIODIC) : 1;
  const int nfx = px ? nx : nx + 1;
  const int nfy = D == 2 ? (py ? ny : ny + 1) : 0;
  const int nface = nfx * ny + (D == 2 ? nx * nfy : 0);
  const int TX = tile_w(D), TY = tile_h(D);
  const int ntx = (nx + TX - 1) / TX;
  I.lvl_of = lvl_of;
  I.slot_of.assign(ncell, -1);
  I.lv.clear();
  I.lv.resize(h->n_levels);
  for (int l = 0; l < h->n_levels; ++l) I.lv[l].space = h->level_space[l];
  for (int c = 0; c < ncell; ++c) {
    const int l = lvl_of[c];
    I.slot_of[c] = (int)I.lv[l].cells.size();
    I.lv[l].cells.push_back(c);
  }
  // faces: roles, cross-level routes
  std::map<int, int> face_level_of_space;   // face levels (no cells) by space
  std::map<std::pair<int, int>, int> space_of_pair;   // common refinement of two cell levels
  std::vector<std::vector<unsigned char>> role(h->n_levels);
  std::vector<std::vector<int>> slot(h->n_levels);
  auto ensure = [&](int l) {
    if ((int)role.size() <= l) { role.resize(l + 1); slot.resize(l + 1); }
    if (role[l].empty()) { role[l].assign(nface, FR_NONE); slot[l].assign(nface, -1); }
  };
  for (int l = 0; l < h->n_levels; ++l) ensure(l);
  std::vector<int> nX, nY;
  auto bump = [&](std::vector<int>& v, int l) { if ((int)v.size() <= l) v.resize(l + 1, 0); return v[l]++; };
  std::map<std::pair<int, int>, std::vector<MapItem>> flux_items;
  std::vector<std::array<int, 3>> face_cells(nface);   // cL, cR, wall-side (-1 none)
  I.n_int = 0;
  I.n_cross = 0;
  for (int f = 0; f < nface; ++f) {
    int cL, cR, wall = -1;
    if (f < nfx * ny) {
      const int gj = f / nfx, gi = f % nfx;
      cL = wrapc(gj, ny, py) * nx + wrapc(gi - 1, nx, px);
      cR = wrapc(gj, ny, py) * nx + wrapc(gi, nx, px);
      if (!px && gi == 0 && bnd(h->cfg.bc[0])) wall = 0;
      if (!px && gi == nx && bnd(h->cfg.bc[1])) wall = 1;
    } else {
      const int r = f - nfx * ny, gj = r / nx, gi = r % nx;
      cL = wrapc(gj - 1, ny, py) * nx + gi;
      cR = wrapc(gj, ny, py) * nx + gi;
      if (!py && gj == 0 && bnd(h->cfg.bc[2])) wall = 2;
      if (!py && gj == ny && bnd(h->cfg.bc[3])) wall = 3;
    }
    face_cells[f] = {cL, cR, wall};
    const int lL = lvl_of[cL], lR = lvl_of[cR];
    if (wall >= 0) {
      const int c = (wall == 0 || wall == 2) ? cR : cL;
      role[lvl_of[c]][f] = FR_NORMAL;
      continue;
    }
    ++I.n_int;
    if (lL == lR) { role[lL][f] = FR_NORMAL; continue; }
    ++I.n_cross;
    // cross-level face: evaluated on the common refinement of the two spaces (Sec. 3.4),
    // which depends only on the pair of levels
    int sf;
    const std::pair<int, int> pair_key(std::min(lL, lR), std::max(lL, lR));
    auto pit = space_of_pair.find(pair_key);
    if (pit != space_of_pair.end()) {
      sf = pit->second;
    } else {
      const SpaceRt& SL = h->spaces[h->level_space[lL]];
      const SpaceRt& SR = h->spaces[h->level_space[lR]];
      std::vector<int> km(SL.keff.size());
      for (size_t b = 0; b < km.size(); ++b) km[b] = std::min(SL.keff[b], SR.keff[b]);
      mlvs_status st = get_space(h, km, &sf);
      if (st != MLVS_OK) return st;
      space_of_pair[pair_key] = sf;
    }
    int lf;
    if (sf == h->level_space[lL]) lf = lL;
    else if (sf == h->level_space[lR]) lf = lR;
    else {
      auto it = face_level_of_space.find(sf);
      if (it == face_level_of_space.end()) {
        lf = (int)I.lv.size();
        I.lv.emplace_back();
        I.lv[lf].space = sf;
        I.lv[lf].real = false;
        face_level_of_space[sf] = lf;
      } else {
        lf = it->second;
      }
    }
    ensure(lf);
    role[lf][f] = FR_CROSS;
    slot[lf][f] = bump(nX, lf);
    for (int c : {cL, cR}) {
      const int lc = lvl_of[c];
      if (lc == lf) continue;
      if (role[lc][f] == FR_RECV) continue;       // both sides on one level
      role[lc][f] = FR_RECV;
      slot[lc][f] = bump(nY, lc);
      flux_items[{lf, lc}].push_back({slot[lf][f], slot[lc][f], f});
    }
  }
  const int nlev = (int)I.lv.size();
  nX.resize(nlev, 0);
  nY.resize(nlev, 0);
  // ghosts: stencil cells of the faces evaluated on a level that live on another level
  std::vector<std::vector<int>> ghost_col(nlev);
  for (int l = 0; l < nlev; ++l) {
    std::set<int> gset;
    for (int f = 0; f < nface; ++f) {
      if (role[l][f] != FR_NORMAL && role[l][f] != FR_CROSS) continue;
      int st[8], ns = 0;   // the face's stencil cells: four normal, four tangential
      if (f < nfx * ny) {
        const int gj = f / nfx, gi = f % nfx;
        for (int d = -2; d <= 1; ++d) st[ns++] = wrapc(gj, ny, py) * nx + wrapc(gi + d, nx, px);
        if (D == 2)
          for (int d : {-1, 1})
            for (int e : {-1, 0}) st[ns++] = wrapc(gj + d, ny, py) * nx + wrapc(gi + e, nx, px);
      } else {
        const int r = f - nfx * ny, gj = r / nx, gi = r % nx;
        for (int d = -2; d <= 1; ++d) st[ns++] = wrapc(gj + d, ny, py) * nx + gi;
        for (int d : {-1, 1})
          for (int e : {-1, 0}) st[ns++] = wrapc(gj + e, ny, py) * nx + wrapc(gi + d, nx, px);
      }
      for (int q = 0; q < ns; ++q)
        if (lvl_of[st[q]] != l) gset.insert(st[q]);
    }
    I.lv[l].ghost_cells.assign(gset.begin(), gset.end());
    ghost_col[l].assign(ncell, -1);
    for (size_t g = 0; g < I.lv[l].ghost_cells.size(); ++g) ghost_col[l][I.lv[l].ghost_cells[g]] = (int)g;
    I.lv[l].nghost = (int)I.lv[l].ghost_cells.size();
  }
  // routes
  I.ghosts.clear();
  for (int l = 0; l < nlev; ++l) {
    std::map<int, std::vector<MapItem>> by_src;
    for (size_t g = 0; g < I.lv[l].ghost_cells.size(); ++g) {
      const int c = I.lv[l].ghost_cells[g];
      by_src[lvl_of[c]].push_back({I.slot_of[c], (int)g, I.slot_of[c]});
    }
    for (auto& s : by_src) {
      Route r;
      r.src = s.first;
      r.dst = l;
      r.items = s.second;
      I.ghosts.push_back(std::move(r));
    }
  }
  I.fluxes.clear();
  for (auto& fi : flux_items) {
    Route r;
    r.src = fi.first.first;
    r.dst = fi.first.second;
    r.items = fi.second;
    I.fluxes.push_back(std::move(r));
  }
  // tiles: tiles with a cell of the level or owning a face evaluated on it
  std::vector<std::vector<int>> tls(nlev);
  int all_tiles = 0;
  for (int l = 0; l < nlev; ++l) {
    std::set<int> ts;
    for (int c : I.lv[l].cells) ts.insert(((c / nx) / TY) * ntx + (c % nx) / TX);
    for (int f = 0; f < nface; ++f) {
      if (role[l][f] == FR_NONE) continue;
      int col, row;
      if (f < nfx * ny) { row = f / nfx; col = std::min(f % nfx, nx - 1); }
      else { const int r = f - nfx * ny; col = r % nx; row = std::min(r / nx, ny - 1); }
      ts.insert((row / TY) * ntx + col / TX);
    }
    tls[l].assign(ts.begin(), ts.end());
    all_tiles += (int)tls[l].size();
  }
  for (int l = 0; l < nlev; ++l) {
    const std::vector<int>& tl = tls[l];
    I.lv[l].ntiles = (int)tl.size();
    I.lv[l].tiles_h = tl;
    I.lv[l].nX = nX[l];
    I.lv[l].nY = nY[l];
    LevelRt& L = I.lv[l];
    StepConst& k = L.k;
    k.nx = nx; k.ny = ny; k.px = px; k.py = py;
    for (int s = 0; s < 4; ++s) k.bc[s] = h->cfg.bc[s];
    if (D == 1) k.bc[2] = k.bc[3] = MLVS_BC_PERIODIC;
    k.nfx = nfx; k.nfy = nfy; k.ncell = ncell; k.nface = nface;
    const SpaceRt& sp = h->spaces[L.space];
    k.nv = sp.vs.nv();
    k.nax = sp.nax;
    k.dx = h->dx; k.dy = h->dy; k.dt = h->dt;
    k.c0 = h->gas.K + 3.0 - D;
    k.twoK = 2.0 * h->gas.K;
    // every level's tiles go in one launch: the chunking aims at the CTA target over all of them
    k.vpc = choose_vpc(all_tiles, k.nv, h->cta_target);
    k.nchunk = (k.nv + k.vpc - 1) / k.vpc;
    // device tables
    CK(upload(L.tiles, tl, h->stream));
    CK(upload(L.ids, L.cells, h->stream));
    CK(upload(L.frole, role[l], h->stream));
    {
      std::vector<int> fl;
      for (int f = 0; f < nface; ++f)
        if (role[l][f] == FR_NORMAL || role[l][f] == FR_CROSS) fl.push_back(f);
      L.nflist = (int)fl.size();
      if (L.nflist < nface && L.nflist > 0) CK(upload(L.flist, fl, h->stream));
    }
    CK(upload(L.fslot, slot[l], h->stream));
    CK(upload(L.ghost_of, ghost_col[l], h->stream));
    {
      std::vector<int> xf(nX[l], 0);
      for (int f = 0; f < nface; ++f)
        if (role[l][f] == FR_CROSS) xf[slot[l][f]] = f;
      CK(upload(L.xfid, xf, h->stream));
    }
    const size_t nc = L.cells.size();
    const size_t fbytes = 2ull * k.nv * nc * h->ssize;
    if (L.f[0].alloc(fbytes) != cudaSuccess || L.f[1].alloc(fbytes) != cudaSuccess ||
        L.prm[0].alloc((size_t)NP * std::max<size_t>(nc, 1) * h->tsize) != cudaSuccess ||
        L.prm[1].alloc((size_t)NP * std::max<size_t>(nc, 1) * h->tsize) != cudaSuccess ||
        L.fprm.alloc((size_t)NP * nface * h->tsize) != cudaSuccess ||
        L.cpart.alloc((size_t)k.nchunk * NMOM * std::max<size_t>(nc, 1) * 8) != cudaSuccess ||
        L.fpart.alloc((size_t)k.nchunk * NMOM * nface * 8) != cudaSuccess ||
        L.ghost.alloc(2ull * k.nv * L.nghost * h->tsize) != cudaSuccess ||
        L.X.alloc(2ull * k.nv * L.nX * h->tsize) != cudaSuccess ||
        L.Y.alloc(2ull * k.nv * L.nY * h->tsize) != cudaSuccess ||
        L.fbar.alloc(L.ntiles > 0 ? 2ull * ((k.nv + 1) / 2) * 2 * nface * h->tsize : 0) != cudaSuccess)
      return fail(h, MLVS_ERR_OOM, "device allocation of a level failed");
    CK(cudaMemsetAsync(L.fprm.p, 0, L.fprm.n, h->stream));
    if (h->cfg.compat_moments == 8) {
      const size_t n8 = 4ull * std::max<size_t>(nc, 1) * h->tsize;
      if (L.prm8[0].alloc(n8) != cudaSuccess || L.prm8[1].alloc(n8) != cudaSuccess ||
          L.fprm8.alloc(4ull * nface * h->tsize) != cudaSuccess)
        return fail(h, MLVS_ERR_OOM, "device allocation of a level failed");
      CK(cudaMemsetAsync(L.prm8[0].p, 0, n8, h->stream));
      CK(cudaMemsetAsync(L.prm8[1].p, 0, n8, h->stream));
      CK(cudaMemsetAsync(L.fprm8.p, 0, L.fprm8.n, h->stream));
    }
    if (h->curvi) CK(ops_for(h->cfg.storage, D).wall_table(h, L));
    if (L.msum.alloc((size_t)NMOM * std::max<size_t>(std::max<size_t>(nface, nc), 1) * sizeof(double)) != cudaSuccess)
      return fail(h, MLVS_ERR_OOM, "device allocation of a level failed");
    {
      const size_t np = std::max<size_t>(std::max<size_t>(nface, nc), 1);
      const size_t nscr = h->cfg.compat_moments == 8 ? (size_t)FIN_SCR8 : (size_t)FIN_SCR;
      if (L.fscr.alloc(nscr * np * sizeof(double)) != cudaSuccess || L.fneed.alloc(np * sizeof(int)) != cudaSuccess)
        return fail(h, MLVS_ERR_OOM, "device allocation of a level failed");
    }
  }
  for (auto& r : I.ghosts) CK(upload(r.items_d, r.items, h->stream));
  for (auto& r : I.fluxes) CK(upload(r.items_d, r.items, h->stream));
  CK(ops_for(h->cfg.storage, D).ghost_batch(h, I));
  CK(ops_for(h->cfg.storage, D).flux_batch(h, I));
  CK(upload(I.lvl_of_d, I.lvl_of, h->stream));
  CK(upload(I.slot_of_d, I.slot_of, h->stream));
  return MLVS_OK;
}

// ---------------------------------------------------------------------------------------

// Geometry of a structured curvilinear mesh from its nodes [ny+1][nx+1][2] (FP64): cells
// A=(i,j), B=(i+1,j), C=(i+1,j+1), D=(i,j+1) counter-clockwise; area from the diagonals,
// centroid of the triangles ABC and ACD, J^{-T} from the mean edge vectors; i-faces from
// node (i,j) to (i,j+1) with n = (e_y, -e_x)/|e|, j-faces from (i,j) to (i+1,j) with
// n = (-e_y, e_x)/|e|; per face the offsets x_b - x_c of both neighbours, the centroid of
// a periodic image moved by the period, the first ghost's reflected through the face.
static mlvs_status build_geometry(mlvs_handle* h, const double* xy) {
  const int nx = h->nx, ny = h->ny, nc = nx * ny;
  const int px = h->cfg.bc[0] == MLVS_BC_PERIODIC, py = h->cfg.bc[2] == MLVS_BC_PERIODIC;
  const int nfx = px ? nx : nx + 1, nfy = py ? ny : ny + 1;
  const int nface = nfx * ny + nx * nfy;
  auto X = [&](int j, int i) { return xy[2 * ((size_t)j * (nx + 1) + i)]; };
  auto Y = [&](int j, int i) { return xy[2 * ((size_t)j * (nx + 1) + i) + 1]; };
  auto cross = [](double ux, double uy, double vx, double vy) { return ux * vy - uy * vx; };
  h->cgeo.assign(5 * (size_t)nc, 0.0);
  std::vector<double> cx(nc), cy(nc);
  double lmin = 1e300;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double Ax = X(j, i), Ay = Y(j, i), Bx = X(j, i + 1), By = Y(j, i + 1);
      const double Cx = X(j + 1, i + 1), Cy = Y(j + 1, i + 1), Dx = X(j + 1, i), Dy = Y(j + 1, i);
      const double area = 0.5 * cross(Cx - Ax, Cy - Ay, Dx - Bx, Dy - By);
      if (!(area > 0.0)) return fail(h, MLVS_ERR_ARG, "mesh cells must be counter-clockwise with positive area");
      const double a1 = 0.5 * cross(Bx - Ax, By - Ay, Cx - Ax, Cy - Ay);
      const double a2 = 0.5 * cross(Cx - Ax, Cy - Ay, Dx - Ax, Dy - Ay);
      const int c = j * nx + i;
      cx[c] = (a1 * (Ax + Bx + Cx) + a2 * (Ax + Cx + Dx)) / (3.0 * area);
      cy[c] = (a1 * (Ay + By + Cy) + a2 * (Ay + Cy + Dy)) / (3.0 * area);
      const double dix = 0.5 * ((Bx - Ax) + (Cx - Dx)), diy = 0.5 * ((By - Ay) + (Cy - Dy));
      const double djx = 0.5 * ((Dx - Ax) + (Cx - Bx)), djy = 0.5 * ((Dy - Ay) + (Cy - By));
      const double det = dix * djy - djx * diy;
      h->cgeo[c] = djy / det;
      h->cgeo[nc + c] = -diy / det;
      h->cgeo[2 * (size_t)nc + c] = -djx / det;
      h->cgeo[3 * (size_t)nc + c] = dix / det;
      h->cgeo[4 * (size_t)nc + c] = area;
      const double l1 = std::hypot(Dx - Ax, Dy - Ay), l2 = std::hypot(Cx - Bx, Cy - By);
      const double l3 = std::hypot(Bx - Ax, By - Ay), l4 = std::hypot(Cx - Dx, Cy - Dy);
      const double wdt = area / std::max(std::max(l1, l2), std::max(l3, l4));
      lmin = std::min(lmin, wdt);
      h->width.push_back(wdt);
    }
  h->lmin = lmin;
  // translation of the periodic images
  double sxx = 0, sxy = 0, syx = 0, syy = 0;
  for (int j = 0; j <= ny; ++j) { sxx += X(j, nx) - X(j, 0); sxy += Y(j, nx) - Y(j, 0); }
  for (int i = 0; i <= nx; ++i) { syx += X(ny, i) - X(0, i); syy += Y(ny, i) - Y(0, i); }
  sxx /= ny + 1; sxy /= ny + 1; syx /= nx + 1; syy /= nx + 1;
  h->fgeo.assign(7 * (size_t)nface, 0.0);
  auto put = [&](int f, double nxv, double nyv, double len, double bx, double by, double lx, double ly,
                 double rx, double ry) {
    double* g = h->fgeo.data();
    g[f] = nxv; g[nface + f] = nyv; g[2 * (size_t)nface + f] = len;
    g[3 * (size_t)nface + f] = bx - lx; g[4 * (size_t)nface + f] = by - ly;
    g[5 * (size_t)nface + f] = bx - rx; g[6 * (size_t)nface + f] = by - ry;
  };
  for (int j = 0; j < ny; ++j)
    for (int p = 0; p < nfx; ++p) {
      const double ex = X(j + 1, p) - X(j, p), ey = Y(j + 1, p) - Y(j, p);
      const double len = std::hypot(ex, ey);
      const double bx = 0.5 * (X(j, p) + X(j + 1, p)), by = 0.5 * (Y(j, p) + Y(j + 1, p));
      double lx, ly, rx, ry;
      if (p == 0) {
        if (px) { lx = cx[j * nx + nx - 1] - sxx; ly = cy[j * nx + nx - 1] - sxy; }
        else { lx = 2.0 * bx - cx[j * nx]; ly = 2.0 * by - cy[j * nx]; }
      } else { lx = cx[j * nx + p - 1]; ly = cy[j * nx + p - 1]; }
      if (p == nx) { rx = 2.0 * bx - cx[j * nx + nx - 1]; ry = 2.0 * by - cy[j * nx + nx - 1]; }
      else { rx = cx[j * nx + p]; ry = cy[j * nx + p]; }
      put(j * nfx + p, ey / len, -ex / len, len, bx, by, lx, ly, rx, ry);
    }
  for (int p = 0; p < nfy; ++p)
    for (int i = 0; i < nx; ++i) {
      const double ex = X(p, i + 1) - X(p, i), ey = Y(p, i + 1) - Y(p, i);
      const double len = std::hypot(ex, ey);
      const double bx = 0.5 * (X(p, i) + X(p, i + 1)), by = 0.5 * (Y(p, i) + Y(p, i + 1));
      double lx, ly, rx, ry;
      if (p == 0) {
        if (py) { lx = cx[(ny - 1) * nx + i] - syx; ly = cy[(ny - 1) * nx + i] - syy; }
        else { lx = 2.0 * bx - cx[i]; ly = 2.0 * by - cy[i]; }
      } else { lx = cx[(p - 1) * nx + i]; ly = cy[(p - 1) * nx + i]; }
      if (p == ny) { rx = 2.0 * bx - cx[(ny - 1) * nx + i]; ry = 2.0 * by - cy[(ny - 1) * nx + i]; }
      else { rx = cx[p * nx + i]; ry = cy[p * nx + i]; }
      put(nfx * ny + p * nx + i, -ey / len, ex / len, len, bx, by, lx, ly, rx, ry);
    }
  h->curvi = true;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_mesh_geometry(int nx, int ny, int periodic_x, int periodic_y, const double* node_xy,
                                          double* cell_geo, double* face_geo, double* width) {
  if (!node_xy || !cell_geo || !face_geo || nx < 1 || ny < 1)
    return fail(nullptr, MLVS_ERR_ARG, "mlvs_mesh_geometry: bad argument");
  // the same construction a handle runs, on a host-only handle (no device resources)
  mlvs_handle tmp;
  std::memset(&tmp.cfg, 0, sizeof(tmp.cfg));
  tmp.nx = nx;
  tmp.ny = ny;
  tmp.cfg.bc[0] = tmp.cfg.bc[1] = periodic_x ? MLVS_BC_PERIODIC : MLVS_BC_WALL;
  tmp.cfg.bc[2] = tmp.cfg.bc[3] = periodic_y ? MLVS_BC_PERIODIC : MLVS_BC_WALL;
  const mlvs_status st = build_geometry(&tmp, node_xy);
  if (st != MLVS_OK) return fail(nullptr, st, "mlvs_mesh_geometry: " + tmp.err);
  std::memcpy(cell_geo, tmp.cgeo.data(), tmp.cgeo.size() * sizeof(double));
  std::memcpy(face_geo, tmp.fgeo.data(), tmp.fgeo.size() * sizeof(double));
  if (width) std::memcpy(width, tmp.width.data(), tmp.width.size() * sizeof(double));
  return MLVS_OK;
}

// Device copies of the curvilinear geometry in the compute type; dt/|V| needs dt.
static mlvs_status upload_geometry(mlvs_handle* h) {
  const size_t nc = (size_t)h->nx * h->ny;
  std::vector<double> c(h->cgeo);
  for (size_t i = 0; i < nc; ++i) c[4 * nc + i] = h->dt / h->cgeo[4 * nc + i];
  if (h->tsize == 8) {
    CK(upload(h->cgeo_d, c, h->stream));
    CK(upload(h->fgeo_d, h->fgeo, h->stream));
  } else {
    CK(upload(h->cgeo_d, std::vector<float>(c.begin(), c.end()), h->stream));
    CK(upload(h->fgeo_d, std::vector<float>(h->fgeo.begin(), h->fgeo.end()), h->stream));
  }
  std::vector<double> fg(5 * nc);
  for (size_t i = 0; i < 4 * nc; ++i) fg[i] = h->cgeo[i];
  for (size_t i = 0; i < nc; ++i) fg[4 * nc + i] = h->width[i];
  CK(upload(h->featgeo_d, fg, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_create(const mlvs_config* cfg, mlvs_handle** out) {
  mlvs_handle* h = nullptr;
  if (!cfg || !out) return fail(nullptr, MLVS_ERR_ARG, "null argument");
  *out = nullptr;
  if (cfg->dim != 1 && cfg->dim != 2) return fail(nullptr, MLVS_ERR_ARG, "dim must be 1 or 2");
  if (cfg->n_instances < 1) return fail(nullptr, MLVS_ERR_ARG, "n_instances < 1");
  if (cfg->nx < 1 || cfg->ny < 1 || (cfg->dim == 1 && cfg->ny != 1))
    return fail(nullptr, MLVS_ERR_ARG, "bad mesh size (dim 1 needs ny = 1)");
  if (!(cfg->Lx > 0) || (cfg->dim == 2 && !(cfg->Ly > 0))) return fail(nullptr, MLVS_ERR_ARG, "bad domain size");
  for (int s = 0; s < 4; ++s)
    if (cfg->bc[s] < 0 || cfg->bc[s] > 3) return fail(nullptr, MLVS_ERR_ARG, "unknown boundary kind");
  for (int s = 0; s < 4; ++s)
    if (cfg->bc[s] == MLVS_BC_FREESTREAM && (!(cfg->far[0] > 0) || !(cfg->far[3] > 0)))
      return fail(nullptr, MLVS_ERR_ARG, "freestream sides need rho > 0 and T > 0 in cfg->far");
  if ((cfg->bc[0] == MLVS_BC_PERIODIC) != (cfg->bc[1] == MLVS_BC_PERIODIC) ||
      (cfg->dim == 2 && (cfg->bc[2] == MLVS_BC_PERIODIC) != (cfg->bc[3] == MLVS_BC_PERIODIC)))
    return fail(nullptr, MLVS_ERR_ARG, "periodic sides must come in pairs");
  if (cfg->storage < 0 || cfg->storage > 2) return fail(nullptr, MLVS_ERR_ARG, "unknown storage type");
  if (cfg->map_moments != 0 && cfg->map_moments != 4 && cfg->map_moments != 9)
    return fail(nullptr, MLVS_ERR_ARG, "map_moments must be 4 or 9 (0: 4)");
  if (cfg->compat_moments != 0 && cfg->compat_moments != 4 && cfg->compat_moments != 8)
    return fail(nullptr, MLVS_ERR_ARG, "compat_moments must be 4 or 8 (0: 4)");
  if (cfg->compat_moments == 8 && cfg->dim != 2)
    return fail(nullptr, MLVS_ERR_ARG, "the eight-moment correction is two-dimensional");
  if (cfg->positive_mapping != 0 && cfg->positive_mapping != 1)
    return fail(nullptr, MLVS_ERR_ARG, "positive_mapping must be 0 or 1");
  if (!(cfg->R > 0) || !(cfg->Pr > 0) || cfg->K_internal < 0) return fail(nullptr, MLVS_ERR_ARG, "bad gas constants");
  if (!(cfg->mu_ref > 0) && !(cfg->Kn > 0)) return fail(nullptr, MLVS_ERR_ARG, "need mu_ref > 0 or Kn > 0");
  if (!(cfg->dt > 0) && !(cfg->cfl > 0)) return fail(nullptr, MLVS_ERR_ARG, "need dt > 0 or cfl > 0");
  if (!cfg->init_W) return fail(nullptr, MLVS_ERR_ARG, "init_W is null");
  const size_t ncell = (size_t)cfg->nx * cfg->ny;
  for (size_t i = 0; i < ncell * cfg->n_instances; ++i) {
    const double* w = cfg->init_W + 4 * i;
    if (!(w[0] > 0) || !(w[3] > 0) || !std::isfinite(w[1]) || !std::isfinite(w[2]))
      return fail(nullptr, MLVS_ERR_ARG, "init_W needs rho > 0, T > 0 and finite velocity");
  }
  h = new (std::nothrow) mlvs_handle();
  if (!h) return fail(nullptr, MLVS_ERR_OOM, "host allocation failed");
  h->cfg = *cfg;
  h->initW.assign(cfg->init_W, cfg->init_W + 4 * ncell * cfg->n_instances);
  h->cfg.init_W = nullptr;
  h->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
  h->D = cfg->dim;
  h->nx = cfg->nx;
  h->ny = cfg->ny;
  h->dx = cfg->Lx / cfg->nx;
  h->dy = cfg->dim == 2 ? cfg->Ly / cfg->ny : 1.0;
  const double Tref = cfg->T_ref > 0 ? cfg->T_ref : 1.0;
  h->gas.R = cfg->R;
  h->gas.K = cfg->K_internal;
  h->gas.Pr = cfg->Pr;
  h->gas.omega = cfg->omega;
  h->gas.T_ref = Tref;
  h->gas.mu_ref = cfg->mu_ref > 0 ? cfg->mu_ref
                                  : vhs_mu_ref(cfg->Kn, cfg->omega, cfg->rho_ref > 0 ? cfg->rho_ref : 1.0, cfg->R,
                                               Tref, cfg->L_ref > 0 ? cfg->L_ref : 1.0);
  h->tsize = cfg->storage == MLVS_F64 ? 8 : 4;
  h->ssize = cfg->storage == MLVS_F64 ? 8 : (cfg->storage == MLVS_F32 ? 4 : 2);
  static std::atomic<unsigned long long> next_uid{1};
  h->uid = next_uid++;
  if (cfg->mesh_kind == 1) {
    if (!cfg->node_xy || cfg->dim != 2) {
      delete h;
      return fail(nullptr, MLVS_ERR_ARG, "a curvilinear mesh needs dim 2 and node_xy");
    }
    mlvs_status gs = build_geometry(h, cfg->node_xy);
    if (gs != MLVS_OK) {
      const std::string m = h->err;
      delete h;
      return fail(nullptr, gs, m);
    }
    h->cfg.node_xy = nullptr;
  } else if (cfg->mesh_kind != 0) {
    delete h;
    return fail(nullptr, MLVS_ERR_ARG, "mesh_kind must be 0 (box) or 1 (curvilinear)");
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    delete h;
    return fail(nullptr, MLVS_ERR_CUDA, "cudaEventCreate failed");
  }
  *out = h;
  return MLVS_OK;
}

extern "C" void mlvs_destroy(mlvs_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ea0) cudaEventDestroy(h->ea0);
  if (h->ea1) cudaEventDestroy(h->ea1);
  if (h->kbuf_host) cudaFreeHost(h->kbuf_host);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.second.first);
  for (auto& g : h->gbufs)
    if (g.second.host) cudaFreeHost(g.second.host);
  for (auto s : h->branch) cudaStreamDestroy(s);
  for (auto e : h->bev) cudaEventDestroy(e);
  for (auto e : h->ev_pre) cudaEventDestroy(e);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_post) cudaEventDestroy(h->ev_post);
  delete h;
}

void mlvs_internal_set_error(const char* msg) { g_create_error = msg ? msg : ""; }

extern "C" const char* mlvs_last_error(const mlvs_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" mlvs_status mlvs_time_step(const mlvs_handle* h, double* dt) {
  if (!h || !dt) return MLVS_ERR_ARG;
  if (!h->ready) return MLVS_ERR_STATE;
  *dt = h->dt;
  return MLVS_OK;
}

static mlvs_status check_flags(mlvs_handle* h) {
  for (size_t n = 0; n < h->inst.size(); ++n) {
    Inst& I = h->inst[n];
    int e[ERR_WORDS] = {0};
    CK(cudaMemcpyAsync(e, I.err.p, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e[0]) {
      mlvs_status s = (e[0] & ERR_NONFINITE) ? MLVS_ERR_NONFINITE
                      : (e[0] & ERR_POSITIVITY) ? MLVS_ERR_POSITIVITY : MLVS_ERR_SINGULAR;
      h->sticky = s;
      char msg[256];
      if (e[1]) {
        double d[2];
        std::memcpy(d, e + 4, sizeof(d));
        std::snprintf(msg, sizeof(msg),
                      "device reported a non-finite, non-positive or singular state (instance %zu, first at "
                      "%s %d of its level: rho = %.6g, T = %.6g)", n, e[3] ? "face" : "cell", e[2], d[0], d[1]);
      } else {
        std::snprintf(msg, sizeof(msg), "device reported a non-finite, non-positive or singular state (instance %zu)", n);
      }
      return fail(h, s, msg);
    }
  }
  return MLVS_OK;
}

// Base-grid tables of the criterion: nodes, weights, level-1 group starts, and for every
// level L the first level-1 block (pstart) and first level-(L-1) group (cstart) of each
// level-L group.  The groups are nested, so both are exact starts.
static mlvs_status build_criterion_tables(mlvs_handle* h, int n) {
  auto g1 = groups_1d(n, 1);
  const int N1 = (int)g1.size();
  h->N1 = N1;
  std::vector<int> g1s(N1 + 1), ps(4 * (N1 + 1), 0), cs(4 * (N1 + 1), 0);
  for (int b = 0; b < N1; ++b) g1s[b] = g1[b].first;
  g1s[N1] = n;
  std::vector<std::vector<std::pair<int, int>>> gl(4);
  for (int L = 0; L <= 3; ++L) gl[L] = groups_1d(n, L);
  h->ng[0] = n;
  for (int L = 1; L <= 3; ++L) {
    const int ngL = (int)gl[L].size();
    h->ng[L] = ngL;
    for (int q = 0; q < ngL; ++q) {
      int b = 0;
      while (b < N1 && g1[b].first != gl[L][q].first) ++b;
      if (b == N1) return fail(h, MLVS_ERR_ARG, "velocity groups are not nested");
      ps[L * (N1 + 1) + q] = b;
      if (L >= 2) {
        int c = 0;
        const int ngc = (int)gl[L - 1].size();
        while (c < ngc && gl[L - 1][c].first != gl[L][q].first) ++c;
        if (c == ngc) return fail(h, MLVS_ERR_ARG, "velocity groups are not nested");
        cs[L * (N1 + 1) + q] = c;
      }
    }
    ps[L * (N1 + 1) + ngL] = N1;
    if (L >= 2) cs[L * (N1 + 1) + ngL] = (int)gl[L - 1].size();
  }
  CK(upload(h->bx_d, h->base.x, h->stream));
  CK(upload(h->bw_d, h->base.w, h->stream));
  CK(upload(h->g1_d, g1s, h->stream));
  CK(upload(h->pstart_d, ps, h->stream));
  CK(upload(h->cstart_d, cs, h->stream));
  std::vector<double> W1(N1, 0.0), X1(N1, 0.0), XX1(N1, 0.0);
  for (int b = 0; b < N1; ++b)
    for (int i = g1[b].first; i < g1[b].second; ++i) {
      W1[b] += h->base.w[i];
      X1[b] += h->base.w[i] * h->base.x[i];
      XX1[b] += h->base.w[i] * h->base.x[i] * h->base.x[i];
    }
  CK(upload(h->w1_d, W1, h->stream));
  CK(upload(h->x1_d, X1, h->stream));
  CK(upload(h->xx1_d, XX1, h->stream));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_set_velocity_levels(mlvs_handle* h, int n_base, double umin, double umax,
                                                int quadrature, int n_levels, const mlvs_level_desc* levels,
                                                int adaptive) {
  if (!h) return MLVS_ERR_ARG;
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (h->ready) return fail(h, MLVS_ERR_STATE, "velocity levels are already set");
  if (n_levels < 1 || !levels) return fail(h, MLVS_ERR_ARG, "need at least one level");
  if (!(umax > umin)) return fail(h, MLVS_ERR_ARG, "umax must exceed umin");
  if (adaptive != 0 && adaptive != 1) return fail(h, MLVS_ERR_ARG, "adaptive must be 0 or 1");
  if (h->cfg.compat_moments == 8 && (n_levels != 1 || adaptive != 0))
    return fail(h, MLVS_ERR_ARG, "the eight-moment correction runs on one level (adaptive = 0)");
  h->adaptive = adaptive;
  try {
    h->base = make_base_1d(n_base, umin, umax, quadrature);
  } catch (const std::exception& e) {
    return fail(h, MLVS_ERR_ARG, e.what());
  }
  h->n_base = n_base;
  const int D = h->D;
  const int N1 = (int)groups_1d(n_base, 1).size();
  const int nb = D == 2 ? N1 * N1 : N1;
  if (D == 2) {
    mlvs_status st = build_criterion_tables(h, n_base);
    if (st != MLVS_OK) return st;
  }
  h->n_levels = n_levels;
  h->level_space.assign(n_levels, 0);
  // time step (reading of CFL = 0.5): dt = cfl * min(dx, dy) / max |xi|_inf on the base grid
  const double vmax = std::max(std::fabs(umin), std::fabs(umax));
  const double hmin = h->curvi ? h->lmin : (D == 2 ? std::min(h->dx, h->dy) : h->dx);
  h->dt = h->cfg.dt > 0 ? h->cfg.dt : h->cfg.cfl * hmin / vmax;
  if (h->curvi) {
    mlvs_status gs = upload_geometry(h);
    if (gs != MLVS_OK) return gs;
  }
  for (int l = 0; l < n_levels; ++l) {
    std::vector<int> kap(nb);
    if (levels[l].uniform_L >= 0) {
      if (levels[l].uniform_L > 3) return fail(h, MLVS_ERR_ARG, "uniform_L must be in 0..3");
      std::fill(kap.begin(), kap.end(), levels[l].uniform_L);
    } else {
      if (!levels[l].kappa) return fail(h, MLVS_ERR_ARG, "kappa is null");
      for (int b = 0; b < nb; ++b) {
        if (levels[l].kappa[b] > 3) return fail(h, MLVS_ERR_ARG, "kappa values must be in 0..3");
        kap[b] = levels[l].kappa[b];
      }
    }
    mlvs_status st = get_space(h, kap, &h->level_space[l]);
    if (st != MLVS_OK) return st;
    const SpaceRt& sp = h->spaces[h->level_space[l]];
    if (h->cfg.compat_moments == 8 && sp.nax == 0 && !sp.rows.p)
      return fail(h, MLVS_ERR_ARG, "the eight-moment correction needs a tensor-product space or one made of level groups");
  }
  Ops ops = ops_for(h->cfg.storage, D);
  const int ncell = h->nx * h->ny;
  h->inst.clear();
  h->inst.resize(h->cfg.n_instances);
  for (int i = 0; i < h->cfg.n_instances; ++i) {
    Inst& I = h->inst[i];
    mlvs_status st = build_levels(h, std::vector<int>(ncell, 0), I);
    if (st != MLVS_OK) return st;
    if (I.ucell.alloc(2ull * ncell * h->tsize) != cudaSuccess || I.W.alloc(11ull * ncell * 8) != cudaSuccess ||
        I.err.alloc(ERR_WORDS * sizeof(int)) != cudaSuccess || I.stepctr.alloc(sizeof(unsigned)) != cudaSuccess)
      return fail(h, MLVS_ERR_OOM, "device allocation failed");
    CK(cudaMemsetAsync(I.err.p, 0, ERR_WORDS * sizeof(int), h->stream));
    CK(cudaMemsetAsync(I.stepctr.p, 0, sizeof(unsigned), h->stream));
    CK(cudaMemsetAsync(I.W.p, 0, I.W.n, h->stream));
    CK(ops.tile_batch(h, I));   // the instance in place, every buffer allocated
    DevBuf dW0;
    CK(upload(dW0, std::vector<double>(h->initW.begin() + 4ull * ncell * i, h->initW.begin() + 4ull * ncell * (i + 1)),
              h->stream));
    CK(ops.init_state(h, I, dW0.as<double>()));
    CK(cudaStreamSynchronize(h->stream));
    int eflag = 0;
    CK(cudaMemcpy(&eflag, I.err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (eflag & ERR_SINGULAR) return fail(h, MLVS_ERR_SINGULAR, "singular compatibility matrix at init");
  }
  h->ready = true;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_set_cell_levels(mlvs_handle* h, int instance, const int* levels) {
  if (!h || !levels) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  const int ncell = h->nx * h->ny;
  std::vector<int> lv(levels, levels + ncell);
  for (int x : lv)
    if (x < 0 || x >= h->n_levels) return fail(h, MLVS_ERR_ARG, "cell level out of range");
  Ops ops = ops_for(h->cfg.storage, h->D);
  Inst& Old = h->inst[instance];
  // the moments of the current state (for the shifts) and its parameters
  for (int l = 0; l < h->n_levels; ++l)
    if (!Old.lv[l].fresh) CK(ops.finalize_cells(h, Old, Old.lv[l]));
  Inst New;
  mlvs_status st = build_levels(h, lv, New);
  if (st != MLVS_OK) return st;
  New.ucell = std::move(Old.ucell);
  New.W = std::move(Old.W);
  New.err = std::move(Old.err);
  New.stepctr = std::move(Old.stepctr);
  CK(ops.transfer(h, Old, New));
  CK(ops.moments_of_levels(h, New));
  CK(cudaStreamSynchronize(h->stream));
  h->inst[instance] = std::move(New);
  CK(ops.tile_batch(h, h->inst[instance]));   // the instance in place, every buffer allocated
  return check_flags(h);
}

static mlvs_status check_adapt_params(mlvs_handle* h, const mlvs_adapt_params* p) {
  if (!p) return fail(h, MLVS_ERR_ARG, "null adaptation parameters");
  if (h->D != 2) return fail(h, MLVS_ERR_ARG, "the criterion is implemented for 2-D velocity spaces");
  if (!(p->C_merge >= 0) || !(p->C_split >= p->C_merge)) return fail(h, MLVS_ERR_ARG, "need 0 <= C_merge <= C_split");
  if (p->max_level < 1 || p->max_level > 3) return fail(h, MLVS_ERR_ARG, "max_level must be 1, 2 or 3");
  if (!(p->tau_clust >= 0)) return fail(h, MLVS_ERR_ARG, "tau_clust must be >= 0");
  return MLVS_OK;
}

static mlvs_status ensure_kbuf(mlvs_handle* h, size_t bytes) {
  if (h->kbuf.n >= bytes) return MLVS_OK;
  if (h->kbuf.alloc(bytes) != cudaSuccess) return fail(h, MLVS_ERR_OOM, "device allocation of the masks failed");
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_criterion(mlvs_handle* h, int instance, const mlvs_adapt_params* p,
                                      unsigned char* kappa_out, int out_on_device) {
  if (!h || !kappa_out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  mlvs_status st = check_adapt_params(h, p);
  if (st != MLVS_OK) return st;
  const size_t bytes = (size_t)h->nx * h->ny * h->N1 * h->N1;
  unsigned char* dst = kappa_out;
  if (!out_on_device) {
    if ((st = ensure_kbuf(h, bytes)) != MLVS_OK) return st;
    dst = h->kbuf.as<unsigned char>();
  }
  Ops ops = ops_for(h->cfg.storage, h->D);
  CK(ops.criterion(h, h->inst[instance], *p, dst, nullptr));
  if (!out_on_device) CK(cudaMemcpyAsync(kappa_out, dst, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MLVS_OK;
}

// Criterion on every cell, grouping, one level per distinct representative space, remap.
using Clock = std::chrono::steady_clock;
static float ms_between(Clock::time_point x, Clock::time_point y) {
  return (float)std::chrono::duration<double, std::milli>(y - x).count();
}

// Criterion masks of the selected cells of every instance (sel: per instance the cells, or
// empty for all), downloaded to the pinned host buffer [instance][cell][N1*N1].
static mlvs_status compute_masks(mlvs_handle* h, const mlvs_adapt_params& p,
                                 const std::vector<std::vector<int>>* sel, float* ms_crit) {
  const int ncell = h->nx * h->ny, nb = h->N1 * h->N1, ninst = h->cfg.n_instances;
  const size_t per = (size_t)ncell * nb;
  mlvs_status st = ensure_kbuf(h, per * ninst);
  if (st != MLVS_OK) return st;
  if (!h->ea0) {
    CK(cudaEventCreate(&h->ea0));
    CK(cudaEventCreate(&h->ea1));
  }
  Ops ops = ops_for(h->cfg.storage, h->D);
  CK(cudaEventRecord(h->ea0, h->stream));
  for (int i = 0; i < ninst; ++i)
    CK(ops.criterion(h, h->inst[i], p, h->kbuf.as<unsigned char>() + per * i, sel ? &(*sel)[i] : nullptr));
  CK(cudaEventRecord(h->ea1, h->stream));
  if (h->kbuf_host_n < per * ninst) {
    if (h->kbuf_host) cudaFreeHost(h->kbuf_host);
    h->kbuf_host = nullptr;
    h->kbuf_host_n = 0;
    CK(cudaMallocHost(&h->kbuf_host, per * ninst));
    h->kbuf_host_n = per * ninst;
  }
  CK(cudaMemcpyAsync(h->kbuf_host, h->kbuf.p, per * ninst, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaEventElapsedTime(ms_crit, h->ea0, h->ea1));
  return MLVS_OK;
}

// Fixed level set: the coarsest level (fewest velocities) whose space encloses the mask
// (keff <= kappa on every block); the finest level when none does.
static int fixed_set_level(const mlvs_handle* h, const unsigned char* k) {
  const int nb = h->N1 * h->N1;
  int pick = -1, pick_nv = 0, finest = 0, finest_nv = -1;
  for (int l = 0; l < h->n_levels; ++l) {
    const SpaceRt& sp = h->spaces[h->level_space[l]];
    const int nv = sp.vs.nv();
    if (nv > finest_nv) { finest = l; finest_nv = nv; }
    if (pick >= 0 && nv >= pick_nv) continue;
    bool ok = true;
    for (int b = 0; b < nb && ok; ++b) ok = sp.keff[b] <= k[b];
    if (ok) { pick = l; pick_nv = nv; }
  }
  return pick >= 0 ? pick : finest;
}

// Move every cell to cell_level (per instance, per cell) on the level set new_space.
static mlvs_status apply_levels(mlvs_handle* h, const std::vector<int>& new_space, const std::vector<int>& cell_level,
                                mlvs_adapt_stats* stats) {
  const int ncell = h->nx * h->ny, ninst = h->cfg.n_instances;
  Ops ops = ops_for(h->cfg.storage, h->D);
  bool same = new_space == h->level_space;
  for (int i = 0; i < ninst && same; ++i)
    for (int c = 0; c < ncell && same; ++c) same = cell_level[(size_t)i * ncell + c] == h->inst[i].lvl_of[c];
  int changed = 0;
  h->exp_corrected = h->exp_failed = 0;
  h->map9_singular = 0;
  if (!same) {
    // the current state's moments and parameters (for the shifts), then the new level set
    for (auto& I : h->inst)
      for (int l = 0; l < h->n_levels; ++l)
        if (!I.lv[l].fresh) CK(ops.finalize_cells(h, I, I.lv[l]));
    const std::vector<int> old_space = h->level_space;
    h->n_levels = (int)new_space.size();
    h->level_space = new_space;
    for (int i = 0; i < ninst; ++i) {
      Inst& Old = h->inst[i];
      std::vector<int> lv(ncell);
      for (int c = 0; c < ncell; ++c) {
        lv[c] = cell_level[(size_t)i * ncell + c];
        if (h->level_space[lv[c]] != old_space[Old.lvl_of[c]]) ++changed;
      }
      Inst New;
      mlvs_status st = build_levels(h, lv, New);
      if (st != MLVS_OK) { h->sticky = st; return st; }
      New.ucell = std::move(Old.ucell);
      New.W = std::move(Old.W);
      New.err = std::move(Old.err);
      New.stepctr = std::move(Old.stepctr);
      cudaError_t e = ops.transfer(h, Old, New);
      if (e == cudaSuccess) e = ops.moments_of_levels(h, New);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        h->sticky = MLVS_ERR_CUDA;
        return fail(h, MLVS_ERR_CUDA, std::string("adaptation remap: ") + cudaGetErrorString(e));
      }
      if (h->map9_singular) {
        h->sticky = MLVS_ERR_SINGULAR;
        return fail(h, MLVS_ERR_SINGULAR, "nine-moment level switch: singular correction block");
      }
      h->inst[i] = std::move(New);
      if ((e = ops.tile_batch(h, h->inst[i])) != cudaSuccess) {   // the instance in place
        h->sticky = MLVS_ERR_CUDA;
        return fail(h, MLVS_ERR_CUDA, std::string("tile tables: ") + cudaGetErrorString(e));
      }
    }
  }
  if (stats) {
    long long upd = 0;
    for (auto& I : h->inst)
      for (int l = 0; l < h->n_levels; ++l) upd += (long long)I.lv[l].cells.size() * I.lv[l].k.nv;
    stats->n_levels = h->n_levels;
    stats->n_changed = changed;
    stats->updates_per_step = upd;
    stats->n_exp_corrected = h->exp_corrected;
    stats->n_exp_failed = h->exp_failed;
    stats->n_interior_faces = 0;
    stats->n_cross_faces = 0;
    for (auto& I : h->inst) {
      stats->n_interior_faces += I.n_int;
      stats->n_cross_faces += I.n_cross;
    }
  }
  return same ? MLVS_OK : check_flags(h);
}

// Criterion on every cell, then grouping (adaptive = 1) or the fixed-set rule, then remap.
static mlvs_status adapt_impl(mlvs_handle* h, const mlvs_adapt_params& p, mlvs_adapt_stats* stats) {
  const auto t0 = Clock::now();
  const int ncell = h->nx * h->ny, nb = h->N1 * h->N1, ninst = h->cfg.n_instances;
  float ms_crit = 0.f;
  mlvs_status st = compute_masks(h, p, nullptr, &ms_crit);
  if (st != MLVS_OK) return st;
  const unsigned char* kap = h->kbuf_host;
  const auto t1 = Clock::now();
  std::vector<int> cell_level((size_t)ncell * ninst), new_space;
  int n_distinct = 0;
  if (h->adaptive) {
    Clustering C = cluster_masks(kap, (long)ncell * ninst, nb, p.tau_clust);
    n_distinct = C.n_distinct;
    // one level per distinct (consistent) representative space
    std::vector<int> lev_of_cluster(C.reps.size());
    std::map<int, int> level_of_space;
    for (size_t c = 0; c < C.reps.size(); ++c) {
      int sp;
      st = get_space(h, std::vector<int>(C.reps[c].begin(), C.reps[c].end()), &sp);
      if (st != MLVS_OK) return st;
      auto it = level_of_space.find(sp);
      if (it == level_of_space.end()) {
        it = level_of_space.emplace(sp, (int)new_space.size()).first;
        new_space.push_back(sp);
      }
      lev_of_cluster[c] = it->second;
    }
    for (size_t r = 0; r < cell_level.size(); ++r) cell_level[r] = lev_of_cluster[C.labels[r]];
  } else {
    new_space = h->level_space;
    for (size_t r = 0; r < cell_level.size(); ++r) cell_level[r] = fixed_set_level(h, kap + r * nb);
  }
  const auto t2 = Clock::now();
  st = apply_levels(h, new_space, cell_level, stats);
  if (st != MLVS_OK) return st;
  if (stats) {
    stats->n_distinct = n_distinct;
    stats->ms_criterion = ms_crit;
    stats->ms_group = ms_between(t1, t2);
    stats->ms_remap = ms_between(t2, Clock::now());
    stats->ms_total = ms_between(t0, Clock::now());
  }
  return MLVS_OK;
}

// Fresh cell moments of an instance (W), as mlvs_moments reads them.
static mlvs_status fresh_moments(mlvs_handle* h, Inst& I) {
  Ops ops = ops_for(h->cfg.storage, h->D);
  for (int l = 0; l < h->n_levels; ++l)
    if (!I.lv[l].fresh) CK(ops.finalize_cells(h, I, I.lv[l]));
  return check_flags(h);
}

static mlvs_status features_into(mlvs_handle* h, Inst& I, float* dst) {
  mlvs_status st = fresh_moments(h, I);
  if (st != MLVS_OK) return st;
  FeatArgs a;
  a.W = I.W.as<double>();
  a.geo = h->curvi ? h->featgeo_d.as<double>() : nullptr;
  a.nx = h->nx;
  a.ny = h->ny;
  a.px = h->cfg.bc[0] == MLVS_BC_PERIODIC;
  a.py = h->D == 2 ? (h->cfg.bc[2] == MLVS_BC_PERIODIC) : 1;
  a.dx = h->dx;
  a.dy = h->dy;
  a.R = h->gas.R;
  a.T_ref = h->gas.T_ref;
  a.mu_ref = h->gas.mu_ref;
  a.omega = h->gas.omega;
  a.L_ref = h->cfg.L_ref > 0 ? h->cfg.L_ref : 1.0;
  a.out = dst;
  const int nc = h->nx * h->ny;
  k_features<<<(nc + 127) / 128, 128, 0, h->stream>>>(a);
  CK(cudaGetLastError());
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_features(mlvs_handle* h, int instance, float* out, int out_on_device) {
  if (!h || !out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  const size_t bytes = (size_t)h->nx * h->ny * 10 * sizeof(float);
  float* dst = out;
  if (!out_on_device) {
    if (h->feat_d.n < bytes && h->feat_d.alloc(bytes) != cudaSuccess) return fail(h, MLVS_ERR_OOM, "features");
    dst = h->feat_d.as<float>();
  }
  mlvs_status st = features_into(h, h->inst[instance], dst);
  if (st != MLVS_OK) return st;
  if (!out_on_device) CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_criterion_levels(mlvs_handle* h, int instance, const mlvs_adapt_params* p, int* levels) {
  if (!h || !levels) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  mlvs_status st = check_adapt_params(h, p);
  if (st != MLVS_OK) return st;
  const int ncell = h->nx * h->ny, nb = h->N1 * h->N1;
  std::vector<std::vector<int>> sel(h->cfg.n_instances);   // only this instance's cells
  for (int c = 0; c < ncell; ++c) sel[instance].push_back(c);
  float ms = 0.f;
  if ((st = compute_masks(h, *p, &sel, &ms)) != MLVS_OK) return st;
  const unsigned char* kap = h->kbuf_host + (size_t)instance * ncell * nb;
  for (int c = 0; c < ncell; ++c) levels[c] = fixed_set_level(h, kap + (size_t)c * nb);
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_adapt_mlp(mlvs_handle* h, mlvs_mlp* m, const mlvs_adapt_params* p, float confidence,
                                      mlvs_adapt_stats* stats) {
  if (!h || !m) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (h->adaptive || h->n_levels != 4) return fail(h, MLVS_ERR_ARG, "the selector needs a fixed set of four levels");
  if (!(confidence >= 0.f && confidence <= 1.f)) return fail(h, MLVS_ERR_ARG, "confidence outside [0, 1]");
  mlvs_status st = check_adapt_params(h, p);
  if (st != MLVS_OK) return st;
  const auto t0 = Clock::now();
  const int ncell = h->nx * h->ny, nb = h->N1 * h->N1, ninst = h->cfg.n_instances;
  const size_t fbytes = (size_t)ncell * 10 * sizeof(float), pbytes = (size_t)ncell * 4 * sizeof(float);
  if ((h->feat_d.n < fbytes && h->feat_d.alloc(fbytes) != cudaSuccess) ||
      (h->prob_d.n < pbytes && h->prob_d.alloc(pbytes) != cudaSuccess))
    return fail(h, MLVS_ERR_OOM, "selector buffers");
  // predictions, instance by instance
  std::vector<int> cell_level((size_t)ncell * ninst);
  std::vector<std::vector<int>> fall(ninst);
  std::vector<float> prob((size_t)ncell * 4);
  int nfall = 0;
  for (int i = 0; i < ninst; ++i) {
    if ((st = features_into(h, h->inst[i], h->feat_d.as<float>())) != MLVS_OK) return st;
    CK(cudaStreamSynchronize(h->stream));
    if ((st = mlvs_mlp_forward(m, h->feat_d.as<float>(), ncell, nullptr, h->prob_d.as<float>())) != MLVS_OK)
      return fail(h, st, "selector forward pass failed");
    CK(cudaDeviceSynchronize());   // the network orders its work on its own stream
    CK(cudaMemcpy(prob.data(), h->prob_d.p, pbytes, cudaMemcpyDeviceToHost));
    for (int c = 0; c < ncell; ++c) {
      const float* q = prob.data() + (size_t)c * 4;
      int k = 0;
      for (int j = 1; j < 4; ++j)
        if (q[j] > q[k]) k = j;
      if (q[k] >= confidence) cell_level[(size_t)i * ncell + c] = k;
      else { fall[i].push_back(c); ++nfall; }
    }
  }
  const auto t1 = Clock::now();
  float ms_crit = 0.f;
  if (nfall > 0) {
    if ((st = compute_masks(h, *p, &fall, &ms_crit)) != MLVS_OK) return st;
    for (int i = 0; i < ninst; ++i)
      for (int c : fall[i])
        cell_level[(size_t)i * ncell + c] = fixed_set_level(h, h->kbuf_host + ((size_t)i * ncell + c) * nb);
  }
  const auto t2 = Clock::now();
  if ((st = apply_levels(h, h->level_space, cell_level, stats)) != MLVS_OK) return st;
  if (stats) {
    stats->n_distinct = nfall;
    stats->ms_criterion = ms_crit;
    stats->ms_group = ms_between(t0, t1);
    stats->ms_remap = ms_between(t2, Clock::now());
    stats->ms_total = ms_between(t0, Clock::now());
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_adapt(mlvs_handle* h, const mlvs_adapt_params* p, mlvs_adapt_stats* stats) {
  if (!h) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  mlvs_status st = check_adapt_params(h, p);
  if (st != MLVS_OK) return st;
  return adapt_impl(h, *p, stats);
}

extern "C" mlvs_status mlvs_set_adaptation(mlvs_handle* h, const mlvs_adapt_params* p, int interval) {
  if (!h) return MLVS_ERR_ARG;
  if (interval < 0) return fail(h, MLVS_ERR_ARG, "interval < 0");
  if (interval > 0) {
    mlvs_status st = check_adapt_params(h, p);
    if (st != MLVS_OK) return st;
    h->adapt = *p;
  }
  h->adapt_interval = interval;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_cluster(const unsigned char* kappa, long nrow, int nb, double tau, int* labels,
                                    unsigned char* reps, int reps_cap, int* n_reps) {
  if (!kappa || !labels || !reps || !n_reps || nb < 1 || nrow < 0 || !(tau >= 0))
    return fail(nullptr, MLVS_ERR_ARG, "mlvs_cluster: bad argument");
  Clustering C = cluster_masks(kappa, nrow, nb, tau);
  *n_reps = (int)C.reps.size();
  if ((int)C.reps.size() > reps_cap) return fail(nullptr, MLVS_ERR_ARG, "mlvs_cluster: reps_cap too small");
  for (long r = 0; r < nrow; ++r) labels[r] = C.labels[r];
  for (size_t c = 0; c < C.reps.size(); ++c) std::memcpy(reps + c * nb, C.reps[c].data(), nb);
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_umesh_geometry(int n_node, const double* node_xy, int n_cell, const int* cell_ptr,
                                           const int* cell_nodes, int face_cap, int* n_face,
                                           double* cell_geo, int* cell_face, int* face_cells,
                                           int* face_nodes, double* face_geo) {
  if (!node_xy || !cell_ptr || !cell_nodes || !n_face || n_node < 3 || n_cell < 1)
    return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_geometry: bad argument");
  UMeshGeo g;
  const std::string why = build_umesh(n_node, node_xy, n_cell, cell_ptr, cell_nodes, g);
  if (!why.empty()) return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_geometry: " + why);
  const int nf = (int)g.fL.size();
  *n_face = nf;
  if (!cell_geo && !cell_face && !face_cells && !face_nodes && !face_geo) return MLVS_OK;
  if (!cell_geo || !cell_face || !face_cells || !face_nodes || !face_geo)
    return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_geometry: outputs must be all given or all NULL");
  if (face_cap < nf) return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_geometry: face_cap too small");
  const size_t nc = n_cell;
  const std::vector<double>* crow[7] = {&g.area, &g.cx, &g.cy, &g.width, &g.mxx, &g.mxy, &g.myy};
  for (int r = 0; r < 7; ++r) std::memcpy(cell_geo + r * nc, crow[r]->data(), nc * sizeof(double));
  std::memcpy(cell_face, g.cf.data(), g.cf.size() * sizeof(int));
  std::memcpy(face_cells, g.fL.data(), nf * sizeof(int));
  std::memcpy(face_cells + nf, g.fR.data(), nf * sizeof(int));
  std::memcpy(face_nodes, g.fn0.data(), nf * sizeof(int));
  std::memcpy(face_nodes + nf, g.fn1.data(), nf * sizeof(int));
  const std::vector<double>* frow[5] = {&g.nx, &g.ny, &g.len, &g.midx, &g.midy};
  for (int r = 0; r < 5; ++r) std::memcpy(face_geo + (size_t)r * nf, frow[r]->data(), nf * sizeof(double));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_umesh_order(int n_cell, const double* cx, const double* cy, int* order) {
  if (!cx || !cy || !order || n_cell < 1) return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_order: bad argument");
  for (int i = 0; i < n_cell; ++i)
    if (!std::isfinite(cx[i]) || !std::isfinite(cy[i]))
      return fail(nullptr, MLVS_ERR_ARG, "mlvs_umesh_order: non-finite centroid");
  hilbert_order(n_cell, cx, cy, order);
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_space_points(int n_base, double umin, double umax, int quadrature,
                                         const unsigned char* kappa, int nkappa, double* xi_x, double* xi_y,
                                         double* w, int cap, int* nv_out, int* n1_out) {
  if (!nv_out || !(umax > umin)) return fail(nullptr, MLVS_ERR_ARG, "mlvs_space_points: bad argument");
  try {
    const Base1D b = make_base_1d(n_base, umin, umax, quadrature);
    const int N1 = (int)groups_1d(n_base, 1).size();
    if (n1_out) *n1_out = N1;
    *nv_out = 0;
    if (!kappa) return MLVS_OK;
    if (nkappa != N1 * N1) return fail(nullptr, MLVS_ERR_ARG, "mlvs_space_points: nkappa != n1 * n1");
    std::vector<int> k(kappa, kappa + nkappa);
    for (int x : k)
      if (x < 0 || x > 3) return fail(nullptr, MLVS_ERR_ARG, "mlvs_space_points: kappa above 3");
    const std::vector<int> keff = enforce_consistency(k, n_base, 2);
    std::vector<int> owner;
    const VSpace vs = kappa_vspace(b, 2, keff, owner);
    *nv_out = vs.nv();
    if (!xi_x && !xi_y && !w) return MLVS_OK;
    if (!xi_x || !xi_y || !w || cap < vs.nv())
      return fail(nullptr, MLVS_ERR_ARG, "mlvs_space_points: outputs missing or cap too small");
    for (int i = 0; i < vs.nv(); ++i) {
      xi_x[i] = vs.xix[i];
      xi_y[i] = vs.xiy[i];
      w[i] = vs.w[i];
    }
  } catch (const std::exception& e) {
    return fail(nullptr, MLVS_ERR_ARG, std::string("mlvs_space_points: ") + e.what());
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_level_kappa(const mlvs_handle* h, int level, unsigned char* out, int cap,
                                        int* nb_out) {
  if (!h || !nb_out) return MLVS_ERR_ARG;
  if (!h->ready) return MLVS_ERR_STATE;
  if (level < 0 || level >= h->n_levels) return MLVS_ERR_ARG;
  const auto& k = h->spaces[h->level_space[level]].keff;
  *nb_out = (int)k.size();
  if (!out) return MLVS_OK;
  if (cap < (int)k.size()) return MLVS_ERR_ARG;
  for (size_t b = 0; b < k.size(); ++b) out[b] = (unsigned char)k[b];
  return MLVS_OK;
}

// ---------------------------------------------------------------------------------------
// stepping: regular launches, or two-step CUDA graphs over a group of handles

// One regular step of every instance of h on its stream, then the adaptation when due.
static mlvs_status regular_step(mlvs_handle* h) {
  Ops ops = ops_for(h->cfg.storage, h->D);
  for (auto& I : h->inst) CK(ops.step(h, I));
  ++h->steps_done;
  h->warm_epoch = h->epoch;
  if (h->adapt_interval > 0 && h->steps_done % h->adapt_interval == 0) {
    mlvs_status st = adapt_impl(h, h->adapt, nullptr);
    if (st != MLVS_OK) return st;
  }
  return MLVS_OK;
}

// A graph can replay the next two steps of h: its tables exist, no cell level holds finished
// parameters from a moments call, and no adaptation falls inside the two steps.
static bool graph_ready(const mlvs_handle* h) {
  if (h->warm_epoch != h->epoch) return false;
  if (h->adapt_interval > 0 &&
      ((h->steps_done + 1) % h->adapt_interval == 0 || (h->steps_done + 2) % h->adapt_interval == 0))
    return false;
  for (auto& I : h->inst)
    for (int l = 0; l < h->n_levels; ++l)
      if (I.lv[l].fresh) return false;
  return true;
}

// Key of the two-step graph of a group: handle ids, structure epochs and the ping-pong parity
// of every level (after two steps every parity is back where it started).
static std::vector<long long> graph_key(mlvs_handle* const* hs, int nh) {
  std::vector<long long> key;
  for (int j = 0; j < nh; ++j) {
    key.push_back((long long)hs[j]->uid);
    key.push_back(hs[j]->epoch);
    for (auto& I : hs[j]->inst)
      for (int l = 0; l < hs[j]->n_levels; ++l) key.push_back(I.lv[l].cur | (I.lv[l].pcur << 1));
  }
  return key;
}

static cudaError_t ensure_capture_resources(mlvs_handle* h0, int nbranch, int nh) {
  cudaError_t e;
  if (!h0->cap && (e = cudaStreamCreateWithFlags(&h0->cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if (!h0->ev_fork && (e = cudaEventCreateWithFlags(&h0->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  if (!h0->ev_post && (e = cudaEventCreateWithFlags(&h0->ev_post, cudaEventDisableTiming)) != cudaSuccess) return e;
  while ((int)h0->branch.size() < nbranch) {
    cudaStream_t s;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    h0->branch.push_back(s);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    h0->bev.push_back(ev);
  }
  while ((int)h0->ev_pre.size() < nh) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    h0->ev_pre.push_back(ev);
  }
  return cudaSuccess;
}

// Two steps of every handle of the group as one graph launch on hs[0]'s stream.  The graph
// forks one branch per instance (instances and handles are independent), so their kernels
// may run concurrently.  Captured on first use for a key, replayed afterwards.
// A group of several handles whose tile passes can share one launch: the same storage,
// dimension, mesh kind and limiter, and no eight-moment correction (its kernels take one level).
static bool group_batchable(mlvs_handle* const* hs, int nh) {
  if (nh < 2) return false;
  for (int j = 0; j < nh; ++j) {
    const mlvs_handle* h = hs[j];
    if (h->cfg.storage != hs[0]->cfg.storage || h->D != hs[0]->D || h->curvi != hs[0]->curvi ||
        h->cfg.limiter != hs[0]->cfg.limiter || h->cfg.compat_moments == 8)
      return false;
  }
  return true;
}

static mlvs_status graph_two_steps(mlvs_handle* const* hs, int nh) {
  mlvs_handle* h0 = hs[0];
  std::vector<long long> key = graph_key(hs, nh);
  auto it = h0->graphs.find(key);
  if (it == h0->graphs.end() && group_batchable(hs, nh)) {
    int nbranch = 0;
    for (int j = 0; j < nh; ++j) nbranch += (int)hs[j]->inst.size();
    cudaError_t e = ensure_capture_resources(h0, nbranch, nh);
    if (e != cudaSuccess) return fail(h0, MLVS_ERR_CUDA, std::string("graph resources: ") + cudaGetErrorString(e));
    std::vector<int> kernels;
    cudaGraphExec_t exec = nullptr;
    mlvs_handle::GroupBufs& B = h0->gbufs[key];
    cudaError_t ce = ops_for(h0->cfg.storage, h0->D).group_capture(hs, nh, B, kernels, &exec);
    if (ce != cudaSuccess) {
      // the host state may have advanced by steps that never ran: the handles cannot continue
      for (int j = 0; j < nh; ++j) hs[j]->sticky = MLVS_ERR_CUDA;
      return fail(h0, MLVS_ERR_CUDA, std::string("group graph capture: ") + cudaGetErrorString(ce));
    }
    it = h0->graphs.emplace(key, std::make_pair(exec, kernels)).first;
  }
  if (it == h0->graphs.end()) {
    int nbranch = 0;
    for (int j = 0; j < nh; ++j) nbranch += (int)hs[j]->inst.size();
    cudaError_t e = ensure_capture_resources(h0, nbranch, nh);
    if (e != cudaSuccess) return fail(h0, MLVS_ERR_CUDA, std::string("graph resources: ") + cudaGetErrorString(e));
    std::vector<int> kernels(nh, 0);
    CK_H(h0, cudaStreamBeginCapture(h0->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaEventRecord(h0->ev_fork, h0->cap);
    int b = 0;
    for (int j = 0; j < nh && ce == cudaSuccess; ++j) {
      mlvs_handle* h = hs[j];
      Ops ops = ops_for(h->cfg.storage, h->D);
      cudaStream_t saved = h->stream;
      const int l0 = h->launches;
      for (auto& I : h->inst) {
        cudaStream_t s = h0->branch[b];
        if ((ce = cudaStreamWaitEvent(s, h0->ev_fork, 0)) != cudaSuccess) break;
        h->stream = s;
        if ((ce = ops.step(h, I)) != cudaSuccess) break;
        if ((ce = ops.step(h, I)) != cudaSuccess) break;
        if ((ce = cudaEventRecord(h0->bev[b], s)) != cudaSuccess) break;
        if ((ce = cudaStreamWaitEvent(h0->cap, h0->bev[b], 0)) != cudaSuccess) break;
        ++b;
      }
      h->stream = saved;
      kernels[j] = h->launches - l0;
      h->launches = l0;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h0->cap, &graph);
    if (ce == cudaSuccess) ce = ee;
    cudaGraphExec_t exec = nullptr;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      // the host state advanced by two steps that never ran: the handles cannot continue
      for (int j = 0; j < nh; ++j) hs[j]->sticky = MLVS_ERR_CUDA;
      return fail(h0, MLVS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    it = h0->graphs.emplace(key, std::make_pair(exec, kernels)).first;
  }
  // order the other handles' streams before and after the launch
  for (int j = 1; j < nh; ++j)
    if (hs[j]->stream != h0->stream) {
      CK_H(h0, cudaEventRecord(h0->ev_pre[j], hs[j]->stream));
      CK_H(h0, cudaStreamWaitEvent(h0->stream, h0->ev_pre[j], 0));
    }
  CK_H(h0, cudaGraphLaunch(it->second.first, h0->stream));
  bool other = false;
  for (int j = 1; j < nh; ++j) other = other || hs[j]->stream != h0->stream;
  if (other) {
    CK_H(h0, cudaEventRecord(h0->ev_post, h0->stream));
    for (int j = 1; j < nh; ++j)
      if (hs[j]->stream != h0->stream) CK_H(h0, cudaStreamWaitEvent(hs[j]->stream, h0->ev_post, 0));
  }
  for (int j = 0; j < nh; ++j) {
    hs[j]->steps_done += 2;
    hs[j]->launches += it->second.second[j];
  }
  return MLVS_OK;
}

// n_steps steps of every handle of the group (graphs where allowed).
static mlvs_status group_steps(mlvs_handle* const* hs, int nh, int n_steps, bool graphs) {
  int done = 0;
  while (done < n_steps) {
    bool g = graphs && n_steps - done >= 2;
    for (int j = 0; j < nh && g; ++j) g = graph_ready(hs[j]);
    if (g) {
      mlvs_status st = graph_two_steps(hs, nh);
      if (st != MLVS_OK) return st;
      done += 2;
      continue;
    }
    for (int j = 0; j < nh; ++j) {
      mlvs_status st = regular_step(hs[j]);
      if (st != MLVS_OK) return st;
    }
    done += 1;
  }
  return MLVS_OK;
}

static void fill_stats(mlvs_handle* const* hs, int nh, int n_steps, float ms, mlvs_step_stats* stats) {
  stats->ms_total = ms;
  stats->dt = hs[0]->dt;
  long long upd = 0;
  int launches = 0;
  for (int j = 0; j < nh; ++j) {
    for (auto& I : hs[j]->inst)
      for (int l = 0; l < hs[j]->n_levels; ++l) upd += (long long)I.lv[l].cells.size() * I.lv[l].k.nv;
    launches += hs[j]->launches;
  }
  stats->cell_velocity_updates = upd * n_steps;
  stats->n_levels = hs[0]->n_levels;
  stats->launches = launches;
}

extern "C" mlvs_status mlvs_step(mlvs_handle* h, int n_steps, mlvs_step_stats* stats) {
  if (!h) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (n_steps < 0) return fail(h, MLVS_ERR_ARG, "n_steps < 0");
  h->profiling = stats && stats->profile;
  h->prof.marks.clear();
  h->prof.used = 0;
  h->launches = 0;
  CK(cudaEventRecord(h->ev0, h->stream));
  mlvs_status st = group_steps(&h, 1, n_steps, h->use_graph && !h->profiling);
  if (st != MLVS_OK) { h->profiling = false; return st; }
  CK(cudaEventRecord(h->ev1, h->stream));
  mlvs_status s = check_flags(h);
  if (s != MLVS_OK) return s;
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    fill_stats(&h, 1, n_steps, ms, stats);
    for (int p = 0; p < 6; ++p) stats->ms_phase[p] = 0.f;
    if (h->profiling) {
      for (auto& m : h->prof.marks) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, h->prof.pool[m.second], h->prof.pool[m.second + 1]));
        stats->ms_phase[m.first] += t;
      }
    }
  }
  h->profiling = false;
  return MLVS_OK;
}

// Re-chunk the velocities of every level for the handle's CTA target, and recompute the cell
// partials of the current state with the new chunks (the next finalisation sums them).
static mlvs_status rechunk(mlvs_handle* h) {
  Ops ops = ops_for(h->cfg.storage, h->D);
  for (auto& I : h->inst) {
    for (int l = 0; l < h->n_levels; ++l)
      if (!I.lv[l].fresh) CK(ops.finalize_cells(h, I, I.lv[l]));
    int all_tiles = 0;
    for (auto& L : I.lv) all_tiles += L.ntiles;
    for (auto& L : I.lv) {
      StepConst& k = L.k;
      k.vpc = choose_vpc(all_tiles, k.nv, h->cta_target);
      k.nchunk = (k.nv + k.vpc - 1) / k.vpc;
      const size_t nc = std::max<size_t>(L.cells.size(), 1);
      if (L.cpart.alloc((size_t)k.nchunk * NMOM * nc * 8) != cudaSuccess ||
          L.fpart.alloc((size_t)k.nchunk * NMOM * k.nface * 8) != cudaSuccess)
        return fail(h, MLVS_ERR_OOM, "device allocation of partial sums failed");
    }
    CK(ops.tile_batch(h, I));
    CK(ops.moments_of_levels(h, I));
  }
  CK(cudaStreamSynchronize(h->stream));
  ++h->epoch;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_autotune(mlvs_handle* h, int steps, int* cta_target, float* ms_table) {
  if (!h || steps < 1) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  // CTAs per tile launch: multiples of the 148 SMs (two tile CTAs fit an SM)
  const int cand[7] = {148, 296, 444, 592, 888, 1184, 1776};
  int best = h->cta_target;
  float best_ms = 1e30f;
  h->profiling = false;
  for (int ci = 0; ci < 7; ++ci) {
    h->cta_target = cand[ci];
    mlvs_status st = rechunk(h);
    if (st == MLVS_OK) st = group_steps(&h, 1, 1, false);   // warm: maps, tables
    if (st != MLVS_OK) return st;
    CK(cudaEventRecord(h->ev0, h->stream));
    if ((st = group_steps(&h, 1, steps, h->use_graph)) != MLVS_OK) return st;
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (ms_table) ms_table[ci] = ms / steps;
    if (ms < best_ms) { best_ms = ms; best = cand[ci]; }
  }
  h->cta_target = best;
  mlvs_status st = rechunk(h);
  if (st != MLVS_OK) return st;
  if (cta_target) *cta_target = best;
  return check_flags(h);
}

extern "C" mlvs_status mlvs_set_tuning(mlvs_handle* h, int cta_target) {
  if (!h || cta_target < 1) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  h->cta_target = cta_target;
  return rechunk(h);
}

extern "C" mlvs_status mlvs_set_graph(mlvs_handle* h, int on) {
  if (!h) return MLVS_ERR_ARG;
  h->use_graph = on != 0;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_step_many(mlvs_handle* const* hs, int nh, int n_steps, int use_graph,
                                      mlvs_step_stats* stats) {
  if (!hs || nh < 1 || n_steps < 0) return fail(nullptr, MLVS_ERR_ARG, "mlvs_step_many: bad argument");
  for (int j = 0; j < nh; ++j) {
    if (!hs[j]) return fail(nullptr, MLVS_ERR_ARG, "mlvs_step_many: null handle");
    for (int q = 0; q < j; ++q)
      if (hs[q] == hs[j]) return fail(nullptr, MLVS_ERR_ARG, "mlvs_step_many: a handle appears twice");
    if (!hs[j]->ready) return fail(hs[j], MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
    if (hs[j]->sticky != MLVS_OK) return fail(hs[j], MLVS_ERR_STATE, "handle holds an earlier error");
    hs[j]->profiling = false;
    hs[j]->launches = 0;
  }
  mlvs_handle* h0 = hs[0];
  mlvs_handle* h = h0;
  CK(cudaEventRecord(h0->ev0, h0->stream));
  mlvs_status st = group_steps(hs, nh, n_steps, use_graph != 0);
  if (st != MLVS_OK) return st;
  // the group's work ends on hs[0]'s stream
  for (int j = 1; j < nh; ++j)
    if (hs[j]->stream != h0->stream) {
      CK(cudaEventRecord(hs[j]->ev1, hs[j]->stream));
      CK(cudaStreamWaitEvent(h0->stream, hs[j]->ev1, 0));
    }
  CK(cudaEventRecord(h0->ev1, h0->stream));
  for (int j = 0; j < nh; ++j) {
    mlvs_status s = check_flags(hs[j]);
    if (s != MLVS_OK) return s;
  }
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h0->ev0, h0->ev1));
    fill_stats(hs, nh, n_steps, ms, stats);
    for (int p = 0; p < 6; ++p) stats->ms_phase[p] = 0.f;
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_moments(mlvs_handle* h, int instance, unsigned fields, double* out, int out_on_device) {
  if (!h || !out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  Ops ops = ops_for(h->cfg.storage, h->D);
  Inst& I = h->inst[instance];
  for (int l = 0; l < h->n_levels; ++l)
    if (!I.lv[l].fresh) CK(ops.finalize_cells(h, I, I.lv[l]));
  mlvs_status s = check_flags(h);
  if (s != MLVS_OK) return s;
  const size_t nc = (size_t)h->nx * h->ny;
  // field order: RHO U V T QX QY LEVEL RHOE SXX SXY SYY
  const int src[11] = {0, 1, 2, 3, 4, 5, -1, 6, 8, 9, 10};
  std::vector<double> lev(nc);
  for (size_t c = 0; c < nc; ++c) lev[c] = I.lvl_of[c];
  int j = 0;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int b = 0; b < 11; ++b) {
    if (!(fields & (1u << b))) continue;
    double* dst = out + j * nc;
    if (src[b] < 0) {
      CK(cudaMemcpyAsync(dst, lev.data(), nc * 8, out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                         h->stream));
    } else {
      CK(cudaMemcpyAsync(dst, I.W.as<double>() + src[b] * nc, nc * 8, kind, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    ++j;
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_read_cells(mlvs_handle* h, int instance, int cell0, int ncells, double* out_g,
                                       double* out_h, int cap, int* nv_out) {
  if (!h || !out_g || !out_h || !nv_out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  Inst& I = h->inst[instance];
  const int nc = h->nx * h->ny;
  if (cell0 < 0 || ncells < 1 || cell0 + ncells > nc) return fail(h, MLVS_ERR_ARG, "cell range out of bounds");
  const int l = I.lvl_of[cell0];
  for (int c = cell0; c < cell0 + ncells; ++c)
    if (I.lvl_of[c] != l) return fail(h, MLVS_ERR_ARG, "cells of the range are on different levels");
  LevelRt& L = I.lv[l];
  const int nv = L.k.nv, ns = (int)L.cells.size();
  if ((long long)cap < (long long)ncells * nv) return fail(h, MLVS_ERR_ARG, "output capacity too small");
  *nv_out = nv;
  std::vector<char> buf((size_t)2 * nv * ns * h->ssize);
  CK(cudaMemcpyAsync(buf.data(), L.f[L.cur].p, buf.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int comp = 0; comp < 2; ++comp) {
    double* dst = comp == 0 ? out_g : out_h;
    for (int c = 0; c < ncells; ++c) {
      const size_t s = I.slot_of[cell0 + c];
      for (int v = 0; v < nv; ++v) {
        const size_t o = ((size_t)comp * nv + v) * ns + s;
        double x;
        if (h->ssize == 8) x = reinterpret_cast<const double*>(buf.data())[o];
        else if (h->ssize == 4) x = reinterpret_cast<const float*>(buf.data())[o];
        else x = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(buf.data())[o]);
        dst[(size_t)c * nv + v] = x;
      }
    }
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_level_info(const mlvs_handle* h, int level, int* nv, double* xi_x, double* xi_y,
                                       double* w, int cap) {
  if (!h || !nv) return MLVS_ERR_ARG;
  if (!h->ready || level < 0 || level >= h->n_levels) return MLVS_ERR_ARG;
  const VSpace& vs = h->spaces[h->level_space[level]].vs;
  *nv = vs.nv();
  if (xi_x && xi_y && w) {
    if (cap < vs.nv()) return MLVS_ERR_ARG;
    for (int v = 0; v < vs.nv(); ++v) { xi_x[v] = vs.xix[v]; xi_y[v] = vs.xiy[v]; w[v] = vs.w[v]; }
  }
  return MLVS_OK;
}
