// C ABI of the MLVS-DUGKS library: handle, memory and the per-step launch sequence.
//
// One DUGKS step (Sec. 2.2) per level is four launches on the handle's stream:
//   1. k_finalize (cells): chunk partials of phi~ -> W, tau, q, model parameters with the
//      compatibility correction (Eqs. discrete_W, discrete_q, Sec. 3.3.1)
//   2. k_tile MODE 0: face phi-bar by the characteristic, face moment partials
//   3. k_finalize (faces): Eq. W_from_bar, Eq. recover_phi weights, wall densities
//   4. k_tile MODE 1: face phi, Eq. explicit_update, phi~^{n+1}, cell moment partials
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mlvs.h"
#include "mlvs_internal.h"
#include "dugks_tile.cuh"
#include "finalize.cuh"
#include "vspace_host.hpp"

using namespace mlvs;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t bytes) {
    if (p) { cudaFree(p); p = nullptr; }
    n = bytes;
    return cudaMalloc(&p, bytes ? bytes : 1);
  }
  template <class X> X* as() const { return reinterpret_cast<X*>(p); }
};

struct Launch {
  int tx, ty;
};

// Per level, per instance device state.
struct LevelInst {
  DevBuf f[2];      // [2][nv][ncell] storage type
  DevBuf prm[2];    // [NP][ncell] compute type
  DevBuf fprm;      // [NP][nface]
  DevBuf W;         // [8][ncell] double
  DevBuf cpart;     // [nchunk][NMOM][ncell]
  DevBuf fpart;     // [nchunk][NMOM][nface]
  DevBuf err;       // int
  int cur = 0;      // f[cur] holds the current phi~
  int pcur = 0;     // prm[pcur] are the parameters used by the current f's last update
  bool fresh = false;  // prm[pcur] already finalised from the current f
};

struct LevelData {
  VSpace vs;
  DevBuf vt;        // [4][nv] compute type
  DevBuf ax;        // [2][nax] one axis of a tensor-product space (compute type)
  int uniform_L = -1;
  StepConst k;
  std::vector<LevelInst> inst;
};

}  // namespace

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

struct mlvs_handle {
  mlvs_config cfg;
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
  std::vector<LevelData> lv;
  bool ready = false;
  int sticky = MLVS_OK;
  std::string err;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

static mlvs_status fail(mlvs_handle* h, mlvs_status s, const std::string& msg) {
  if (h) {
    h->err = msg;
  } else {
    g_create_error = msg;
  }
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, MLVS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------------------
// typed launchers

namespace {

template <class S, class T, int D> struct Runner {
  static constexpr int TX = (D == 2) ? 32 : 128;
  static constexpr int TY = (D == 2) ? 8 : 1;
  static constexpr int VB = 2;   // velocities per barrier round
  static constexpr size_t SM0 = TileSmem<T, TX, TY, D, VB, 0>::BYTES;
  static constexpr size_t SM1 = TileSmem<T, TX, TY, D, VB, 1>::BYTES;

  static cudaError_t set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(k_tile<S, T, D, TX, TY, VB, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM0);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tile<S, T, D, TX, TY, VB, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM1);
  }

  static void tiles(const StepConst& k, int& ntx, int& nty) {
    ntx = (k.nx + TX - 1) / TX;
    nty = (D == 2) ? (k.ny + TY - 1) / TY : 1;
  }

  static PointArgs pargs(mlvs_handle* h, LevelData& L, LevelInst& I, bool face) {
    PointArgs a;
    a.k = L.k;
    a.gas = h->gas;
    a.is_face = face ? 1 : 0;
    a.npt = face ? L.k.nface : L.k.ncell;
    a.part = face ? I.fpart.as<double>() : I.cpart.as<double>();
    a.vt = L.vt.p;
    a.ax = L.ax.p;
    a.compat = face ? h->cfg.compat_face : h->cfg.compat_cell;
    for (int s = 0; s < 4; ++s)
      for (int j = 0; j < 3; ++j) a.wall[s][j] = h->cfg.wall[s][j];
    a.err = I.err.as<int>();
    a.W = nullptr;
    a.cprm = nullptr;
    a.prm_out = nullptr;
    return a;
  }

  // finalisation: one thread per point
  static constexpr int FIN_BLOCK = 64;
  static int fin_grid(int npt) { return std::max(1, (npt + FIN_BLOCK - 1) / FIN_BLOCK); }

  static cudaError_t init(mlvs_handle* h, LevelData& L, LevelInst& I, const double* dW0) {
    cudaError_t es = set_smem_limits();
    if (es != cudaSuccess) return es;
    PointArgs a = pargs(h, L, I, false);
    a.compat = h->cfg.compat_cell;
    a.prm_out = I.prm[0].p;
    k_init_params<T, D><<<fin_grid(L.k.ncell), FIN_BLOCK, 0, h->stream>>>(a, dW0);
    dim3 g((L.k.ncell + 127) / 128, std::min(L.k.nv, 1024));
    k_init_f<S, T, D><<<g, 128, 0, h->stream>>>(L.k, I.prm[0].as<T>(), L.vt.as<T>(), I.f[0].as<S>());
    dim3 gm((L.k.ncell + 127) / 128, L.k.nchunk);
    k_moments<S, T, D><<<gm, 128, 0, h->stream>>>(L.k, I.prm[0].as<T>(), L.vt.as<T>(), I.f[0].as<S>(),
                                                   I.cpart.as<double>());
    I.cur = 0;
    I.pcur = 0;
    I.fresh = false;
    return cudaGetLastError();
  }

  // profiling marks around a launch of phase ph
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

  // cell finalisation into prm[pcur^1]; afterwards pcur flips and fresh = true
  static cudaError_t finalize_cells(mlvs_handle* h, LevelData& L, LevelInst& I) {
    PointArgs a = pargs(h, L, I, false);
    a.cprm = I.prm[I.pcur].p;
    a.prm_out = I.prm[I.pcur ^ 1].p;
    a.W = I.W.as<double>();
    mark_begin(h, 0);
    k_finalize<T, D><<<fin_grid(a.npt), FIN_BLOCK, 0, h->stream>>>(a);
    mark_end(h);
    I.pcur ^= 1;
    I.fresh = true;
    return cudaGetLastError();
  }

  static cudaError_t step(mlvs_handle* h, LevelData& L, LevelInst& I, int limiter) {
    cudaError_t e;
    if (!I.fresh) {
      e = finalize_cells(h, L, I);
      if (e != cudaSuccess) return e;
    }
    TileArgs t;
    t.k = L.k;
    tiles(L.k, t.ntx, t.nty);
    t.f_in = I.f[I.cur].p;
    t.f_out = I.f[I.cur ^ 1].p;
    t.cparam = I.prm[I.pcur].p;
    t.fparam = I.fprm.p;
    t.vt = L.vt.p;
    dim3 grid(t.ntx * t.nty, L.k.nchunk);
    t.part = I.fpart.as<double>();
    mark_begin(h, 1);
    k_tile<S, T, D, TX, TY, VB, 0><<<grid, TX * TY, SM0, h->stream>>>(t, limiter);
    mark_end(h);
    PointArgs a = pargs(h, L, I, true);
    a.cprm = I.prm[I.pcur].p;
    a.prm_out = I.fprm.p;
    mark_begin(h, 2);
    k_finalize<T, D><<<fin_grid(a.npt), FIN_BLOCK, 0, h->stream>>>(a);
    mark_end(h);
    t.part = I.cpart.as<double>();
    mark_begin(h, 3);
    k_tile<S, T, D, TX, TY, VB, 1><<<grid, TX * TY, SM1, h->stream>>>(t, limiter);
    mark_end(h);
    I.cur ^= 1;
    I.fresh = false;
    return cudaGetLastError();
  }

  static int tile_ctas(const StepConst& k) {
    int ntx, nty;
    tiles(k, ntx, nty);
    return ntx * nty;
  }
};

struct Ops {
  cudaError_t (*init)(mlvs_handle*, LevelData&, LevelInst&, const double*);
  cudaError_t (*finalize_cells)(mlvs_handle*, LevelData&, LevelInst&);
  cudaError_t (*step)(mlvs_handle*, LevelData&, LevelInst&, int);
  int (*tile_ctas)(const StepConst&);
};

template <class S, class T, int D> Ops make_ops() {
  return Ops{&Runner<S, T, D>::init, &Runner<S, T, D>::finalize_cells, &Runner<S, T, D>::step,
             &Runner<S, T, D>::tile_ctas};
}

Ops ops_for(int storage, int D) {
  if (storage == MLVS_F64) return D == 2 ? make_ops<double, double, 2>() : make_ops<double, double, 1>();
  if (storage == MLVS_F32) return D == 2 ? make_ops<float, float, 2>() : make_ops<float, float, 1>();
  return D == 2 ? make_ops<__nv_bfloat16, float, 2>() : make_ops<__nv_bfloat16, float, 1>();
}

double vhs_mu_ref(double Kn, double omega, double rho_ref, double R, double T_ref, double L_ref) {
  const double alpha = 1.0;
  const double c = 5.0 * (alpha + 1.0) * (alpha + 2.0) * std::sqrt(M_PI) /
                   (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
  return c * Kn * rho_ref * std::sqrt(2.0 * R * T_ref) * L_ref;
}

}  // namespace

// ---------------------------------------------------------------------------------------

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
    if (cfg->bc[s] < 0 || cfg->bc[s] > 2) return fail(nullptr, MLVS_ERR_ARG, "unknown boundary kind");
  if ((cfg->bc[0] == MLVS_BC_PERIODIC) != (cfg->bc[1] == MLVS_BC_PERIODIC) ||
      (cfg->dim == 2 && (cfg->bc[2] == MLVS_BC_PERIODIC) != (cfg->bc[3] == MLVS_BC_PERIODIC)))
    return fail(nullptr, MLVS_ERR_ARG, "periodic sides must come in pairs");
  if (cfg->storage < 0 || cfg->storage > 2) return fail(nullptr, MLVS_ERR_ARG, "unknown storage type");
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

static int choose_chunks(int tile_ctas, int nv) {
  // aim at about four CTAs per SM of the 148, with at most 384 velocities per chunk
  const int target = 148 * 4;
  int nchunk = std::max(1, (target + tile_ctas - 1) / tile_ctas);
  nchunk = std::min(nchunk, nv);
  int vpc = (nv + nchunk - 1) / nchunk;
  vpc = std::min(vpc, 384);
  return vpc;
}

extern "C" mlvs_status mlvs_set_velocity_levels(mlvs_handle* h, int n_base, double umin, double umax,
                                                int quadrature, int n_levels, const mlvs_level_desc* levels,
                                                int adaptive) {
  if (!h) return MLVS_ERR_ARG;
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (n_levels < 1 || !levels) return fail(h, MLVS_ERR_ARG, "need at least one level");
  if (!(umax > umin)) return fail(h, MLVS_ERR_ARG, "umax must exceed umin");
  if (adaptive != 0) return fail(h, MLVS_ERR_ARG, "adaptive level construction is not available in this build");
  if (n_levels != 1) return fail(h, MLVS_ERR_ARG, "this build advances a single velocity space");
  Base1D b;
  try {
    b = make_base_1d(n_base, umin, umax, quadrature);
  } catch (const std::exception& e) {
    return fail(h, MLVS_ERR_ARG, e.what());
  }
  h->lv.clear();
  h->lv.resize(n_levels);
  const int D = h->D;
  for (int l = 0; l < n_levels; ++l) {
    if (levels[l].uniform_L < 0 || levels[l].uniform_L > 3)
      return fail(h, MLVS_ERR_ARG, "uniform_L must be in 0..3 in this build");
    h->lv[l].vs = uniform_vspace(b, D, levels[l].uniform_L);
  }
  // time step (reading of CFL = 0.5): dt = cfl * min(dx, dy) / max |xi|_inf on the base grid
  const double vmax = std::max(std::fabs(umin), std::fabs(umax));
  const double hmin = D == 2 ? std::min(h->dx, h->dy) : h->dx;
  h->dt = h->cfg.dt > 0 ? h->cfg.dt : h->cfg.cfl * hmin / vmax;

  Ops ops = ops_for(h->cfg.storage, D);
  for (int l = 0; l < n_levels; ++l) {
    LevelData& L = h->lv[l];
    StepConst& k = L.k;
    k.nx = h->nx;
    k.ny = h->ny;
    k.px = h->cfg.bc[0] == MLVS_BC_PERIODIC;
    k.py = D == 2 ? (h->cfg.bc[2] == MLVS_BC_PERIODIC) : 1;
    for (int s = 0; s < 4; ++s) k.bc[s] = h->cfg.bc[s];
    if (D == 1) { k.bc[2] = k.bc[3] = MLVS_BC_PERIODIC; }
    k.nfx = k.px ? k.nx : k.nx + 1;
    k.nfy = D == 2 ? (k.py ? k.ny : k.ny + 1) : 0;
    k.ncell = k.nx * k.ny;
    k.nface = k.nfx * k.ny + (D == 2 ? k.nx * k.nfy : 0);
    k.nv = L.vs.nv();
    k.dx = h->dx;
    k.dy = h->dy;
    k.dt = h->dt;
    k.c0 = h->gas.K + 3.0 - D;
    k.twoK = 2.0 * h->gas.K;
    k.vpc = choose_chunks(ops.tile_ctas(k), k.nv);
    k.nchunk = (k.nv + k.vpc - 1) / k.vpc;
    // velocity table
    std::vector<double> vt(4 * (size_t)k.nv);
    for (int v = 0; v < k.nv; ++v) {
      vt[v] = L.vs.xix[v];
      vt[k.nv + v] = L.vs.xiy[v];
      vt[2 * k.nv + v] = L.vs.wx[v];
      vt[3 * k.nv + v] = L.vs.wy[v];
    }
    // one axis of the tensor-product space (uniform levels): coordinates and weights
    L.uniform_L = levels[l].uniform_L;
    std::vector<double> axd;
    {
      auto gr = groups_1d(n_base, L.uniform_L);
      k.nax = (int)gr.size();
      axd.resize(2 * gr.size());
      for (size_t g = 0; g < gr.size(); ++g) merged(b, gr[g].first, gr[g].second, axd[g], axd[gr.size() + g]);
    }
    if (L.vt.alloc(vt.size() * h->tsize) != cudaSuccess || L.ax.alloc(axd.size() * h->tsize) != cudaSuccess)
      return fail(h, MLVS_ERR_OOM, "velocity table");
    if (h->tsize == 8) {
      CK(cudaMemcpy(L.vt.p, vt.data(), vt.size() * 8, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(L.ax.p, axd.data(), axd.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> vf(vt.begin(), vt.end());
      CK(cudaMemcpy(L.vt.p, vf.data(), vf.size() * 4, cudaMemcpyHostToDevice));
      std::vector<float> af(axd.begin(), axd.end());
      CK(cudaMemcpy(L.ax.p, af.data(), af.size() * 4, cudaMemcpyHostToDevice));
    }
    if (l != 0) continue;  // distributions live on level 0 in this build
    L.inst.resize(h->cfg.n_instances);
    for (int i = 0; i < h->cfg.n_instances; ++i) {
      LevelInst& I = L.inst[i];
      const size_t fbytes = 2ull * k.nv * k.ncell * h->ssize;
      if (I.f[0].alloc(fbytes) != cudaSuccess || I.f[1].alloc(fbytes) != cudaSuccess ||
          I.prm[0].alloc((size_t)NP * k.ncell * h->tsize) != cudaSuccess ||
          I.prm[1].alloc((size_t)NP * k.ncell * h->tsize) != cudaSuccess ||
          I.fprm.alloc((size_t)NP * k.nface * h->tsize) != cudaSuccess ||
          I.W.alloc(8ull * k.ncell * 8) != cudaSuccess ||
          I.cpart.alloc((size_t)k.nchunk * NMOM * k.ncell * 8) != cudaSuccess ||
          I.fpart.alloc((size_t)k.nchunk * NMOM * k.nface * 8) != cudaSuccess ||
          I.err.alloc(sizeof(int)) != cudaSuccess)
        return fail(h, MLVS_ERR_OOM, "device allocation of the distributions failed");
      CK(cudaMemsetAsync(I.err.p, 0, sizeof(int), h->stream));
      CK(cudaMemsetAsync(I.W.p, 0, I.W.n, h->stream));
      DevBuf dW0;
      if (dW0.alloc(4ull * k.ncell * 8) != cudaSuccess) return fail(h, MLVS_ERR_OOM, "init W");
      CK(cudaMemcpyAsync(dW0.p, h->initW.data() + 4ull * k.ncell * i, 4ull * k.ncell * 8,
                         cudaMemcpyHostToDevice, h->stream));
      CK(ops.init(h, L, I, dW0.as<double>()));
      CK(cudaStreamSynchronize(h->stream));
      int eflag = 0;
      CK(cudaMemcpy(&eflag, I.err.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (eflag & ERR_SINGULAR) return fail(h, MLVS_ERR_SINGULAR, "singular compatibility matrix at init");
    }
  }
  h->ready = true;
  return MLVS_OK;
}

static mlvs_status check_flags(mlvs_handle* h) {
  for (auto& L : h->lv)
    for (auto& I : L.inst) {
      int eflag = 0;
      CK(cudaMemcpyAsync(&eflag, I.err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (eflag) {
        mlvs_status s = (eflag & ERR_NONFINITE) ? MLVS_ERR_NONFINITE
                        : (eflag & ERR_POSITIVITY) ? MLVS_ERR_POSITIVITY : MLVS_ERR_SINGULAR;
        h->sticky = s;
        return fail(h, s, "device reported a non-finite, non-positive or singular state");
      }
    }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_step(mlvs_handle* h, int n_steps, mlvs_step_stats* stats) {
  if (!h) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (n_steps < 0) return fail(h, MLVS_ERR_ARG, "n_steps < 0");
  Ops ops = ops_for(h->cfg.storage, h->D);
  h->profiling = stats && stats->profile;
  h->prof.marks.clear();
  h->prof.used = 0;
  h->launches = 0;
  CK(cudaEventRecord(h->ev0, h->stream));
  for (int n = 0; n < n_steps; ++n)
    for (auto& L : h->lv)
      for (auto& I : L.inst) CK(ops.step(h, L, I, h->cfg.limiter));
  CK(cudaEventRecord(h->ev1, h->stream));
  mlvs_status s = check_flags(h);
  if (s != MLVS_OK) return s;
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    stats->ms_total = ms;
    stats->dt = h->dt;
    long long upd = 0;
    for (auto& L : h->lv)
      if (!L.inst.empty()) upd += (long long)L.k.ncell * L.k.nv * (long long)L.inst.size();
    stats->cell_velocity_updates = upd * n_steps;
    stats->n_levels = (int)h->lv.size();
    stats->launches = h->launches;
    for (int p = 0; p < 4; ++p) stats->ms_phase[p] = 0.f;
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

extern "C" mlvs_status mlvs_moments(mlvs_handle* h, int instance, unsigned fields, double* out, int out_on_device) {
  if (!h || !out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (h->sticky != MLVS_OK) return fail(h, MLVS_ERR_STATE, "handle holds an earlier error");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  Ops ops = ops_for(h->cfg.storage, h->D);
  LevelData& L = h->lv[0];
  LevelInst& I = L.inst[instance];
  if (!I.fresh) CK(ops.finalize_cells(h, L, I));
  mlvs_status s = check_flags(h);
  if (s != MLVS_OK) return s;
  const size_t nc = L.k.ncell;
  // field order: RHO U V T QX QY LEVEL RHOE
  const int src[8] = {0, 1, 2, 3, 4, 5, -1, 6};
  int j = 0;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int b = 0; b < 8; ++b) {
    if (!(fields & (1u << b))) continue;
    double* dst = out + j * nc;
    if (src[b] < 0) {
      std::vector<double> z(nc, 0.0);
      CK(cudaMemcpyAsync(dst, z.data(), nc * 8, out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
    } else {
      CK(cudaMemcpyAsync(dst, I.W.as<double>() + src[b] * nc, nc * 8, kind, h->stream));
    }
    ++j;
  }
  CK(cudaStreamSynchronize(h->stream));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_read_cells(mlvs_handle* h, int instance, int cell0, int ncells, double* out_g,
                                       double* out_h, int cap, int* nv_out) {
  if (!h || !out_g || !out_h || !nv_out) return MLVS_ERR_ARG;
  if (!h->ready) return fail(h, MLVS_ERR_STATE, "mlvs_set_velocity_levels has not been called");
  if (instance < 0 || instance >= h->cfg.n_instances) return fail(h, MLVS_ERR_ARG, "instance out of range");
  LevelData& L = h->lv[0];
  const int nc = L.k.ncell, nv = L.k.nv;
  if (cell0 < 0 || ncells < 0 || cell0 + ncells > nc) return fail(h, MLVS_ERR_ARG, "cell range out of bounds");
  if ((long long)cap < (long long)ncells * nv) return fail(h, MLVS_ERR_ARG, "output capacity too small");
  *nv_out = nv;
  LevelInst& I = L.inst[instance];
  std::vector<char> buf((size_t)ncells * h->ssize);
  for (int comp = 0; comp < 2; ++comp) {
    double* dst = comp == 0 ? out_g : out_h;
    for (int v = 0; v < nv; ++v) {
      const char* src = reinterpret_cast<const char*>(I.f[I.cur].p) +
                        (((size_t)comp * nv + v) * nc + cell0) * h->ssize;
      CK(cudaMemcpyAsync(buf.data(), src, (size_t)ncells * h->ssize, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int c = 0; c < ncells; ++c) {
        double x;
        if (h->ssize == 8) x = reinterpret_cast<const double*>(buf.data())[c];
        else if (h->ssize == 4) x = reinterpret_cast<const float*>(buf.data())[c];
        else x = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(buf.data())[c]);
        dst[(size_t)c * nv + v] = x;
      }
    }
  }
  return MLVS_OK;
}
