// C ABI of the unstructured-mesh step (one velocity space): handle, buffers, kernel launches.
//
// Each pass of ustep.cuh runs as one kernel, a grid-stride loop over the pass's flat index
// (consecutive threads take consecutive cells or faces of one velocity plane, so every load of
// a distribution and every store is coalesced).  Grids are capped at 16 CTAs of 256 threads
// per SM, and the passes are ordered on the handle's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlvs.h"
#include "mlvs_internal.h"
#include "ustep.cuh"
#include "ustep_host.hpp"

using namespace mlvs;

namespace {

constexpr int U_BLOCK = 256;
constexpr long U_MAX_BLOCKS = 148L * 16;

template <int E, class T>
__global__ void __launch_bounds__(U_BLOCK) k_u(const UArgs<T> a, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    u_elem<E, T>(a, i);
}

template <class T> struct GpuRun {
  const UArgs<T>* a;
  cudaStream_t s;
  template <int E> void pass(long n) {
    if (n <= 0) return;
    long blocks = (n + U_BLOCK - 1) / U_BLOCK;
    if (blocks > U_MAX_BLOCKS) blocks = U_MAX_BLOCKS;
    k_u<E, T><<<(unsigned)blocks, U_BLOCK, 0, s>>>(*a, n);
  }
};

struct UBuf {
  void* p = nullptr;
  UBuf() = default;
  UBuf(const UBuf&) = delete;
  UBuf& operator=(const UBuf&) = delete;
  ~UBuf() { if (p) cudaFree(p); }
};

mlvs_status ufail(mlvs_status s, const std::string& msg) {
  mlvs_internal_set_error(msg.c_str());
  return s;
}

}  // namespace

struct mlvs_uhandle {
  UHost u;
  UHostConfig c;
  int storage = MLVS_F64;
  cudaStream_t stream = nullptr;
  UBuf buf[UB_N];
  UArgs<double> a64;
  UArgs<float> a32;
  int failed = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~mlvs_uhandle() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

namespace {

template <class T> mlvs_status u_setup(mlvs_uhandle* h, const double* W0) {
  void* p[UB_N];
  for (int b = 0; b < UB_N; ++b) {
    int type;
    size_t count;
    u_buffer(h->u, b, type, count);
    const size_t es = type == 0 ? sizeof(T) : type == 1 ? sizeof(int) : sizeof(double);
    const size_t bytes = count * es;
    if (cudaMalloc(&h->buf[b].p, bytes ? bytes : 16) != cudaSuccess)
      return ufail(MLVS_ERR_OOM, "mlvs_ucreate: device allocation failed");
    p[b] = h->buf[b].p;
    std::vector<T> tv;
    std::vector<int> iv;
    u_constant<T>(h->u, b, tv, iv);
    cudaError_t e = cudaSuccess;
    if (!tv.empty()) e = cudaMemcpy(p[b], tv.data(), tv.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (!iv.empty()) e = cudaMemcpy(p[b], iv.data(), iv.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (b == UB_W0) e = cudaMemcpy(p[b], W0, bytes, cudaMemcpyHostToDevice);
    if (b == UB_ERR || b == UB_W || b == UB_CPRM8 || b == UB_FPRM8) e = cudaMemset(p[b], 0, bytes);
    if (e != cudaSuccess) return ufail(MLVS_ERR_CUDA, std::string("mlvs_ucreate: ") + cudaGetErrorString(e));
  }
  UArgs<T> a = u_wire<T>(h->u, h->c, p);
  if constexpr (sizeof(T) == 8) h->a64 = a;
  else h->a32 = a;
  GpuRun<T> run{&a, h->stream};
  u_init_sequence<T>(run, a);
  int err = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p[UB_ERR], sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return ufail(MLVS_ERR_CUDA, std::string("mlvs_ucreate: ") + cudaGetErrorString(e));
  if (err) return ufail(MLVS_ERR_SINGULAR, "mlvs_ucreate: the corrected initial Maxwellian failed");
  return MLVS_OK;
}

mlvs_status u_status_of(int err) {
  if (err & ERR_NONFINITE) return MLVS_ERR_NONFINITE;
  if (err & ERR_POSITIVITY) return MLVS_ERR_POSITIVITY;
  if (err & ERR_SINGULAR) return MLVS_ERR_SINGULAR;
  return MLVS_OK;
}

}  // namespace

extern "C" mlvs_status mlvs_ucreate(const mlvs_uconfig* cfg, int n_node, const double* node_xy, int n_cell,
                                    const int* cell_ptr, const int* cell_nodes, const int* edge_wall,
                                    const double* init_W, mlvs_uhandle** out) {
  if (!cfg || !node_xy || !cell_ptr || !cell_nodes || !init_W || !out)
    return ufail(MLVS_ERR_ARG, "mlvs_ucreate: null argument");
  *out = nullptr;
  if (n_node < 3 || n_cell < 1) return ufail(MLVS_ERR_ARG, "mlvs_ucreate: need three nodes and one cell");
  for (int i = 0; i < n_cell; ++i) {
    const double* w = init_W + 4 * (size_t)i;
    if (!(w[0] > 0) || !(w[3] > 0) || !std::isfinite(w[0]) || !std::isfinite(w[1]) || !std::isfinite(w[2]) ||
        !std::isfinite(w[3]))
      return ufail(MLVS_ERR_ARG, "mlvs_ucreate: initial density and temperature must be finite and > 0");
  }
  mlvs_uhandle* h = new (std::nothrow) mlvs_uhandle();
  if (!h) return ufail(MLVS_ERR_OOM, "mlvs_ucreate: host allocation failed");
  std::string why = u_config(*cfg, h->c);
  if (why.empty()) why = u_build_host(n_node, node_xy, n_cell, cell_ptr, cell_nodes, edge_wall, h->c, h->u);
  if (!why.empty()) {
    delete h;
    return ufail(MLVS_ERR_ARG, "mlvs_ucreate: " + why);
  }
  h->storage = cfg->storage;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  if (cudaEventCreate(&h->e0) != cudaSuccess || cudaEventCreate(&h->e1) != cudaSuccess) {
    delete h;
    return ufail(MLVS_ERR_CUDA, "mlvs_ucreate: cudaEventCreate failed");
  }
  const mlvs_status st = h->storage == MLVS_F64 ? u_setup<double>(h, init_W) : u_setup<float>(h, init_W);
  if (st != MLVS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_ustep(mlvs_uhandle* h, int n_steps, float* ms) {
  if (!h || n_steps < 0) return ufail(MLVS_ERR_ARG, "mlvs_ustep: bad argument");
  if (h->failed) return ufail(MLVS_ERR_STATE, "mlvs_ustep: an earlier step failed");
  cudaError_t e = cudaEventRecord(h->e0, h->stream);
  for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
    if (h->storage == MLVS_F64) {
      GpuRun<double> run{&h->a64, h->stream};
      u_step_sequence<double>(run, h->a64);
    } else {
      GpuRun<float> run{&h->a32, h->stream};
      u_step_sequence<float>(run, h->a32);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->e1, h->stream);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->buf[UB_ERR].p, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return ufail(MLVS_ERR_CUDA, std::string("mlvs_ustep: ") + cudaGetErrorString(e));
  if (ms) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, h->e0, h->e1);
    *ms = t;
  }
  const mlvs_status st = u_status_of(err);
  if (st != MLVS_OK) {
    h->failed = 1;
    return ufail(st, "mlvs_ustep: a cell or face state failed (non-finite, non-positive or singular)");
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_uread(const mlvs_uhandle* h, double* g, double* hh) {
  if (!h || !g || !hh) return ufail(MLVS_ERR_ARG, "mlvs_uread: null argument");
  const size_t nc = h->u.nc, nv = h->u.nv, n = 2 * nc * nv;
  std::vector<double> f(n);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) {
    if (h->storage == MLVS_F64) {
      e = cudaMemcpy(f.data(), h->buf[UB_F].p, n * sizeof(double), cudaMemcpyDeviceToHost);
    } else {
      std::vector<float> t(n);
      e = cudaMemcpy(t.data(), h->buf[UB_F].p, n * sizeof(float), cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < n; ++i) f[i] = t[i];
    }
  }
  if (e != cudaSuccess) return ufail(MLVS_ERR_CUDA, std::string("mlvs_uread: ") + cudaGetErrorString(e));
  for (size_t v = 0; v < nv; ++v)
    for (size_t i = 0; i < nc; ++i) {
      g[i * nv + v] = f[v * nc + i];
      hh[i * nv + v] = f[(nv + v) * nc + i];
    }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_ucells(const mlvs_uhandle* h, double* W) {
  if (!h || !W) return ufail(MLVS_ERR_ARG, "mlvs_ucells: null argument");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(W, h->buf[UB_W].p, 11 * sizeof(double) * h->u.nc, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ufail(MLVS_ERR_CUDA, std::string("mlvs_ucells: ") + cudaGetErrorString(e));
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_uinfo(const mlvs_uhandle* h, int* nv, int* n_face, double* dt) {
  if (!h) return ufail(MLVS_ERR_ARG, "mlvs_uinfo: null handle");
  if (nv) *nv = h->u.nv;
  if (n_face) *n_face = h->u.nf;
  if (dt) *dt = h->u.dt;
  return MLVS_OK;
}

extern "C" void mlvs_udestroy(mlvs_uhandle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}
