// mlvs_moments_noalloc: conservative moments of caller-owned distributions without any device
// allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: a host process that reserves all of its
// device memory at start-up and must never allocate afterwards (an allocation synchronises the
// device and can fail under memory pressure), or a pipeline that records its work into a CUDA
// graph, where a stray allocation breaks the recording.  This entry point serves them: the
// caller passes inputs and outputs, and the partial sums live in a fixed file-scope device
// array that every GPU which loads the library holds until the process exits.
//
// Two kernels: per (cell, velocity chunk) partial sums into the scratch array, then a sum of
// the chunks in chunk order per cell (deterministic).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mlvs.h"
#include "mlvs_internal.h"

namespace {

constexpr int NA_MAX_CELLS = 16384;   // largest ncell accepted
constexpr int NA_CHUNKS = 16;         // velocity chunks (fixed)
constexpr int NA_MOM = 4;             // rho, rho u, rho v, rho E

// [chunk][moment][cell] partial sums: 16 x 4 x 16384 doubles = 8 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[NA_CHUNKS * NA_MOM * NA_MAX_CELLS];

constexpr int NA_MAX_DEVICES = 64;
double* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;

__global__ void k_na_partials(const float* __restrict__ g, const float* __restrict__ h, int nv, int ncell,
                              const float* __restrict__ xx, const float* __restrict__ xy,
                              const float* __restrict__ wx, const float* __restrict__ wy,
                              double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y;
  if (c >= ncell) return;
  const int per = (nv + NA_CHUNKS - 1) / NA_CHUNKS;
  const int v0 = chunk * per;
  const int v1 = min(nv, v0 + per);
  double r = 0.0, mx = 0.0, my = 0.0, e = 0.0;
  for (int v = v0; v < v1; ++v) {
    const double w = (double)wx[v] * (double)wy[v];
    const double gv = g[(long)v * ncell + c], hv = h[(long)v * ncell + c];
    const double x = xx[v], y = xy[v];
    r += w * gv;
    mx += w * x * gv;
    my += w * y * gv;
    e += 0.5 * w * ((x * x + y * y) * gv + hv);
  }
  // every slot of the rows this call reads is written here, empty chunks included
  part[((long)chunk * NA_MOM + 0) * NA_MAX_CELLS + c] = r;
  part[((long)chunk * NA_MOM + 1) * NA_MAX_CELLS + c] = mx;
  part[((long)chunk * NA_MOM + 2) * NA_MAX_CELLS + c] = my;
  part[((long)chunk * NA_MOM + 3) * NA_MAX_CELLS + c] = e;
}

__global__ void k_na_reduce(int ncell, const double* __restrict__ part, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  for (int m = 0; m < NA_MOM; ++m) {
    double s = 0.0;
    for (int k = 0; k < NA_CHUNKS; ++k) s += part[((long)k * NA_MOM + m) * NA_MAX_CELLS + c];
    out[(long)m * ncell + c] = s;
  }
}

// Device address of the scratch array on the current device, looked up once per device.
mlvs_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    mlvs_internal_set_error("mlvs_moments_noalloc: no usable current device");
    return MLVS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      mlvs_internal_set_error("mlvs_moments_noalloc: cudaGetSymbolAddress failed");
      return MLVS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MLVS_OK;
}

}  // namespace

extern "C" mlvs_status mlvs_moments_noalloc(const float* g, const float* h, int nv, int ncell,
                                            const float* xi_x, const float* xi_y, const float* w_x,
                                            const float* w_y, double* out, void* stream) {
  if (!g || !h || !xi_x || !xi_y || !w_x || !w_y || !out) {
    mlvs_internal_set_error("mlvs_moments_noalloc: null pointer");
    return MLVS_ERR_ARG;
  }
  if (nv < 1 || ncell < 1) {
    mlvs_internal_set_error("mlvs_moments_noalloc: nv and ncell must be positive");
    return MLVS_ERR_ARG;
  }
  if (ncell > NA_MAX_CELLS) {
    mlvs_internal_set_error("mlvs_moments_noalloc: ncell exceeds the 16384 cells of the fixed scratch array");
    return MLVS_ERR_ARG;
  }
  double* part = nullptr;
  mlvs_status st = scratch_for_current_device(&part);
  if (st != MLVS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  dim3 g1((ncell + 127) / 128, NA_CHUNKS);
  k_na_partials<<<g1, 128, 0, s>>>(g, h, nv, ncell, xi_x, xi_y, w_x, w_y, part);
  k_na_reduce<<<(ncell + 127) / 128, 128, 0, s>>>(ncell, part, out);
  if (cudaGetLastError() != cudaSuccess) {
    mlvs_internal_set_error("mlvs_moments_noalloc: kernel launch failed");
    return MLVS_ERR_CUDA;
  }
  return MLVS_OK;
}
