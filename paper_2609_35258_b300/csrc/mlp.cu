// Level selector: a 10 -> 64 -> 64 -> 4 ReLU network, forward, gradient and training step.
//
// The network maps cell features to logits over four velocity levels; it is trained with
// softmax cross-entropy on labels that the criterion of Sec. 3.2 produces (not part of the
// paper's method: a cheaper stand-in for the criterion, kept behind a confidence threshold).
//
// Precision: the forward and backward passes read BF16 weights and accumulate in FP32; the
// update keeps an FP32 master copy (SGD with momentum) and rounds it to BF16 (nearest even).
// Every reduction has a fixed order: a block of MLP_BATCH samples sums its per-sample
// gradient terms sample by sample, and the block partials are summed block by block.
//
// Parameter layout (5,124): W1 [64][10], b1 [64], W2 [64][64], b2 [64], W3 [4][64], b3 [4].
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <string>

#include "../../include/mlvs.h"
#include "mlvs_internal.h"

namespace {

constexpr int NI = 10, NH = 64, NO = 4;
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NO * NH, NPAR = OB3 + NO;
static_assert(NPAR == 5124, "parameter count");
constexpr int FWD_BLOCK = 128;
constexpr int MLP_BATCH = 64;     // samples per backward block
constexpr int BWD_THREADS = 128;

// Logits (and softmax probabilities) of n samples, one thread per sample.
__global__ void __launch_bounds__(FWD_BLOCK) k_mlp_forward(const float* __restrict__ X, int n,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            float* __restrict__ logits, float* __restrict__ prob) {
  __shared__ float w[NPAR];
  for (int i = threadIdx.x; i < NPAR; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[NI], h1[NH];
#pragma unroll
  for (int c = 0; c < NI; ++c) x[c] = X[(long)s * NI + c];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float z = w[OB1 + j];
#pragma unroll
    for (int c = 0; c < NI; ++c) z = fmaf(w[OW1 + j * NI + c], x[c], z);
    h1[j] = fmaxf(z, 0.f);
  }
  float lg[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) lg[k] = w[OB3 + k];
  for (int j = 0; j < NH; ++j) {
    float z = w[OB2 + j];
#pragma unroll
    for (int i = 0; i < NH; ++i) z = fmaf(w[OW2 + j * NH + i], h1[i], z);
    const float h2 = fmaxf(z, 0.f);
#pragma unroll
    for (int k = 0; k < NO; ++k) lg[k] = fmaf(w[OW3 + k * NH + j], h2, lg[k]);
  }
  float m = lg[0];
#pragma unroll
  for (int k = 1; k < NO; ++k) m = fmaxf(m, lg[k]);
  float e[NO], se = 0.f;
#pragma unroll
  for (int k = 0; k < NO; ++k) { e[k] = expf(lg[k] - m); se += e[k]; }
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    if (logits) logits[(long)s * NO + k] = lg[k];
    if (prob) prob[(long)s * NO + k] = e[k] / se;
  }
}

// Shared memory of a backward block (floats).
constexpr int SX = 0, SH1 = SX + MLP_BATCH * NI, SH2 = SH1 + MLP_BATCH * NH, SD3 = SH2 + MLP_BATCH * NH,
              SD2 = SD3 + MLP_BATCH * NO, SD1 = SD2 + MLP_BATCH * NH, SW = SD1 + MLP_BATCH * NH,
              SLOSS = SW + NPAR, SBWD = SLOSS + MLP_BATCH;

// Per-block gradient of the mean cross-entropy over n samples (block b covers samples
// [b MLP_BATCH, (b+1) MLP_BATCH)): gpart[b][NPAR], lpart[b] = the block's sum of -log p_y.
__global__ void __launch_bounds__(BWD_THREADS) k_mlp_backward(const float* __restrict__ X, const int* __restrict__ y,
                                                              int n, const __nv_bfloat16* __restrict__ wb,
                                                              float* __restrict__ gpart, float* __restrict__ lpart,
                                                              int* __restrict__ err) {
  extern __shared__ float sm[];
  float* w = sm + SW;
  for (int i = threadIdx.x; i < NPAR; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  const int s0 = blockIdx.x * MLP_BATCH;
  const float inv_n = 1.f / (float)n;
  __syncthreads();
  // per sample: activations, softmax, output and hidden deltas
  for (int t = threadIdx.x; t < MLP_BATCH; t += blockDim.x) {
    const int s = s0 + t;
    float* x = sm + SX + t * NI;
    float* h1 = sm + SH1 + t * NH;
    float* h2 = sm + SH2 + t * NH;
    float* d3 = sm + SD3 + t * NO;
    float* d2 = sm + SD2 + t * NH;
    float* d1 = sm + SD1 + t * NH;
    if (s >= n) {
      for (int c = 0; c < NI; ++c) x[c] = 0.f;
      for (int j = 0; j < NH; ++j) { h1[j] = 0.f; h2[j] = 0.f; d2[j] = 0.f; d1[j] = 0.f; }
      for (int k = 0; k < NO; ++k) d3[k] = 0.f;
      sm[SLOSS + t] = 0.f;
      continue;
    }
    for (int c = 0; c < NI; ++c) x[c] = X[(long)s * NI + c];
    for (int j = 0; j < NH; ++j) {
      float z = w[OB1 + j];
      for (int c = 0; c < NI; ++c) z = fmaf(w[OW1 + j * NI + c], x[c], z);
      h1[j] = fmaxf(z, 0.f);
    }
    float lg[NO];
    for (int k = 0; k < NO; ++k) lg[k] = w[OB3 + k];
    for (int j = 0; j < NH; ++j) {
      float z = w[OB2 + j];
      for (int i = 0; i < NH; ++i) z = fmaf(w[OW2 + j * NH + i], h1[i], z);
      h2[j] = fmaxf(z, 0.f);
      for (int k = 0; k < NO; ++k) lg[k] = fmaf(w[OW3 + k * NH + j], h2[j], lg[k]);
    }
    float m = lg[0];
    for (int k = 1; k < NO; ++k) m = fmaxf(m, lg[k]);
    float e[NO], se = 0.f;
    for (int k = 0; k < NO; ++k) { e[k] = expf(lg[k] - m); se += e[k]; }
    int lab = y[s];
    if (lab < 0 || lab >= NO) { atomicOr(err, 1); lab = 0; }
    sm[SLOSS + t] = -(lg[lab] - m - logf(se));
    for (int k = 0; k < NO; ++k) d3[k] = (e[k] / se - (k == lab ? 1.f : 0.f)) * inv_n;
    for (int j = 0; j < NH; ++j) {
      float a = 0.f;
      for (int k = 0; k < NO; ++k) a = fmaf(d3[k], w[OW3 + k * NH + j], a);
      d2[j] = h2[j] > 0.f ? a : 0.f;
    }
    for (int i = 0; i < NH; ++i) {
      float a = 0.f;
      for (int j = 0; j < NH; ++j) a = fmaf(d2[j], w[OW2 + j * NH + i], a);
      d1[i] = h1[i] > 0.f ? a : 0.f;
    }
  }
  __syncthreads();
  // per parameter: the block's sum over its samples, in sample order
  float* gp = gpart + (long)blockIdx.x * NPAR;
  for (int p = threadIdx.x; p < NPAR; p += blockDim.x) {
    const float* a;
    const float* b;
    int sa, sb;
    if (p < OB1) { a = sm + SD1 + p / NI; sa = NH; b = sm + SX + p % NI; sb = NI; }
    else if (p < OW2) { a = sm + SD1 + (p - OB1); sa = NH; b = nullptr; sb = 0; }
    else if (p < OB2) { const int q = p - OW2; a = sm + SD2 + q / NH; sa = NH; b = sm + SH1 + q % NH; sb = NH; }
    else if (p < OW3) { a = sm + SD2 + (p - OB2); sa = NH; b = nullptr; sb = 0; }
    else if (p < OB3) { const int q = p - OW3; a = sm + SD3 + q / NH; sa = NO; b = sm + SH2 + q % NH; sb = NH; }
    else { a = sm + SD3 + (p - OB3); sa = NO; b = nullptr; sb = 0; }
    float g = 0.f;
    if (b) {
      for (int t = 0; t < MLP_BATCH; ++t) g = fmaf(a[t * sa], b[t * sb], g);
    } else {
      for (int t = 0; t < MLP_BATCH; ++t) g += a[t * sa];
    }
    gp[p] = g;
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int t = 0; t < MLP_BATCH; ++t) l += sm[SLOSS + t];
    lpart[blockIdx.x] = l;
  }
}

// Sum of the block partials in block order (one thread per parameter); optionally the SGD
// step with momentum on the FP32 master weights and their BF16 copy.
__global__ void k_mlp_reduce(const float* __restrict__ gpart, const float* __restrict__ lpart, int nblk, int n,
                             float* __restrict__ grad, float* __restrict__ master, float* __restrict__ vel,
                             __nv_bfloat16* __restrict__ wb, float lr, float mom, int update,
                             float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += (double)lpart[b];
    *loss = (float)(l / (double)n);
  }
  if (p >= NPAR) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += gpart[(long)b * NPAR + p];
  if (grad) grad[p] = g;
  if (update) {
    const float v = fmaf(mom, vel[p], g);
    vel[p] = v;
    const float m = fmaf(-lr, v, master[p]);
    master[p] = m;
    wb[p] = __float2bfloat16_rn(m);
  }
}

__global__ void k_mlp_to_bf16(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPAR) wb[p] = __float2bfloat16_rn(master[p]);
}

}  // namespace

struct mlvs_mlp {
  cudaStream_t stream = nullptr;
  float* master = nullptr;        // FP32 master weights [NPAR]
  float* vel = nullptr;           // momentum [NPAR]
  __nv_bfloat16* wb = nullptr;    // BF16 weights [NPAR]
  float* gpart = nullptr;         // [cap][NPAR]
  float* lpart = nullptr;         // [cap]
  float* loss = nullptr;          // [1]
  int* err = nullptr;             // [1]
  int cap = 0;                    // backward blocks the scratch holds
};

namespace {

mlvs_status mlp_fail(mlvs_status s, const char* msg) {
  mlvs_internal_set_error(msg);
  return s;
}

mlvs_status ensure_scratch(mlvs_mlp* m, int nblk) {
  if (nblk <= m->cap) return MLVS_OK;
  cudaFree(m->gpart);
  cudaFree(m->lpart);
  m->gpart = nullptr;
  m->lpart = nullptr;
  m->cap = 0;
  if (cudaMalloc(&m->gpart, (size_t)nblk * NPAR * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->lpart, (size_t)nblk * sizeof(float)) != cudaSuccess)
    return mlp_fail(MLVS_ERR_OOM, "mlp scratch allocation failed");
  m->cap = nblk;
  return MLVS_OK;
}

// Gradient (and optionally the update) over n samples; loss written to *loss_host if non-null.
mlvs_status mlp_grad(mlvs_mlp* m, const float* X, const int* y, int n, float* grad, float lr, float mom,
                     int update, float* loss_host) {
  if (!m || !X || !y || n < 1) return mlp_fail(MLVS_ERR_ARG, "mlp: bad argument");
  const int nblk = (n + MLP_BATCH - 1) / MLP_BATCH;
  mlvs_status st = ensure_scratch(m, nblk);
  if (st != MLVS_OK) return st;
  const size_t smem = (size_t)SBWD * sizeof(float);
  if (cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return mlp_fail(MLVS_ERR_CUDA, "mlp: shared memory attribute");
  k_mlp_backward<<<nblk, BWD_THREADS, smem, m->stream>>>(X, y, n, m->wb, m->gpart, m->lpart, m->err);
  k_mlp_reduce<<<(NPAR + 127) / 128, 128, 0, m->stream>>>(m->gpart, m->lpart, nblk, n, grad, m->master, m->vel,
                                                           m->wb, lr, mom, update, m->loss);
  if (cudaGetLastError() != cudaSuccess) return mlp_fail(MLVS_ERR_CUDA, "mlp: launch failed");
  int e = 0;
  if (cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess) return MLVS_ERR_CUDA;
  if (loss_host && cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return MLVS_ERR_CUDA;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(MLVS_ERR_CUDA, "mlp: stream failed");
  if (e) {
    cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
    return mlp_fail(MLVS_ERR_ARG, "mlp: a label is outside 0..3");
  }
  return MLVS_OK;
}

}  // namespace

extern "C" mlvs_status mlvs_mlp_create(void* stream, mlvs_mlp** out) {
  if (!out) return MLVS_ERR_ARG;
  *out = nullptr;
  mlvs_mlp* m = new (std::nothrow) mlvs_mlp();
  if (!m) return MLVS_ERR_OOM;
  m->stream = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMalloc(&m->master, NPAR * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->vel, NPAR * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->wb, NPAR * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess || cudaMalloc(&m->err, sizeof(int)) != cudaSuccess) {
    mlvs_mlp_destroy(m);
    return mlp_fail(MLVS_ERR_OOM, "mlp allocation failed");
  }
  cudaMemsetAsync(m->master, 0, NPAR * sizeof(float), m->stream);
  cudaMemsetAsync(m->vel, 0, NPAR * sizeof(float), m->stream);
  cudaMemsetAsync(m->wb, 0, NPAR * sizeof(__nv_bfloat16), m->stream);
  cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    mlvs_mlp_destroy(m);
    return mlp_fail(MLVS_ERR_CUDA, "mlp initialisation failed");
  }
  *out = m;
  return MLVS_OK;
}

extern "C" void mlvs_mlp_destroy(mlvs_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  cudaFree(m->master);
  cudaFree(m->vel);
  cudaFree(m->wb);
  cudaFree(m->gpart);
  cudaFree(m->lpart);
  cudaFree(m->loss);
  cudaFree(m->err);
  delete m;
}

extern "C" mlvs_status mlvs_mlp_set_weights(mlvs_mlp* m, const float* w, int n) {
  if (!m || !w || n != NPAR) return mlp_fail(MLVS_ERR_ARG, "mlvs_mlp_set_weights: need 5124 weights");
  if (cudaMemcpyAsync(m->master, w, NPAR * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->vel, 0, NPAR * sizeof(float), m->stream) != cudaSuccess)
    return mlp_fail(MLVS_ERR_CUDA, "mlvs_mlp_set_weights: copy failed");
  k_mlp_to_bf16<<<(NPAR + 127) / 128, 128, 0, m->stream>>>(m->master, m->wb);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(MLVS_ERR_CUDA, "mlvs_mlp_set_weights");
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_mlp_get_weights(const mlvs_mlp* m, float* master, float* bf16_values, int n) {
  if (!m || n != NPAR) return mlp_fail(MLVS_ERR_ARG, "mlvs_mlp_get_weights: need 5124 weights");
  if (master && cudaMemcpy(master, m->master, NPAR * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MLVS_ERR_CUDA;
  if (bf16_values) {
    __nv_bfloat16 tmp[NPAR];
    if (cudaMemcpy(tmp, m->wb, sizeof(tmp), cudaMemcpyDeviceToHost) != cudaSuccess) return MLVS_ERR_CUDA;
    for (int i = 0; i < NPAR; ++i) bf16_values[i] = __bfloat162float(tmp[i]);
  }
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_mlp_forward(mlvs_mlp* m, const float* X, int n, float* logits, float* prob) {
  if (!m || !X || n < 0 || (!logits && !prob)) return mlp_fail(MLVS_ERR_ARG, "mlvs_mlp_forward: bad argument");
  if (n == 0) return MLVS_OK;
  k_mlp_forward<<<(n + FWD_BLOCK - 1) / FWD_BLOCK, FWD_BLOCK, 0, m->stream>>>(X, n, m->wb, logits, prob);
  if (cudaGetLastError() != cudaSuccess) return mlp_fail(MLVS_ERR_CUDA, "mlvs_mlp_forward: launch failed");
  return MLVS_OK;
}

extern "C" mlvs_status mlvs_mlp_gradient(mlvs_mlp* m, const float* X, const int* y, int n, float* grad,
                                         float* loss) {
  if (!grad) return mlp_fail(MLVS_ERR_ARG, "mlvs_mlp_gradient: grad is null");
  return mlp_grad(m, X, y, n, grad, 0.f, 0.f, 0, loss);
}

extern "C" mlvs_status mlvs_mlp_train_step(mlvs_mlp* m, const float* X, const int* y, int n, float lr,
                                           float momentum, float* loss) {
  if (!(lr > 0.f) || !(momentum >= 0.f) || !(momentum < 1.f)) return mlp_fail(MLVS_ERR_ARG, "mlvs_mlp_train_step: lr, momentum");
  return mlp_grad(m, X, y, n, nullptr, lr, momentum, 1, loss);
}
