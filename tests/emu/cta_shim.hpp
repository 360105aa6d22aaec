// Host emulation of CUDA thread blocks for kernels that cooperate through shared memory and
// barriers (test infrastructure): one block at a time, its threads as std::threads, a
// std::barrier for __syncthreads, and __shared__ arrays as static storage (one block runs at
// a time, and each kernel instantiation has its own).  Launch coordinates are thread-local.
// Warp shuffles and atomics are not provided: kernels that need them are not run this way.
#pragma once
#include <barrier>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#ifndef __launch_bounds__
#define __launch_bounds__(...)
#endif
#undef __shared__
#define __shared__ static

using std::isfinite;
using std::max;
using std::min;
float __expf(float a) { return std::exp(a); }
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fdividef(float a, float b) { return a / b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
template <class X> static inline X __ldg(const X* p) { return *p; }
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }

thread_local uint3 threadIdx, blockIdx;
static dim3 blockDim, gridDim;
static std::barrier<>* g_block_barrier = nullptr;
static inline void __syncthreads() { g_block_barrier->arrive_and_wait(); }

// Runs body() as every thread of every block of grid x block (x dimension only).
template <class F> void emu_launch(unsigned grid, unsigned block, F body) {
  gridDim = dim3(grid, 1, 1);
  blockDim = dim3(block, 1, 1);
  for (unsigned b = 0; b < grid; ++b) {
    std::barrier<> bar(block);
    g_block_barrier = &bar;
    std::vector<std::thread> th;
    th.reserve(block);
    for (unsigned t = 0; t < block; ++t)
      th.emplace_back([&body, t, b] {
        threadIdx = {t, 0, 0};
        blockIdx = {b, 0, 0};
        body();
      });
    for (auto& x : th) x.join();
  }
}
