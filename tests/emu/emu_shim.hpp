// Host definitions of the CUDA built-ins the library's per-element device functions use, so
// that those functions compile as plain C++ and run in loops on the CPU (test infrastructure).
// Rounded arithmetic intrinsics map to IEEE operations in the same precision (fma stays fused);
// the fast exponential maps to the C library's; warp shuffles return the lane's own value (the
// per-element functions run with one lane per point); atomics are plain updates (one thread).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#ifndef __launch_bounds__
#define __launch_bounds__(...)
#endif

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
template <class X> static inline X __shfl_xor_sync(unsigned, X v, int, int = 32) { return v; }
static inline void __syncthreads() {}
static inline int atomicOr(int* p, int v) { const int o = *p; *p |= v; return o; }
static inline int atomicAdd(int* p, int v) { const int o = *p; *p += v; return o; }
// launch coordinates: referenced by kernels the emulator compiles but never runs
static const uint3 threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0};
static const dim3 blockDim(1, 1, 1), gridDim(1, 1, 1);
