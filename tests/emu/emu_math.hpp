// Host definitions of the CUDA arithmetic built-ins the library's device code uses, shared by
// every CPU emulation of it (test infrastructure).  Rounded intrinsics map to IEEE operations
// in the same precision (fma stays fused) and stay separately rounded even where the caller is
// compiled with contraction on: an empty asm makes each result opaque to fusion, as the GPU
// never fuses an explicitly rounded intrinsic.  The fast exponential maps to the C library's.
// Warp shuffles are not emulated here: a kernel that reaches one aborts, so an emulated launch
// that needs lanes to exchange values cannot pass by accident; the block emulation of
// cta_shim.hpp defines EMU_WARPS and provides them.
#pragma once
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#ifndef __launch_bounds__
#define __launch_bounds__(...)
#endif

using std::isfinite;
using std::max;
using std::min;
template <class X> static inline X emu_opaque(X r) {
  asm("" : "+x"(r));
  return r;
}
float __expf(float a) { return std::exp(a); }
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline float __fmul_rn(float a, float b) { return emu_opaque(a * b); }
static inline float __fadd_rn(float a, float b) { return emu_opaque(a + b); }
static inline float __fsub_rn(float a, float b) { return emu_opaque(a - b); }
static inline float __fdividef(float a, float b) { return a / b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline double __dmul_rn(double a, double b) { return emu_opaque(a * b); }
static inline double __dadd_rn(double a, double b) { return emu_opaque(a + b); }
static inline double __dsub_rn(double a, double b) { return emu_opaque(a - b); }
template <class X> static inline X __ldg(const X* p) { return *p; }
static inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}
#ifndef EMU_WARPS   // the block emulation (cta_shim.hpp) provides real warp exchanges
template <class X> static inline X __shfl_xor_sync(unsigned, X v, int, int = 32) {
  std::fprintf(stderr, "emulation: a warp shuffle was reached; lanes are not emulated\n");
  std::abort();
  return v;
}
template <class X> static inline X __shfl_up_sync(unsigned, X v, unsigned, int = 32) {
  std::fprintf(stderr, "emulation: a warp shuffle was reached; lanes are not emulated\n");
  std::abort();
  return v;
}
static inline bool __any_sync(unsigned, int v) {
  std::fprintf(stderr, "emulation: a warp vote was reached; lanes are not emulated\n");
  std::abort();
  return v != 0;
}
static inline void __syncwarp(unsigned = 0xffffffffu) {
  std::fprintf(stderr, "emulation: a warp barrier was reached; lanes are not emulated\n");
  std::abort();
}
#endif
// packed two-lane FP32 (sm_100 and later): each lane an IEEE operation, as on the GPU
static inline float2 __fadd2_rn(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
static inline float2 __fmul2_rn(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
}
static inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline float __uint2float_rn(unsigned u) { return (float)u; }
