// Host definitions of the CUDA built-ins the library's per-element device functions use, so
// that those functions compile as plain C++ and run in loops on the CPU (test infrastructure).
// Arithmetic built-ins come from emu_math.hpp; a barrier is a no-op and atomics are plain
// updates (one thread runs).
#pragma once
#include <algorithm>

#include "emu_math.hpp"

static inline void __syncthreads() {}
static inline int atomicOr(int* p, int v) { const int o = *p; *p |= v; return o; }
static inline int atomicAdd(int* p, int v) { const int o = *p; *p += v; return o; }
static inline int atomicCAS(int* p, int cmp, int v) { const int o = *p; if (o == cmp) *p = v; return o; }
// launch coordinates: referenced by kernels the emulator compiles but never runs
static const uint3 threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0};
static const dim3 blockDim(1, 1, 1), gridDim(1, 1, 1);
