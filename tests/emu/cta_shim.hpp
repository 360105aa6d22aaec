// Host emulation of CUDA thread blocks for kernels that cooperate through shared memory and
// barriers (test infrastructure): one block at a time, its threads as std::threads, a
// std::barrier for __syncthreads.  Arithmetic built-ins come from emu_math.hpp; atomics are
// sequentially consistent host atomics.  Launch coordinates are thread-local.
// __shared__ arrays become static storage (one block runs at a time, and each kernel
// instantiation has its own); a file that emulates a kernel with dynamic shared memory
// defines EMU_SHARED_SPEC as empty before including this header and provides the buffer.
#pragma once
#include <barrier>
#include <thread>
#include <vector>

#include "emu_math.hpp"

#ifndef EMU_SHARED_SPEC
#define EMU_SHARED_SPEC static
#endif
#undef __shared__
#define __shared__ EMU_SHARED_SPEC

static inline int atomicOr(int* p, int v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
static inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
static inline int atomicCAS(int* p, int cmp, int v) {
  __atomic_compare_exchange_n(p, &cmp, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
  return cmp;
}

thread_local uint3 threadIdx, blockIdx;
static dim3 blockDim, gridDim;
static std::barrier<>* g_block_barrier = nullptr;
static inline void __syncthreads() { g_block_barrier->arrive_and_wait(); }

// Runs body() as every thread of every block of grid (x, y) x block (x dimension only).
template <class F> void emu_launch(dim3 grid, unsigned block, F body) {
  gridDim = grid;
  blockDim = dim3(block, 1, 1);
  for (unsigned by = 0; by < grid.y; ++by)
    for (unsigned bx = 0; bx < grid.x; ++bx) {
      std::barrier<> bar(block);
      g_block_barrier = &bar;
      std::vector<std::thread> th;
      th.reserve(block);
      for (unsigned t = 0; t < block; ++t)
        th.emplace_back([&body, t, bx, by] {
          threadIdx = {t, 0, 0};
          blockIdx = {bx, by, 0};
          body();
        });
      for (auto& x : th) x.join();
    }
}
template <class F> void emu_launch(unsigned grid, unsigned block, F body) { emu_launch(dim3(grid, 1, 1), block, body); }
