// Host emulation of CUDA thread blocks for kernels that cooperate through shared memory and
// barriers (test infrastructure): one block at a time, its threads as std::threads, a
// std::barrier for __syncthreads, and per warp of 32 threads a std::barrier and an exchange
// slot per thread for the warp shuffles, votes and __syncwarp (every lane of a warp takes part
// in each, as the full-mask calls of the library's kernels require).  A thread that returns
// drops out of its barriers, as an exited thread no longer holds a CUDA barrier up.  Arithmetic built-ins come from emu_math.hpp; atomics are
// sequentially consistent host atomics.  Launch coordinates are thread-local.
// __shared__ arrays become static storage (one block runs at a time, and each kernel
// instantiation has its own); a file that emulates a kernel with dynamic shared memory
// defines EMU_SHARED_SPEC as empty before including this header and provides the buffer.
#pragma once
#include <barrier>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#define EMU_WARPS
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

// warp exchanges of the running block
static std::vector<std::unique_ptr<std::barrier<>>> g_warp_barriers;
static unsigned long long g_warp_slot[1024];
static inline void emu_warp_wait() { g_warp_barriers[threadIdx.x >> 5]->arrive_and_wait(); }
template <class X> static inline X emu_warp_read(X v, int src_lane) {
  static_assert(sizeof(X) <= sizeof(unsigned long long), "exchange of at most 8 bytes");
  const int t = (int)threadIdx.x, base = t & ~31;
  std::memcpy(&g_warp_slot[t], &v, sizeof(X));
  emu_warp_wait();
  X r;
  std::memcpy(&r, &g_warp_slot[base + src_lane], sizeof(X));
  emu_warp_wait();
  return r;
}
template <class X> static inline X __shfl_xor_sync(unsigned, X v, int o, int w = 32) {
  const int l = (int)(threadIdx.x & 31);
  return emu_warp_read(v, (l & ~(w - 1)) | ((l ^ o) & (w - 1)));
}
template <class X> static inline X __shfl_up_sync(unsigned, X v, unsigned d, int w = 32) {
  const int l = (int)(threadIdx.x & 31), s = l - (int)d;
  return emu_warp_read(v, (s >= (l & ~(w - 1))) ? s : l);
}
static inline bool __any_sync(unsigned, int p) {
  const int t = (int)threadIdx.x, base = t & ~31;
  g_warp_slot[t] = p != 0;
  emu_warp_wait();
  bool any = false;
  for (int l = 0; l < 32; ++l) any = any || g_warp_slot[base + l] != 0;
  emu_warp_wait();
  return any;
}
static inline void __syncwarp(unsigned = 0xffffffffu) { emu_warp_wait(); }

// Runs body() as every thread of every block of grid (x, y) x block (x dimension only).
template <class F> void emu_launch(dim3 grid, unsigned block, F body) {
  gridDim = grid;
  blockDim = dim3(block, 1, 1);
  for (unsigned by = 0; by < grid.y; ++by)
    for (unsigned bx = 0; bx < grid.x; ++bx) {
      std::barrier<> bar(block);
      g_block_barrier = &bar;
      g_warp_barriers.clear();
      for (unsigned w = 0; w * 32 < block; ++w)
        g_warp_barriers.push_back(std::make_unique<std::barrier<>>((std::ptrdiff_t)std::min(32u, block - 32 * w)));
      std::vector<std::thread> th;
      th.reserve(block);
      for (unsigned t = 0; t < block; ++t)
        th.emplace_back([&body, t, bx, by] {
          threadIdx = {t, 0, 0};
          blockIdx = {bx, by, 0};
          body();
          g_warp_barriers[t >> 5]->arrive_and_drop();
          g_block_barrier->arrive_and_drop();
        });
      for (auto& x : th) x.join();
    }
}
template <class F> void emu_launch(unsigned grid, unsigned block, F body) { emu_launch(dim3(grid, 1, 1), block, body); }
