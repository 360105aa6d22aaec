// Moment-consistent mapping between velocity spaces (Sec. 3.3.2 and Sec. 3.4).
//
// One CTA maps one item (a cell state, a ghost stencil value or a face flux) from a source
// space s to a target space t:
//   1. target moments (rho, rho u, rho v, rho E) of the source values (Eq. mapping_four_targets),
//      reduced over the source velocities;
//   2. hierarchical projection P_{s->t} (Eq. hierarchical_projection_operator ...
//      Eq. mapping_h_projection) from a CSR table: coarsening averages g and
//      H = h + |xi|^2 g with the source weights, refinement inherits them; h = H - |xi_t|^2 g;
//   3. the four-moment correction with unit weighting, raw basis [1, xi_x, xi_y, xi^2]
//      (Eq. raw_four_g_basis) and delta h = (3 - D + K) R T_tar delta g
//      (Eq. raw_four_gh_coupling).  The energy row minus (3-D+K) R T_tar / 2 times the mass row
//      leaves a matrix that depends on the target space only; its inverse is computed once per
//      space on the host (Sec. 3.3.2, last paragraph).
// Sources:
//   SRC_TILDE  phi~ of a cell (level switch, Eq. level_switch_conservation)
//   SRC_BARP   phi-bar-plus of a cell, formed from phi~ and the cell's model parameters
//              (Eq. interface_state_moment_matching)
//   SRC_FLUX   a face microflux (xi.n) phi (Eq. native_flux_moment_matching); T_tar = the face
//              temperature
#pragma once
#include "mlvs_common.cuh"

namespace mlvs {

enum { SRC_TILDE = 0, SRC_BARP = 1, SRC_FLUX = 2 };

struct SpaceView {
  int nv;
  const void* vt;        // [4][nv] (T): xi_x, xi_y, w_x, w_y
  const double* ainv;    // [16] inverse of the T-independent mapping matrix
};

struct MapItem {
  int src_slot;          // column of the source buffer
  int dst_slot;          // column of the target buffer
  int prm_slot;          // SRC_BARP: column of the source cell parameters; SRC_FLUX: face id
};

struct MapArgs {
  SpaceView s, t;
  const int* off;        // CSR: target point i -> [off[i], off[i+1])
  const int* idx;        // source points
  const void* wgt;       // (T) projection weights
  const void* src;       // source buffer [2][s.nv][src_ld]
  int src_ld;
  void* dst;             // target buffer [2][t.nv][dst_ld]
  int dst_ld;
  const void* prm;       // SRC_BARP: cell params [NP][prm_ld]; SRC_FLUX: face params [NP][prm_ld]
  int prm_ld;
  const MapItem* items;
  int nitems;
  double R, c0, cv, twoK; // gas: R, K+3-D, c_V/R... cv = c_V = (3+K)R/2
  int correct;           // 0: projection only
};

template <class T>
__device__ __forceinline__ double block_sum(double x, double* red) {
  // deterministic tree over the block (fixed order for a fixed blockDim)
  const int tid = threadIdx.x;
  red[tid] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Value of source point j of the item (g, h).
template <class SrcT, class T, int D, int KIND>
__device__ __forceinline__ void src_value(const MapArgs& a, const MapItem& it, int j, T& g, T& h) {
  const SrcT* S = reinterpret_cast<const SrcT*>(a.src);
  const long ld = a.src_ld;
  g = ldf<SrcT, T>(S + (long)j * ld + it.src_slot);
  h = ldf<SrcT, T>(S + ((long)a.s.nv + j) * ld + it.src_slot);
  if (KIND == SRC_BARP) {
    MP<T> m;
    m.load(reinterpret_cast<const T*>(a.prm), a.prm_ld, it.prm_slot);
    const T* vt = reinterpret_cast<const T*>(a.s.vt);
    T gs, hs;
    model_eval<T, D>(m, vt[j], (D == 2) ? vt[a.s.nv + j] : T(0), T(a.c0), T(a.twoK), gs, hs);
    g = Num<T>::fma(m.c1, Num<T>::sub(gs, g), g);
    h = Num<T>::fma(m.c1, Num<T>::sub(hs, h), h);
  }
}

template <class SrcT, class DstT, class T, int D, int KIND>
__global__ void __launch_bounds__(256) k_map(const MapArgs a) {
  __shared__ double red[256];
  __shared__ double coef[5];
  const int tid = threadIdx.x;
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* vtt = reinterpret_cast<const T*>(a.t.vt);
  const T* wgt = reinterpret_cast<const T*>(a.wgt);
  DstT* Dd = reinterpret_cast<DstT*>(a.dst);
  const int ns = a.s.nv, nt = a.t.nv;
  for (int itn = blockIdx.x; itn < a.nitems; itn += gridDim.x) {
    const MapItem it = a.items[itn];
    // 1. target moments over the source space
    KSum<T> r0, r1, r2, r3;
    r0.zero(); r1.zero(); r2.zero(); r3.zero();
    for (int j = tid; j < ns; j += blockDim.x) {
      T g, h;
      src_value<SrcT, T, D, KIND>(a, it, j, g, h);
      const T x = vs[j], y = (D == 2) ? vs[ns + j] : T(0);
      const T wg = vs[2 * ns + j] * (vs[3 * ns + j] * g);
      const T we = vs[2 * ns + j] * (vs[3 * ns + j] * ((x * x + y * y) * g + h));
      r0.add(wg); r1.add(wg * x); r2.add(wg * y); r3.add(T(0.5) * we);
    }
    const double M0 = block_sum<T>(r0.val(), red), M1 = block_sum<T>(r1.val(), red);
    const double M2 = block_sum<T>(r2.val(), red), M3 = block_sum<T>(r3.val(), red);
    // 2. projected values on the target space: their moments
    KSum<T> p0, p1, p2, p3;
    p0.zero(); p1.zero(); p2.zero(); p3.zero();
    for (int i = tid; i < nt; i += blockDim.x) {
      T g = T(0), H = T(0);
      for (int q = a.off[i]; q < a.off[i + 1]; ++q) {
        const int j = a.idx[q];
        T gj, hj;
        src_value<SrcT, T, D, KIND>(a, it, j, gj, hj);
        const T xj = vs[j], yj = (D == 2) ? vs[ns + j] : T(0);
        g += wgt[q] * gj;
        H += wgt[q] * (hj + (xj * xj + yj * yj) * gj);
      }
      const T x = vtt[i], y = (D == 2) ? vtt[nt + i] : T(0);
      const T h = H - (x * x + y * y) * g;
      const T wg = vtt[2 * nt + i] * (vtt[3 * nt + i] * g);
      const T we = vtt[2 * nt + i] * (vtt[3 * nt + i] * ((x * x + y * y) * g + h));
      p0.add(wg); p1.add(wg * x); p2.add(wg * y); p3.add(T(0.5) * we);
    }
    const double P0 = block_sum<T>(p0.val(), red), P1 = block_sum<T>(p1.val(), red);
    const double P2 = block_sum<T>(p2.val(), red), P3 = block_sum<T>(p3.val(), red);
    // 3. coefficients of the correction
    if (tid == 0) {
      double RT;
      if (KIND == SRC_FLUX) {
        RT = (double)reinterpret_cast<const T*>(a.prm)[(long)P_RT * a.prm_ld + it.prm_slot];
      } else {
        const double ux = M1 / M0, uy = M2 / M0;
        RT = a.R * (M3 / M0 - 0.5 * (ux * ux + uy * uy)) / a.cv;
      }
      const double cK = a.c0 * RT;
      double d[4] = {M0 - P0, M1 - P1, M2 - P2, M3 - P3};
      d[3] -= 0.5 * cK * d[0];
      for (int r = 0; r < 4; ++r) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) s += a.t.ainv[4 * r + c] * d[c];
        coef[r] = a.correct ? s : 0.0;
      }
      coef[4] = cK;
    }
    __syncthreads();
    const T a0 = T(coef[0]), a1 = T(coef[1]), a2 = T(coef[2]), a3 = T(coef[3]), cK = T(coef[4]);
    // 4. write projection + correction
    for (int i = tid; i < nt; i += blockDim.x) {
      T g = T(0), H = T(0);
      for (int q = a.off[i]; q < a.off[i + 1]; ++q) {
        const int j = a.idx[q];
        T gj, hj;
        src_value<SrcT, T, D, KIND>(a, it, j, gj, hj);
        const T xj = vs[j], yj = (D == 2) ? vs[ns + j] : T(0);
        g += wgt[q] * gj;
        H += wgt[q] * (hj + (xj * xj + yj * yj) * gj);
      }
      const T x = vtt[i], y = (D == 2) ? vtt[nt + i] : T(0);
      const T x2 = x * x + y * y;
      const T h = H - x2 * g;
      const T dg = a0 + a1 * x + a2 * y + a3 * x2;
      stf<DstT, T>(Dd + (long)i * a.dst_ld + it.dst_slot, g + dg);
      stf<DstT, T>(Dd + ((long)nt + i) * a.dst_ld + it.dst_slot, h + cK * dg);
    }
    __syncthreads();
  }
}

// Column copy between two level buffers [rows][ld] (cells whose space does not change).
template <class S>
__global__ void k_copy_cols(const S* __restrict__ src, int src_ld, S* __restrict__ dst, int dst_ld, int rows,
                            const MapItem* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const MapItem m = items[it];
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      dst[(long)r * dst_ld + m.dst_slot] = src[(long)r * src_ld + m.src_slot];
  }
}

// Moment shift of every cell of a level: the cell velocity before a change of level.
template <class T>
__global__ void k_set_shift(T* __restrict__ prm, int n, const int* __restrict__ cells,
                            const T* __restrict__ uc, int ncell) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int c = cells[s];
  prm[P_UX * (long)n + s] = uc[c];
  prm[P_UY * (long)n + s] = uc[ncell + c];
}

// Per-cell velocity (u, v) of the cells of one level, scattered to the global cell index,
// from the level's parameter array (used for face shifts across levels).
template <class T>
__global__ void k_scatter_velocity(const T* __restrict__ prm, int n, const int* __restrict__ cells,
                                   T* __restrict__ uc, int ncell) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int c = cells[s];
  uc[c] = prm[P_UX * (long)n + s];
  uc[ncell + c] = prm[P_UY * (long)n + s];
}

}  // namespace mlvs
