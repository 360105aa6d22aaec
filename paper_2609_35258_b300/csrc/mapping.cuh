// Moment-consistent mapping between velocity spaces (Sec. 3.3.2 and Sec. 3.4).
//
// A CTA maps a group of items (cell states, ghost stencil values or face fluxes) from a source
// space s to a target space t, each item independently:
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

// Value of source point j of an item (g, h); m holds the item's cell parameters (SRC_BARP).
template <class SrcT, class T, int D, int KIND>
__device__ __forceinline__ void src_value(const MapArgs& a, int slot, const MP<T>& m, int j, T& g, T& h) {
  const SrcT* S = reinterpret_cast<const SrcT*>(a.src);
  const long ld = a.src_ld;
  g = ldf<SrcT, T>(S + (long)j * ld + slot);
  h = ldf<SrcT, T>(S + ((long)a.s.nv + j) * ld + slot);
  if (KIND == SRC_BARP) {
    const T* vt = reinterpret_cast<const T*>(a.s.vt);
    T gs, hs;
    model_eval<T, D>(m, vt[j], (D == 2) ? vt[a.s.nv + j] : T(0), T(a.c0), T(a.twoK), gs, hs);
    g = Num<T>::fma(m.c1, Num<T>::sub(gs, g), g);
    h = Num<T>::fma(m.c1, Num<T>::sub(hs, h), h);
  }
}

// Sums over the velocity stripes of the four values of every item of the CTA, in a fixed
// tree order; the results go to mom[off + r][item].
template <int G>
__device__ __forceinline__ void stripe_sums(double v0, double v1, double v2, double v3, double (*red)[256],
                                            double (*mom)[G], int off) {
  constexpr int S = 256 / G;
  const int t = threadIdx.x, s = t / G;
  red[0][t] = v0; red[1][t] = v1; red[2][t] = v2; red[3][t] = v3;
  __syncthreads();
#pragma unroll
  for (int hs = S / 2; hs > 0; hs >>= 1) {
    if (s < hs)
#pragma unroll
      for (int r = 0; r < 4; ++r) red[r][t] += red[r][t + hs * G];
    __syncthreads();
  }
  if (s == 0)
#pragma unroll
    for (int r = 0; r < 4; ++r) mom[off + r][t] = red[r][t];
  __syncthreads();
}

// Projection of item values onto target point i through the CSR table: (g, H = h + |xi|^2 g).
template <class SrcT, class T, int D, int KIND>
__device__ __forceinline__ void project(const MapArgs& a, int slot, const MP<T>& m, int i, T& g, T& H) {
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* wgt = reinterpret_cast<const T*>(a.wgt);
  const int ns = a.s.nv;
  g = T(0);
  H = T(0);
  for (int q = a.off[i]; q < a.off[i + 1]; ++q) {
    const int j = a.idx[q];
    T gj, hj;
    src_value<SrcT, T, D, KIND>(a, slot, m, j, gj, hj);
    const T xj = vs[j], yj = (D == 2) ? vs[ns + j] : T(0);
    g += wgt[q] * gj;
    H += wgt[q] * (hj + (xj * xj + yj * yj) * gj);
  }
}

// Items base .. base + n - 1 (n <= G) of one route, by a CTA of 256 threads: thread t works on
// item t % G over the velocity stripe t / G, so one warp load touches G neighbouring columns in
// each of 32 / G velocity rows (for G = 8 in FP32, one 32-byte sector per row when the items'
// columns are consecutive).
template <class SrcT, class DstT, class T, int D, int KIND, int G>
__device__ __forceinline__ void map_items(const MapArgs& a, int base, int n, double (*red)[256], double (*mom)[G],
                                          double (*coef)[G]) {
  constexpr int S = 256 / G;
  const int t = threadIdx.x, k = t % G, s = t / G;
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* vtt = reinterpret_cast<const T*>(a.t.vt);
  DstT* Dd = reinterpret_cast<DstT*>(a.dst);
  const int ns = a.s.nv, nt = a.t.nv;
  {
    const bool act = k < n;
    const MapItem it = a.items[base + (act ? k : n - 1)];   // idle lanes repeat the last item
    MP<T> m;
    if (KIND == SRC_BARP) m.load(reinterpret_cast<const T*>(a.prm), a.prm_ld, it.prm_slot);
    // 1. target moments over the source space
    KSum<T> r0, r1, r2, r3;
    r0.zero(); r1.zero(); r2.zero(); r3.zero();
    for (int j = s; j < ns; j += S) {
      T g, h;
      src_value<SrcT, T, D, KIND>(a, it.src_slot, m, j, g, h);
      const T x = vs[j], y = (D == 2) ? vs[ns + j] : T(0);
      const T wg = vs[2 * ns + j] * (vs[3 * ns + j] * g);
      const T we = vs[2 * ns + j] * (vs[3 * ns + j] * ((x * x + y * y) * g + h));
      r0.add(wg); r1.add(wg * x); r2.add(wg * y); r3.add(T(0.5) * we);
    }
    stripe_sums<G>(r0.val(), r1.val(), r2.val(), r3.val(), red, mom, 0);
    // 2. projected values on the target space: their moments
    KSum<T> p0, p1, p2, p3;
    p0.zero(); p1.zero(); p2.zero(); p3.zero();
    for (int i = s; i < nt; i += S) {
      T g, H;
      project<SrcT, T, D, KIND>(a, it.src_slot, m, i, g, H);
      const T x = vtt[i], y = (D == 2) ? vtt[nt + i] : T(0);
      const T h = H - (x * x + y * y) * g;
      const T wg = vtt[2 * nt + i] * (vtt[3 * nt + i] * g);
      const T we = vtt[2 * nt + i] * (vtt[3 * nt + i] * ((x * x + y * y) * g + h));
      p0.add(wg); p1.add(wg * x); p2.add(wg * y); p3.add(T(0.5) * we);
    }
    stripe_sums<G>(p0.val(), p1.val(), p2.val(), p3.val(), red, mom, 4);
    // 3. coefficients of the correction, one thread per item
    if (t < G) {
      const double M0 = mom[0][t], M1 = mom[1][t], M2 = mom[2][t], M3 = mom[3][t];
      double RT;
      if (KIND == SRC_FLUX) {
        RT = (double)reinterpret_cast<const T*>(a.prm)[(long)P_RT * a.prm_ld + it.prm_slot];
      } else {
        const double ux = M1 / M0, uy = M2 / M0;
        RT = a.R * (M3 / M0 - 0.5 * (ux * ux + uy * uy)) / a.cv;
      }
      const double cK = a.c0 * RT;
      double d[4] = {M0 - mom[4][t], M1 - mom[5][t], M2 - mom[6][t], M3 - mom[7][t]};
      d[3] -= 0.5 * cK * d[0];
      for (int r = 0; r < 4; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += a.t.ainv[4 * r + c] * d[c];
        coef[r][t] = a.correct ? acc : 0.0;
      }
      coef[4][t] = cK;
    }
    __syncthreads();
    const T a0 = T(coef[0][k]), a1 = T(coef[1][k]), a2 = T(coef[2][k]), a3 = T(coef[3][k]), cK = T(coef[4][k]);
    // 4. write projection + correction
    if (act) {
      for (int i = s; i < nt; i += S) {
        T g, H;
        project<SrcT, T, D, KIND>(a, it.src_slot, m, i, g, H);
        const T x = vtt[i], y = (D == 2) ? vtt[nt + i] : T(0);
        const T x2 = x * x + y * y;
        const T h = H - x2 * g;
        const T dg = a0 + a1 * x + a2 * y + a3 * x2;
        stf<DstT, T>(Dd + (long)i * a.dst_ld + it.dst_slot, g + dg);
        stf<DstT, T>(Dd + ((long)nt + i) * a.dst_ld + it.dst_slot, h + cK * dg);
      }
    }
    __syncthreads();
  }
}

// One route: groups of G items, grid-stride.
template <class SrcT, class DstT, class T, int D, int KIND, int G>
__global__ void __launch_bounds__(256) k_map(const MapArgs a) {
  __shared__ double red[4][256];
  __shared__ double mom[8][G];
  __shared__ double coef[5][G];
  for (int base = blockIdx.x * G; base < a.nitems; base += gridDim.x * G)
    map_items<SrcT, DstT, T, D, KIND, G>(a, base, min(G, a.nitems - base), red, mom, coef);
}

// A group of at most G items of one route.
struct MapWork {
  int route, base, count;
};

// Many routes in one launch: a table of route arguments and a list of item groups.
template <class SrcT, class DstT, class T, int D, int KIND, int G>
__global__ void __launch_bounds__(256) k_map_multi(const MapArgs* __restrict__ routes,
                                                   const MapWork* __restrict__ work, int nwork) {
  __shared__ double red[4][256];
  __shared__ double mom[8][G];
  __shared__ double coef[5][G];
  __shared__ MapArgs sa;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const MapWork wk = work[w];
    if (threadIdx.x == 0) sa = routes[wk.route];
    __syncthreads();
    map_items<SrcT, DstT, T, D, KIND, G>(sa, wk.base, wk.count, red, mom, coef);
  }
}

// Items per CTA for a launch of n items: the largest G whose CTA count still fills the GPU
// (about four CTAs per SM), else one item per CTA.
inline int map_items_per_cta(int n) {
  for (int g : {8, 4, 2})
    if (n / g >= 148 * 4) return g;
  return 1;
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
