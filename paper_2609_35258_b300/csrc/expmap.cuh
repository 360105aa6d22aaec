// Positivity fallback of the state mapping (Sec. 3.3.2): the exponential moment-constrained
// correction of Eq. exponential_moment_correction,
//   phi* = phi^p exp(a . psi),  psi = [1, xi_x, xi_y, |xi|^2 / 2]  (one factor for g and h),
// with a solving the four constraints (rho, rho u, rho v, rho E) of Eq. mapping_four_targets
// (the moments of the source values).  It replaces an additive result that has a negative g
// where the projection phi^p had none.  Damped Newton from a = 0: each step is halved until
// the scaled residual norm decreases; converged when every residual is below 1e-13 of its
// scale max(|target|, 1e-3 max |target|).  All sums and the factor are FP64.
//
// One item per call (one thread per item): the projection of the source column onto every
// target point is recomputed from the CSR table in each residual evaluation, so the pass
// needs no scratch memory; it is a fallback for the items that need it.  The source values
// are the stored phi~ (a level switch) or phi-bar-plus formed as k_map forms it (SRC_BARP).
#pragma once
#include "finalize.cuh"
#include "mapping.cuh"

namespace mlvs {

enum { EXPMAP_KEPT = 0, EXPMAP_REPLACED = 1, EXPMAP_FAILED = 2 };

// Source value j of an item in FP64: the stored value, or for SRC_BARP phi-bar-plus formed from
// phi~ and the cell's parameters m (as k_map forms it).
template <class SrcT, class T, int KIND>
__device__ __forceinline__ void map_src(const MapArgs& a, const MP<T>& m, int slot, int j, double& g, double& h) {
  T gt, ht;
  src_value<SrcT, T, 2, KIND>(a, slot, m, j, gt, ht);
  g = (double)gt;
  h = (double)ht;
}

// Projection of the item's source values onto target point i (coarsening averages g and
// H = h + |xi|^2 g with the CSR weights, refinement inherits them; h = H - |xi_t|^2 g).
template <class SrcT, class T, int KIND>
__device__ inline void map_project(const MapArgs& a, const MP<T>& m, int slot, int i, double& g, double& h) {
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* vt = reinterpret_cast<const T*>(a.t.vt);
  const T* wgt = reinterpret_cast<const T*>(a.wgt);
  const int ns = a.s.nv, nt = a.t.nv;
  double G = 0.0, H = 0.0;
  for (int q = a.off[i]; q < a.off[i + 1]; ++q) {
    const int j = a.idx[q];
    double gj, hj;
    map_src<SrcT, T, KIND>(a, m, slot, j, gj, hj);
    const double xj = (double)vs[j], yj = (double)vs[ns + j];
    G += (double)wgt[q] * gj;
    H += (double)wgt[q] * (hj + (xj * xj + yj * yj) * gj);
  }
  const double xi = (double)vt[i], yi = (double)vt[nt + i];
  g = G;
  h = H - (xi * xi + yi * yi) * G;
}

// Residuals F_k = sum_i w_i kern_k(i) e_i - tar_k of the factor exp(a . psi), and with J the
// Jacobian J_km = sum_i w_i kern_k(i) e_i psi_m(i).
template <class SrcT, class T, int KIND>
__device__ inline void expmap_residual(const MapArgs& a, const MP<T>& mp, int slot, const double c[4],
                                       const double tar[4], double F[4], double (*J)[4]) {
  const T* vt = reinterpret_cast<const T*>(a.t.vt);
  const int nt = a.t.nv;
  double acc[4] = {0, 0, 0, 0}, jac[4][4] = {{0}};
  for (int i = 0; i < nt; ++i) {
    double gp, hp;
    map_project<SrcT, T, KIND>(a, mp, slot, i, gp, hp);
    const double x = (double)vt[i], y = (double)vt[nt + i];
    const double w = (double)vt[2 * nt + i] * (double)vt[3 * nt + i];
    const double psi[4] = {1.0, x, y, 0.5 * (x * x + y * y)};
    const double e = exp(c[0] + c[1] * x + c[2] * y + c[3] * psi[3]);
    const double k[4] = {gp, x * gp, y * gp, 0.5 * ((x * x + y * y) * gp + hp)};
    for (int r = 0; r < 4; ++r) {
      acc[r] += w * k[r] * e;
      if (J)
        for (int m = 0; m < 4; ++m) jac[r][m] += w * k[r] * e * psi[m];
    }
  }
  for (int r = 0; r < 4; ++r) {
    F[r] = acc[r] - tar[r];
    if (J)
      for (int m = 0; m < 4; ++m) J[r][m] = jac[r][m];
  }
}

// The fallback for one item (a level switch, or a ghost state with KIND = SRC_BARP): the
// additive result in dst is kept unless it has a negative g where the projection has none.
template <class SrcT, class DstT, class T, int KIND>
__device__ inline int expmap_item(const MapArgs& a, int item) {
  const MapItem it = a.items[item];
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* vt = reinterpret_cast<const T*>(a.t.vt);
  DstT* dst = reinterpret_cast<DstT*>(a.dst);
  const int ns = a.s.nv, nt = a.t.nv;
  const long dld = a.dst_ld;
  MP<T> mp;
  if (KIND == SRC_BARP) mp.load(reinterpret_cast<const T*>(a.prm), a.prm_ld, it.prm_slot);
  bool neg = false, proj_neg = false;
  for (int i = 0; i < nt && !proj_neg; ++i) {
    if ((double)ldf<DstT, T>(dst + (long)i * dld + it.dst_slot) < 0.0) neg = true;
    double gp, hp;
    map_project<SrcT, T, KIND>(a, mp, it.src_slot, i, gp, hp);
    if (gp < 0.0) proj_neg = true;
  }
  if (!neg || proj_neg) return EXPMAP_KEPT;
  // targets: the source moments (rho, rho u, rho v, rho E)
  double tar[4] = {0, 0, 0, 0};
  for (int j = 0; j < ns; ++j) {
    double g, h;
    map_src<SrcT, T, KIND>(a, mp, it.src_slot, j, g, h);
    const double x = (double)vs[j], y = (double)vs[ns + j];
    const double w = (double)vs[2 * ns + j] * (double)vs[3 * ns + j];
    tar[0] += w * g;
    tar[1] += w * x * g;
    tar[2] += w * y * g;
    tar[3] += 0.5 * w * ((x * x + y * y) * g + h);
  }
  double big = 0.0;
  for (int r = 0; r < 4; ++r) big = fmax(big, fabs(tar[r]));
  double scale[4];
  for (int r = 0; r < 4; ++r) scale[r] = fmax(fabs(tar[r]), 1e-3 * big);
  auto norm = [&](const double F[4]) {
    double s = 0.0;
    for (int r = 0; r < 4; ++r) s += (F[r] / scale[r]) * (F[r] / scale[r]);
    return sqrt(s);
  };
  auto done = [&](const double F[4]) {
    for (int r = 0; r < 4; ++r)
      if (!(fabs(F[r]) / scale[r] < 1e-13)) return false;
    return true;
  };
  double c[4] = {0, 0, 0, 0}, F[4], J[4][4];
  expmap_residual<SrcT, T, KIND>(a, mp, it.src_slot, c, tar, F, J);
  bool ok = done(F);
  for (int iter = 0; iter < 60 && !ok; ++iter) {
    double M[4][4], d[4];
    for (int r = 0; r < 4; ++r) {
      d[r] = -F[r];
      for (int m = 0; m < 4; ++m) M[r][m] = J[r][m];
    }
    const int idx[4] = {0, 1, 2, 3};
    if (!solve_small(M, d, idx, 4)) return EXPMAP_FAILED;
    double t = 1.0, c1[4], F1[4];
    const double n0 = norm(F);
    for (;;) {
      for (int r = 0; r < 4; ++r) c1[r] = c[r] + t * d[r];
      expmap_residual<SrcT, T, KIND>(a, mp, it.src_slot, c1, tar, F1, nullptr);
      if (norm(F1) < n0 || t < 1e-8) break;
      t *= 0.5;
    }
    for (int r = 0; r < 4; ++r) c[r] = c1[r];
    expmap_residual<SrcT, T, KIND>(a, mp, it.src_slot, c, tar, F, J);
    ok = done(F);
  }
  if (!ok) return EXPMAP_FAILED;
  for (int i = 0; i < nt; ++i) {
    double gp, hp;
    map_project<SrcT, T, KIND>(a, mp, it.src_slot, i, gp, hp);
    const double x = (double)vt[i], y = (double)vt[nt + i];
    const double e = exp(c[0] + c[1] * x + c[2] * y + c[3] * 0.5 * (x * x + y * y));
    stf<DstT, T>(dst + (long)i * dld + it.dst_slot, T(gp * e));
    stf<DstT, T>(dst + ((long)nt + i) * dld + it.dst_slot, T(hp * e));
  }
  return EXPMAP_REPLACED;
}

// The fallback over the items of one route; counts (may be null): counts[0] += replaced
// items, counts[1] += items whose iteration did not converge.
template <class SrcT, class DstT, class T, int KIND>
__global__ void k_expmap(const MapArgs a, int* counts) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= a.nitems) return;
  const int r = expmap_item<SrcT, DstT, T, KIND>(a, it);
  if (counts && r == EXPMAP_REPLACED) atomicAdd(counts, 1);
  if (counts && r == EXPMAP_FAILED) atomicAdd(counts + 1, 1);
}

}  // namespace mlvs
