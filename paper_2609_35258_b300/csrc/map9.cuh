// Nine-moment mapping of a cell state between velocity spaces (Sec. 3.3.2, Eqs.
// mapping_nine_targets, raw_six_g_basis, raw_three_h_basis, mapping_h_residual_correction):
// the projection phi^p plus a block-triangular additive correction with unit weighting whose
// targets are the source's nine raw moments (rho, rho u, rho v, rho E, G_xx, G_yy, G_xy, J_x,
// J_y; Eqs. source_second_raw_moments, source_energy_flux_moments):
//   g-block: dg = sum_m a_m phi_m, phi = [1, xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y], from the
//            six g-moment defects and A_g = sum w phi phi^T;
//   h-block: dh = sum_m b_m chi_m, chi = [1, xi_x, xi_y], from the defects of (rho E, J_x, J_y)
//            left after dg and A_h = 1/2 sum w chi chi^T.
// One item per call (one thread per item), FP64 sums and solves; the projection comes from the
// CSR table as in the exponential fallback.
#pragma once
#include "expmap.cuh"

namespace mlvs {

// nine raw moments of (g, h) at one point, weighted, added to R
__device__ __forceinline__ void map9_add(double R[9], double w, double x, double y, double g, double h) {
  const double e = h + (x * x + y * y) * g;
  R[0] += w * g; R[1] += w * x * g; R[2] += w * y * g; R[3] += 0.5 * w * e;
  R[4] += w * x * x * g; R[5] += w * y * y * g; R[6] += w * x * y * g;
  R[7] += 0.5 * w * x * e; R[8] += 0.5 * w * y * e;
}

// Maps one item (a column of source kind KIND from space s to space t) with the nine-moment
// correction into dst; returns false if a block is singular (dst then holds the projection).
template <class SrcT, class DstT, class T, int KIND>
__device__ inline bool map9_item(const MapArgs& a, int item) {
  const MapItem it = a.items[item];
  const T* vs = reinterpret_cast<const T*>(a.s.vt);
  const T* vt = reinterpret_cast<const T*>(a.t.vt);
  DstT* dst = reinterpret_cast<DstT*>(a.dst);
  const int ns = a.s.nv, nt = a.t.nv;
  const long dld = a.dst_ld;
  MP<T> m;
  if (KIND == SRC_BARP) m.load(reinterpret_cast<const T*>(a.prm), a.prm_ld, it.prm_slot);
  double tar[9] = {0}, cur[9] = {0};
  for (int j = 0; j < ns; ++j) {
    const double w = (double)vs[2 * ns + j] * (double)vs[3 * ns + j];
    double g, h;
    map_src<SrcT, T, KIND>(a, m, it.src_slot, j, g, h);
    map9_add(tar, w, (double)vs[j], (double)vs[ns + j], g, h);
  }
  double Ag[6][6] = {{0}}, Ah[6][6] = {{0}};
  for (int i = 0; i < nt; ++i) {
    double gp, hp;
    map_project<SrcT, T, KIND>(a, m, it.src_slot, i, gp, hp);
    const double x = (double)vt[i], y = (double)vt[nt + i];
    const double w = (double)vt[2 * nt + i] * (double)vt[3 * nt + i];
    map9_add(cur, w, x, y, gp, hp);
    const double ph[6] = {1.0, x, y, x * x, y * y, x * y};
    for (int r = 0; r < 6; ++r)
      for (int q = 0; q < 6; ++q) Ag[r][q] += w * ph[r] * ph[q];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) Ah[r][q] += 0.5 * w * ph[r] * ph[q];
  }
  // g-block: defects of (rho, rho u, rho v, G_xx, G_yy, G_xy)
  const int gk[6] = {0, 1, 2, 4, 5, 6};
  double ag[6];
  for (int r = 0; r < 6; ++r) ag[r] = tar[gk[r]] - cur[gk[r]];
  bool ok = solve_pivoted<6>(Ag, ag, 6);
  // h-block: defects of (rho E, J_x, J_y) less what dg contributes to them
  double bh[6] = {tar[3] - cur[3], tar[7] - cur[7], tar[8] - cur[8], 0, 0, 0};
  if (ok) {
    for (int i = 0; i < nt; ++i) {
      const double x = (double)vt[i], y = (double)vt[nt + i];
      const double w = (double)vt[2 * nt + i] * (double)vt[3 * nt + i];
      const double dg = ag[0] + ag[1] * x + ag[2] * y + ag[3] * x * x + ag[4] * y * y + ag[5] * x * y;
      const double x2 = x * x + y * y;
      bh[0] -= 0.5 * w * x2 * dg;
      bh[1] -= 0.5 * w * x * x2 * dg;
      bh[2] -= 0.5 * w * y * x2 * dg;
    }
    ok = solve_pivoted<6>(Ah, bh, 3);
  }
  for (int i = 0; i < nt; ++i) {
    double gp, hp;
    map_project<SrcT, T, KIND>(a, m, it.src_slot, i, gp, hp);
    if (ok) {
      const double x = (double)vt[i], y = (double)vt[nt + i];
      gp += ag[0] + ag[1] * x + ag[2] * y + ag[3] * x * x + ag[4] * y * y + ag[5] * x * y;
      hp += bh[0] + bh[1] * x + bh[2] * y;
    }
    stf<DstT, T>(dst + (long)i * dld + it.dst_slot, T(gp));
    stf<DstT, T>(dst + ((long)nt + i) * dld + it.dst_slot, T(hp));
  }
  return ok;
}

// The nine-moment mapping over the items of one route (a level switch, the ghost states of a
// stencil, or the microfluxes of cross-level faces); a singular block sets ERR_SINGULAR in err.
template <class SrcT, class DstT, class T, int KIND>
__global__ void k_map9(const MapArgs a, int* err) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= a.nitems) return;
  if (!map9_item<SrcT, DstT, T, KIND>(a, it)) atomicOr(err, ERR_SINGULAR);
}

}  // namespace mlvs
