// Point finalisation: from velocity-chunk partial moments to the model parameters of a cell
// or a face, including the four-moment compatibility correction (Sec. 3.3.1).
//
// One thread per point.  The chunk partials are summed in chunk order (deterministic); the
// macroscopic state follows Eq. discrete_W / discrete_q (cells) or Eq. W_from_bar (faces).
//
// Compatibility correction (Eq. gh_model_correction, chi^g = g^S, chi^h = h^S).  The basis
// {1, xi_x, xi_y, E_xi} of Eq. eq_four_basis spans the same functions as {1, c_x, c_y, |c|^2}
// with c = xi - u, and the constraint rows (1, xi, (xi^2 g + h)/2) combine into the peculiar
// rows (1, c, (|c|^2 g + h)/2) with targets (rho, rho(u - u_p), rho e + rho|u - u_p|^2/2), u_p
// the velocity stored in the parameters.  The corrected distribution is therefore the same
// as with the paper's basis.  The sums of Eq. joint_gh_correction_matrix and
// Eq. linear_moment_defect are evaluated
//   * on tensor-product spaces, from one-axis sums S_a = sum_i W_i e_i c_i^a (a <= 7) of the
//     same per-axis Gaussian factors e_i that the tile kernels multiply (Num::gauss), so
//     sum_{ij} W_i W_j e_i e_j c_x^a c_y^b = S_a S_b and the correction matches the values
//     the tile kernels evaluate up to the rounding of their own products;
//   * otherwise, directly over the velocities with the tile kernels' model_eval.
// Sums that enter the moment defect are compensated (FP32) and combined in FP64.
//
// On spaces that are not tensor products the direct sums run over every velocity of the
// point; there a warp serves one point (LANES = 32): each lane sums a strided share of the
// velocities and the shares are combined by an xor butterfly, which leaves the same bits in
// every lane.
#pragma once
#include "mlvs_common.cuh"

namespace mlvs {

struct GasDev {
  double R, K, Pr, omega, mu_ref, T_ref;
};

struct PointArgs {
  StepConst k;
  GasDev gas;
  const double* part;   // [nchunk][NMOM][npt]
  const double* msum;   // [NMOM][npt] the chunk sums of part (k_sum_chunks), or null
  int npt;              // number of points (the stride of every per-point array)
  const int* pts;       // the points to finalise (faces a level evaluates), or null: 0..npt-1
  int nwork;            // number of points to finalise (length of pts, else npt)
  int is_face;          // 0: cells, 1: faces
  const void* cprm;     // [NP][ncell] current cell params (T): shift source
  void* prm_out;        // [NP][npt] (T)
  double* W;            // cells: [11][ncell] rho,u,v,T,qx,qy,rhoE,tau,sxx,sxy,syy (null for faces)
  const void* vt;       // [4][nv] (T)
  const void* ax;       // [2][nax] (T) when k.nax > 0
  const int* ids;       // cells: global cell id of every point (null: identity)
  const unsigned char* frole;  // faces: role on this level (null: every face)
  const void* ucell;    // faces: (T) [2][ncell] cell velocities for the moment shift
  int compat;
  double wall[4][3];    // (u_w, v_w, T_w)
  double far[4];        // freestream (rho, u, v, T)
  int* err;             // device error bits
  const double* wden;   // curvilinear walls: [nface] normalisation of the wall Maxwellian (or null)
  double* scr;          // split finalisation: [FIN_SCR][npt] state and velocity sums
  int* need;            // split finalisation: [npt] what the velocity sums are for
  // rows of a 2-D space that is not a tensor product (null: the direct sums): the distinct
  // axis ranges of its points (entries, grouped by level: block L = [lst[L], lst[L+1])), the
  // rows (points sharing a y entry: {y entry, first segment, segments, 0}) and the segments of
  // a row (runs of consecutive x entries of one level, as prefix positions {e0 + L, e1 + L})
  const void* e1;       // (T) [2][n1] entry abscissa X and weight W
  int n1;
  const int* lst;       // [5]
  const int4* rows;
  int nrows;
  const int2* segs;
  // the eight-moment correction (2-D, tensor-product spaces, one thread per point): b4..b7 of
  // every point into prm8_out [4][npt] (T; zeros where the four-moment correction or none
  // applies); null: the four-moment correction
  void* prm8_out;
};

// Split finalisation: k_fin_pre (thread per point: state, uncorrected model), k_fin_sums (warp
// per point: the velocity sums, or on tensor-product spaces the one-axis sums), k_fin_post
// (thread per point: correction).  k_finalize does all three in one thread per point.  Scratch rows: rho ux uy T, then G[5][5], H[3][3], den.
enum { FS_RHO = 0, FS_UX, FS_UY, FS_T, FS_G = 4, FS_H = 29, FS_DEN = 38, FIN_SCR = 39 };
// the eight-moment correction on the split path: heat-flux target, G[7][7] and H[5][5]
enum { FS_QX = 39, FS_QY = 40, FS_G8 = 41, FS_H8 = 90, FIN_SCR8 = 115 };

enum { ERR_NONFINITE = 1, ERR_POSITIVITY = 2, ERR_SINGULAR = 4 };

// The device error word and, behind it, the first failing point of a finalisation:
//   int [0] error bits, [1] claim, [2] point index, [3] 1 for a face; double [2] rho, T.
constexpr int ERR_WORDS = 8;   // ints (the two doubles start at int 4)

// Record a failing point state: the error bit, and the first such point with its density and
// temperature (the host adds them to the error message).
__device__ __forceinline__ void report_point(int* err, int bit, int i, int is_face, double rho, double Tm) {
  atomicOr(err, bit);
  if (atomicCAS(err + 1, 0, 1) == 0) {
    err[2] = i;
    err[3] = is_face;
    double* d = reinterpret_cast<double*>(err + 4);
    d[0] = rho;
    d[1] = Tm;
  }
}

// Sum over the LANES lanes of a warp segment (all lanes receive the same value).
template <int LANES>
__device__ __forceinline__ double lane_sum(double x) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Gaussian elimination with partial pivoting on the rows/columns listed in idx.
__device__ inline bool solve_small(double A[4][4], double b[4], const int* idx, int n) {
  double M[4][4], r[4];
  for (int i = 0; i < n; ++i) {
    r[i] = b[idx[i]];
    for (int j = 0; j < n; ++j) M[i][j] = A[idx[i]][idx[j]];
  }
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(M[c][c]);
    for (int q = c + 1; q < n; ++q)
      if (fabs(M[q][c]) > best) { best = fabs(M[q][c]); p = q; }
    if (!(best > 1e-300)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) { double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
      double t = r[c]; r[c] = r[p]; r[p] = t;
    }
    for (int q = c + 1; q < n; ++q) {
      const double f = M[q][c] / M[c][c];
      for (int j = c; j < n; ++j) M[q][j] -= f * M[c][j];
      r[q] -= f * r[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = r[c];
    for (int j = c + 1; j < n; ++j) s -= M[c][j] * r[j];
    r[c] = s / M[c][c];
  }
  for (int i = 0; i < 4; ++i) b[i] = 0.0;
  for (int i = 0; i < n; ++i) b[idx[i]] = r[i];
  return true;
}

// Gaussian elimination with partial pivoting on the leading n x n block of M (row stride N),
// in place; b receives the solution.  Returns false on a zero pivot.
template <int N>
__device__ inline bool solve_pivoted(double (*M)[N], double* b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(M[c][c]);
    for (int q = c + 1; q < n; ++q)
      if (fabs(M[q][c]) > best) { best = fabs(M[q][c]); p = q; }
    if (!(best > 1e-300)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) { const double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
      const double t = b[c]; b[c] = b[p]; b[p] = t;
    }
    for (int q = c + 1; q < n; ++q) {
      const double f = M[q][c] / M[c][c];
      for (int j = c; j < n; ++j) M[q][j] -= f * M[c][j];
      b[q] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int j = c + 1; j < n; ++j) s -= M[c][j] * b[j];
    b[c] = s / M[c][c];
  }
  return true;
}

// One-axis sums S[a] = sum_i W_i gauss(X_i - u) (X_i - u)^a, a = 0..7.
template <class T>
__device__ inline void axis_sums(const T* ax, int nax, T u, T inv2RT, T lnh, double S[8]) {
  KSum<T> acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a].zero();
  for (int i = 0; i < nax; ++i) {
    const T c = ax[i] - u;
    T p = ax[nax + i] * Num<T>::gauss(c, inv2RT, lnh);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      acc[a].add(p);
      p *= c;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) S[a] = acc[a].val();
}

// A compensated sum merged over the LANES lanes of a warp segment (xor butterfly): each merge
// keeps its own rounding error exactly (TwoSum) in the compensation, and every lane receives
// the same value.  FP64 sums carry no compensation and are added directly.
template <int LANES, class T>
__device__ __forceinline__ double ksum_lanes(const KSum<T>& k) {
  if constexpr (sizeof(T) == 8) {
    double x = k.val();
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  } else {
    T s = k.s, c = k.c;
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
      const T so = __shfl_xor_sync(0xffffffffu, s, o), co = __shfl_xor_sync(0xffffffffu, c, o);
      const T t = s + so;
      const T bb = t - s;
      const T e = (s - (t - bb)) + (so - bb);   // t + e = s + so exactly
      c = (c + co) - e;
      s = t;
    }
    return (double)s - (double)c;
  }
}

// axis_sums split over the LANES lanes of a warp segment: lane j takes the points j, j + LANES,
// ...; every lane receives S.
template <class T, int LANES>
__device__ inline void axis_sums_lanes(const T* ax, int nax, T u, T inv2RT, T lnh, int lane, double S[8]) {
  KSum<T> acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a].zero();
  for (int i = lane; i < nax; i += LANES) {
    const T c = ax[i] - u;
    T p = ax[nax + i] * Num<T>::gauss(c, inv2RT, lnh);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      acc[a].add(p);
      p *= c;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) S[a] = ksum_lanes<LANES, T>(acc[a]);
}

// Sum over the LANES lanes of a warp segment in the compute type (all lanes receive it).
template <int LANES, class T>
__device__ __forceinline__ T lane_sum_t(T x) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Peculiar moments of the uncorrected model of mp:
//   G[a][b] = sum w g^S c_x^a c_y^b (a+b <= 4),  H[a][b] = sum w h^S c_x^a c_y^b (a+b <= 2),
// on a tensor-product space from the one-axis sums.
// G and H of the uncorrected model from its pair moments P[i][j] = sum w gauss c_x^i c_y^j
// (i + j <= 7; on a tensor-product space P[i][j] = Sx[i] Sy[j]).
template <class T, int D>
__device__ inline void pair_combine(const PointArgs& A, const MP<T>& mp, const double P[8][8], double G[5][5],
                                    double H[3][3]) {
  const StepConst& k = A.k;
  const double kx = (double)mp.kqx, ky = (double)mp.kqy;
  const double i2 = 2.0 * (double)mp.inv2RT;      // 1/RT as the tile kernels form it
  const double RT = (double)mp.RT, c0 = k.c0;
  const double al = RT * c0 * i2, be = RT * (D * c0 + k.twoK);
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) G[a][b] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = 0.0;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; a + b < 5; ++b) {
      const double cub = kx * (P[a + 3][b] + P[a + 1][b + 2]) + ky * (P[a + 2][b + 1] + P[a][b + 3]);
      const double lin = kx * P[a + 1][b] + ky * P[a][b + 1];
      G[a][b] = P[a][b] - (D + 2) * lin + i2 * cub;
      if (a + b < 3) H[a][b] = RT * c0 * P[a][b] + al * cub - be * lin;
    }
}

template <class T, int D>
__device__ inline void axis_combine(const PointArgs& A, const MP<T>& mp, const double Sx[8], const double Sy[8],
                                    double G[5][5], double H[3][3]) {
  double P[8][8];
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) P[i][j] = (i + j <= 7) ? Sx[i] * Sy[j] : 0.0;
  pair_combine<T, D>(A, mp, P, G, H);
}

template <class T, int D>
__device__ inline void axis_moments(const PointArgs& A, const MP<T>& mp, double G[5][5], double H[3][3]) {
  const StepConst& k = A.k;
  const T* ax = reinterpret_cast<const T*>(A.ax);
  double Sx[8], Sy[8];
  axis_sums<T>(ax, k.nax, mp.ux, mp.inv2RT, mp.lnh, Sx);
  if (D == 2) {
    axis_sums<T>(ax, k.nax, mp.uy, mp.inv2RT, mp.lnh, Sy);
  } else {
    Sy[0] = 1.0;
    for (int b = 1; b < 8; ++b) Sy[b] = 0.0;
  }
  axis_combine<T, D>(A, mp, Sx, Sy, G, H);
}

// The same moments summed directly over the velocities, two at a time: lane `lane` of LANES
// takes the velocity pairs (v, v+1), v = 2 (lane + j LANES), in packed two-lane arithmetic (a
// pair past the last velocity has a zero-weight lane), and the lanes are combined at the end
// (compensated sums in FP64, the others in the compute type).
template <class T, int D, int LANES>
__device__ inline void direct_moments(const PointArgs& A, const MP<T>& mp, int lane, double G[5][5],
                                      double H[3][3]) {
  using P = Pk<T>;
  using V = V2<T>;
  const StepConst& k = A.k;
  const T* vt = reinterpret_cast<const T*>(A.vt);
  const int nv = k.nv;
  const T c0 = T(k.c0), twoK = T(k.twoK);
  // packed Kahan pairs (s, c) of the four conserved rows
  V ks[4], kc[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) ks[r] = kc[r] = P::splat(T(0));
  V gs[15], hs[6];
#pragma unroll
  for (int j = 0; j < 15; ++j) gs[j] = P::splat(T(0));
#pragma unroll
  for (int j = 0; j < 6; ++j) hs[j] = P::splat(T(0));
  const V ux = P::splat(mp.ux), uy = P::splat(mp.uy);
  for (int v = 2 * lane; v < nv; v += 2 * LANES) {
    const int v2 = v + 1 < nv ? v + 1 : v;
    const T on = v + 1 < nv ? T(1) : T(0);
    const V xx = P::mk(vt[v], vt[v2]);
    const V yy = (D == 2) ? P::mk(vt[nv + v], vt[nv + v2]) : P::splat(T(0));
    const V wxv = P::mk(vt[2 * nv + v], on * vt[2 * nv + v2]);
    const V wyv = P::mk(vt[3 * nv + v], vt[3 * nv + v2]);
    V gv, hv;
    model_eval2<T, D>(mp, xx, yy, c0, twoK, gv, hv);
    const V cx = P::sub(xx, ux), cy = (D == 2) ? P::sub(yy, uy) : P::splat(T(0));
    const V wg = P::mul(wxv, P::mul(wyv, gv)), wh = P::mul(wxv, P::mul(wyv, hv));
    const V x4[4] = {wg, P::mul(wg, cx), P::mul(wg, cy),
                     P::mul(P::splat(T(0.5)), P::fma(P::fma(cy, cy, P::mul(cx, cx)), wg, wh))};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const V y = P::sub(x4[r], kc[r]);
      const V t = P::add(ks[r], y);
      kc[r] = P::sub(P::sub(t, ks[r]), y);
      ks[r] = t;
    }
    int j = 0, jh = 0;
    V px = wg, qx = wh;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      V pp = px, q = qx;
#pragma unroll
      for (int b = 0; a + b < 5; ++b) {
        gs[j] = P::add(gs[j], pp);
        ++j;
        if (a + b < 3) { hs[jh] = P::add(hs[jh], q); ++jh; }
        pp = P::mul(pp, cy);
        q = P::mul(q, cy);
      }
      px = P::mul(px, cx);
      qx = P::mul(qx, cx);
    }
  }
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) G[a][b] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = 0.0;
  int j = 0, jh = 0;
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; a + b < 5; ++b) {
      G[a][b] = (double)lane_sum_t<LANES, T>(gs[j].x + gs[j].y);
      ++j;
      if (a + b < 3) {
        H[a][b] = (double)lane_sum_t<LANES, T>(hs[jh].x + hs[jh].y);
        ++jh;
      }
    }
  double kv[4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    kv[r] = lane_sum<LANES>(((double)ks[r].x - (double)kc[r].x) + ((double)ks[r].y - (double)kc[r].y));
  G[0][0] = kv[0];
  G[1][0] = kv[1];
  G[0][1] = kv[2];
  // keep the compensated energy-row sum: fold it into the H[0][0] slot
  H[0][0] = 2.0 * kv[3] - G[2][0] - G[0][2];
}

// Compensated sum helpers (value s - c; FP64 sums carry no compensation).
template <class T> __device__ __forceinline__ void csum_add(T& s, T& c, T x) {
  if constexpr (sizeof(T) == 8) {
    s += x;
  } else {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
}
// (s, c) = (so, co) + (s, c), the rounding error of the sum kept exactly (TwoSum)
template <class T> __device__ __forceinline__ void csum_merge(T& s, T& c, T so, T co) {
  if constexpr (sizeof(T) == 8) {
    s += so;
  } else {
    const T t = so + s;
    const T bb = t - so;
    const T e = (so - (t - bb)) + (s - bb);
    c = (co + c) - e;
    s = t;
  }
}

// Shared-memory values (type T) a warp needs for row_moments<T, NO> on a space with n1
// entries: the prefix sums [NO + 3][n1 + 4] (NO orders, three of them compensated); the same
// area later holds the lanes' pair moments (NE = NO (NO + 1) / 2 rows of 33, the row padded so
// that a lane reading its row meets no other lane's bank) and then the NE sums as FP64 at the
// even offset row_pd(NO).  The count is rounded up to an even number, so that every warp's
// area, and with it the FP64 sums, starts on an 8-byte boundary.
__host__ __device__ constexpr int row_pd(int NO) { return ((NO * (NO + 1) / 2) * 33 + 1) & ~1; }
__host__ __device__ inline int row_smem_values(int n1, int NO = 8) {
  const int q = (NO + 3) * (n1 + 4), r = row_pd(NO) + NO * (NO + 1);
  return ((q > r ? q : r) + 1) & ~1;
}

// The pair moments P[i][j] = sum over the space of w gauss(c_x) gauss(c_y) c_x^i c_y^j
// (i + j < NO) of a 2-D space that is not a tensor product, from its rows, by one warp.  For
// every entry e (a distinct axis range, abscissa X_e, weight W_e) the factor W_e gauss(X_e - u_x)
// (X_e - u_x)^i is summed into prefix sums per level block of entries (compensated for the
// orders 0..2 that the conserved rows take; the block's entries split into one contiguous run
// per lane, the runs joined by a warp scan), so that a row's x sums are differences of prefix
// sums over its segments; a row's y factor is one Gaussian.  P = sum over rows of Rx[i] Ry[j],
// summed per lane and then over the lanes (compensated, four interleaved chains per entry):
// entry k (i-major, i + j < NO) as an FP64 value at wsm + row_pd(NO), for every lane to read.
// wsm: row_smem_values(n1, NO) values of this warp.
template <class T, int NO = 8>
__device__ inline void row_moments(const PointArgs& A, const MP<T>& mp, int lane, T* wsm) {
  constexpr int NE = NO * (NO + 1) / 2;
  const T* e1 = reinterpret_cast<const T*>(A.e1);
  const int n1 = A.n1, nq = n1 + 4;
  T* Qs = wsm;             // [NO][nq] prefix sums (s)
  T* Qc = wsm + NO * nq;   // [3][nq] their compensation (c), orders 0..2
  for (int L = 0; L < 4; ++L) {
    const int ls = A.lst[L], n = A.lst[L + 1] - ls;
    if (n == 0) continue;
    const int cs = (n + 31) / 32;
    const int i0 = ls + min(n, lane * cs), i1 = ls + min(n, (lane + 1) * cs);
    T s[NO], c[NO];
#pragma unroll
    for (int a = 0; a < NO; ++a) s[a] = c[a] = T(0);
    for (int e = i0; e < i1; ++e) {
      const T x = e1[e] - mp.ux;
      T p = e1[n1 + e] * Num<T>::gauss(x, mp.inv2RT, mp.lnh);
#pragma unroll
      for (int a = 0; a < NO; ++a) {
        if (a < 3) csum_add(s[a], c[a], p);
        else s[a] += p;
        p *= x;
      }
    }
    // exclusive scan over the lanes: the start of every lane's run
#pragma unroll
    for (int a = 0; a < NO; ++a) {
      T ss = s[a], cc = c[a];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T so = __shfl_up_sync(0xffffffffu, ss, o);
        if (a < 3) {
          const T co = __shfl_up_sync(0xffffffffu, cc, o);
          if (lane >= o) csum_merge(ss, cc, so, co);
        } else if (lane >= o) {
          ss += so;
        }
      }
      T xs = __shfl_up_sync(0xffffffffu, ss, 1), xc = T(0);
      if (a < 3) xc = __shfl_up_sync(0xffffffffu, cc, 1);
      if (lane == 0) xs = xc = T(0);
      s[a] = xs;
      c[a] = xc;
    }
    if (lane == 0)
#pragma unroll
      for (int a = 0; a < NO; ++a) {
        Qs[a * nq + ls + L] = T(0);
        if (a < 3) Qc[a * nq + ls + L] = T(0);
      }
    for (int e = i0; e < i1; ++e) {
      const T x = e1[e] - mp.ux;
      T p = e1[n1 + e] * Num<T>::gauss(x, mp.inv2RT, mp.lnh);
#pragma unroll
      for (int a = 0; a < NO; ++a) {
        if (a < 3) {
          csum_add(s[a], c[a], p);
          Qc[a * nq + e + L + 1] = c[a];
        } else {
          s[a] += p;
        }
        Qs[a * nq + e + L + 1] = s[a];
        p *= x;
      }
    }
  }
  __syncwarp();
  // rows: Rx from the segments, Ry from the row's y entry; the first-order entries compensated
  T M[NE], Mc[3];
#pragma unroll
  for (int k = 0; k < NE; ++k) M[k] = T(0);
  Mc[0] = Mc[1] = Mc[2] = T(0);
  for (int r = lane; r < A.nrows; r += 32) {
    const int4 R = A.rows[r];
    const T y = e1[R.x] - mp.uy;
    T py = e1[n1 + R.x] * Num<T>::gauss(y, mp.inv2RT, mp.lnh);
    T Ry[NO], Rs[NO], Rc[3];
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      Ry[b] = py;
      py *= y;
      Rs[b] = T(0);
      if (b < 3) Rc[b] = T(0);
    }
    for (int sg = R.y; sg < R.y + R.z; ++sg) {
      const int2 q = A.segs[sg];
#pragma unroll
      for (int a = 0; a < NO; ++a) {
        Rs[a] += Qs[a * nq + q.y] - Qs[a * nq + q.x];
        if (a < 3) Rc[a] += Qc[a * nq + q.y] - Qc[a * nq + q.x];
      }
    }
    int k = 0;
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; i + j < NO; ++j, ++k) {
        const T v = (i < 3 ? Rs[i] - Rc[i] : Rs[i]) * Ry[j];
        if (k == 0 || k == 1 || k == NO) csum_add(M[k], Mc[k == 0 ? 0 : (k == 1 ? 1 : 2)], v);
        else M[k] += v;
      }
  }
  __syncwarp();
  // over the lanes: through shared memory, one entry per lane (compensated)
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const T cm = (k == 0) ? Mc[0] : (k == 1) ? Mc[1] : (k == NO) ? Mc[2] : T(0);
    wsm[k * 33 + lane] = M[k] - cm;
  }
  __syncwarp();
  double* Pd = reinterpret_cast<double*>(wsm + row_pd(NO));
  for (int k = lane; k < NE; k += 32) {
    T as[4], ac[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) as[j] = ac[j] = T(0);
#pragma unroll
    for (int l = 0; l < 32; l += 4)
#pragma unroll
      for (int j = 0; j < 4; ++j) csum_add(as[j], ac[j], wsm[k * 33 + l + j]);
    csum_merge(as[0], ac[0], as[1], ac[1]);
    csum_merge(as[2], ac[2], as[3], ac[3]);
    csum_merge(as[0], ac[0], as[2], ac[2]);
    Pd[k] = (double)as[0] - (double)ac[0];
  }
  __syncwarp();
}

// The G and H entries of pair_combine from row_moments' pair moments, one entry per lane (FP64
// work spread over the warp), stored to the split finalisation's scratch of point i: lane l <
// 25 writes G slot l, lanes 25..31 H slots 0..6, lanes 0 and 1 also H slots 7 and 8.
template <class T, int D>
__device__ inline void row_store_gh(const PointArgs& A, const MP<T>& mp, int lane, const T* wsm, long i) {
  const double* Pd = reinterpret_cast<const double*>(wsm + row_pd(8));
  auto P = [&](int a, int b) -> double { return Pd[8 * a - a * (a - 1) / 2 + b]; };
  const StepConst& k = A.k;
  const double kx = (double)mp.kqx, ky = (double)mp.kqy;
  const double i2 = 2.0 * (double)mp.inv2RT;
  const double RT = (double)mp.RT, c0 = k.c0;
  const double al = RT * c0 * i2, be = RT * (D * c0 + k.twoK);
  const long n = A.npt;
  auto entry = [&](int a, int b, bool h) -> double {
    if (a + b > (h ? 2 : 4)) return 0.0;
    const double cub = kx * (P(a + 3, b) + P(a + 1, b + 2)) + ky * (P(a + 2, b + 1) + P(a, b + 3));
    const double lin = kx * P(a + 1, b) + ky * P(a, b + 1);
    return h ? RT * c0 * P(a, b) + al * cub - be * lin : P(a, b) - (D + 2) * lin + i2 * cub;
  };
  if (lane < 25) A.scr[(FS_G + lane) * n + i] = entry(lane / 5, lane % 5, false);
  else A.scr[(FS_H + lane - 25) * n + i] = entry((lane - 25) / 3, (lane - 25) % 3, true);
  if (lane < 2) A.scr[(FS_H + 7 + lane) * n + i] = 0.0;
}

// ---- eight-moment compatibility correction (Sec. 3.3.1, Eq. eq_eight_basis) ----
// The correction factor 1 + sum_m b_m phi_m uses the basis, in peculiar velocity c = xi - u,
//   {1, c_x, c_y, |c|^2, |c|^2 c_x, |c|^2 c_y, c_x^2 - c_y^2, c_x c_y},
// the span of Eq. eq_eight_basis {1, xi_x, xi_y, E_xi, E_c c_x, E_c c_y, c_x^2 - c_y^2, c_x c_y}.
// The constraint rows are (g, c g, (|c|^2 g + h)/2, (|c|^2 g + h) c / 2, (c_x^2 - c_y^2) g,
// c_x c_y g) with targets (rho, rho (u - u_p), rho e + rho |u - u_p|^2 / 2, q^tar, 0, 0), u_p the
// velocity of the parameters: the conserved rows combine the paper's, and the heat-flux and
// stress rows are the paper's about u (u_p = u up to the rounding of the stored velocity).

// one-axis sums S[a] = sum_i W_i gauss(X_i - u) (X_i - u)^a, a = 0..9
template <class T>
__device__ inline void u_axis_sums10(const T* ax, int nax, T u, T inv2RT, T lnh, double S[10]) {
  KSum<T> acc[10];
  for (int k = 0; k < 10; ++k) acc[k].zero();
  for (int i = 0; i < nax; ++i) {
    const T c = ax[i] - u;
    T p = ax[nax + i] * Num<T>::gauss(c, inv2RT, lnh);
    for (int k = 0; k < 10; ++k) {
      acc[k].add(p);
      p *= c;
    }
  }
  for (int k = 0; k < 10; ++k) S[k] = acc[k].val();
}

// peculiar moments of the uncorrected Shakhov model on the tensor-product space:
//   G[a][b] = sum w g^S c_x^a c_y^b (a + b <= 6),  H[a][b] = sum w h^S c_x^a c_y^b (a + b <= 4)
template <class T>
__device__ inline void u_moments8(const PointArgs& A, const MP<T>& mp, double G[7][7], double H[5][5]) {
  const T* ax = reinterpret_cast<const T*>(A.ax);
  double Sx[10], Sy[10];
  u_axis_sums10<T>(ax, A.k.nax, mp.ux, mp.inv2RT, mp.lnh, Sx);
  u_axis_sums10<T>(ax, A.k.nax, mp.uy, mp.inv2RT, mp.lnh, Sy);
  const double kx = (double)mp.kqx, ky = (double)mp.kqy;
  const double i2 = 2.0 * (double)mp.inv2RT, RT = (double)mp.RT, c0 = A.k.c0;
  const double al = RT * c0 * i2, be = RT * (2.0 * c0 + A.k.twoK);
  for (int x = 0; x < 7; ++x)
    for (int y = 0; y < 7; ++y) G[x][y] = 0.0;
  for (int x = 0; x < 5; ++x)
    for (int y = 0; y < 5; ++y) H[x][y] = 0.0;
  for (int x = 0; x < 7; ++x)
    for (int y = 0; x + y < 7; ++y) {
      const double cub = kx * (Sx[x + 3] * Sy[y] + Sx[x + 1] * Sy[y + 2]) + ky * (Sx[x + 2] * Sy[y + 1] + Sx[x] * Sy[y + 3]);
      const double lin = kx * Sx[x + 1] * Sy[y] + ky * Sx[x] * Sy[y + 1];
      G[x][y] = Sx[x] * Sy[y] - 4.0 * lin + i2 * cub;
      if (x + y < 5) H[x][y] = RT * c0 * Sx[x] * Sy[y] + al * cub - be * lin;
    }
}

// Polynomials in (c_x, c_y): up to four terms (coefficient, power of c_x, power of c_y).
struct UPoly {
  int n;
  double c[4];
  int px[4], py[4];
};

__device__ inline UPoly u_basis8(int m) {
  UPoly p;
  switch (m) {
    case 0: p = {1, {1, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}; break;
    case 1: p = {1, {1, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}}; break;
    case 2: p = {1, {1, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}}; break;
    case 3: p = {2, {1, 1, 0, 0}, {2, 0, 0, 0}, {0, 2, 0, 0}}; break;
    case 4: p = {2, {1, 1, 0, 0}, {3, 1, 0, 0}, {0, 2, 0, 0}}; break;
    case 5: p = {2, {1, 1, 0, 0}, {2, 0, 0, 0}, {1, 3, 0, 0}}; break;
    case 6: p = {2, {1, -1, 0, 0}, {2, 0, 0, 0}, {0, 2, 0, 0}}; break;
    default: p = {1, {1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}}; break;
  }
  return p;
}

// constraint row k: g-part and h-part polynomials (the h-part of rows 3..5 is h/2 times c^e)
__device__ inline void u_row8(int k, UPoly& pg, UPoly& ph) {
  ph.n = 0;
  if (k <= 2) {
    pg = u_basis8(k);
  } else if (k == 3) {
    pg = {2, {0.5, 0.5, 0, 0}, {2, 0, 0, 0}, {0, 2, 0, 0}};
    ph = {1, {0.5, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
  } else if (k == 4) {
    pg = {2, {0.5, 0.5, 0, 0}, {3, 1, 0, 0}, {0, 2, 0, 0}};
    ph = {1, {0.5, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}};
  } else if (k == 5) {
    pg = {2, {0.5, 0.5, 0, 0}, {2, 0, 0, 0}, {1, 3, 0, 0}};
    ph = {1, {0.5, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}};
  } else {
    pg = u_basis8(k);
  }
}

// b0..b7 of the eight-moment correction of mp (uncorrected Shakhov parameters of the state
// rho, u, T with heat-flux target q_tar) from the model's peculiar moments G, H; b0..b3 go to
// mp, b4..b7 to b8.
template <class T>
__device__ inline bool u_solve8(const GasDev& gas, double rho, double ux, double uy, double Tm, double qtx,
                                double qty, const double G[7][7], const double H[5][5], MP<T>& mp, T b8[4]) {
  double M[8][8], r[8];
  for (int k = 0; k < 8; ++k) {
    UPoly pg, ph;
    u_row8(k, pg, ph);
    for (int m = 0; m < 8; ++m) {
      const UPoly q = u_basis8(m);
      double s = 0.0;
      for (int i = 0; i < pg.n; ++i)
        for (int j = 0; j < q.n; ++j) s += pg.c[i] * q.c[j] * G[pg.px[i] + q.px[j]][pg.py[i] + q.py[j]];
      for (int i = 0; i < ph.n; ++i)
        for (int j = 0; j < q.n; ++j) s += ph.c[i] * q.c[j] * H[ph.px[i] + q.px[j]][ph.py[i] + q.py[j]];
      M[k][m] = s;
    }
  }
  const double RT = gas.R * Tm;
  const double dux = ux - (double)mp.ux, duy = uy - (double)mp.uy;
  const double tar[8] = {rho, rho * dux, rho * duy,
                         0.5 * (3.0 + gas.K) * rho * RT + 0.5 * rho * (dux * dux + duy * duy), qtx, qty, 0.0, 0.0};
  for (int k = 0; k < 8; ++k) r[k] = tar[k] - M[k][0];
  if (!solve_pivoted<8>(M, r, 8)) return false;
  mp.b0 = T(r[0]); mp.b1 = T(r[1]); mp.b2 = T(r[2]); mp.b3 = T(r[3]);
  for (int m = 0; m < 4; ++m) b8[m] = T(r[4 + m]);
  return true;
}

// The eight-moment correction on a tensor-product space (the moments from one-axis sums).
template <class T>
__device__ inline bool u_correct8(const PointArgs& A, double rho, double ux, double uy, double Tm, double qtx,
                                  double qty, MP<T>& mp, T b8[4]) {
  double G[7][7], H[5][5];
  u_moments8<T>(A, mp, G, H);
  return u_solve8<T>(A.gas, rho, ux, uy, Tm, qtx, qty, G, H, mp, b8);
}

// G[7][7] and H[5][5] of u_moments8 from row_moments<T, 10>'s pair moments (P(i, j) in place
// of the products of one-axis sums), one entry per lane and round, stored to the split
// finalisation's scratch of point i (entries beyond the orders zero).
template <class T>
__device__ inline void row_store_gh8(const PointArgs& A, const MP<T>& mp, int lane, const T* wsm, long i) {
  const double* Pd = reinterpret_cast<const double*>(wsm + row_pd(10));
  auto P = [&](int a, int b) -> double { return Pd[10 * a - a * (a - 1) / 2 + b]; };
  const double kx = (double)mp.kqx, ky = (double)mp.kqy;
  const double i2 = 2.0 * (double)mp.inv2RT, RT = (double)mp.RT, c0 = A.k.c0;
  const double al = RT * c0 * i2, be = RT * (2.0 * c0 + A.k.twoK);
  const long n = A.npt;
  for (int e = lane; e < 74; e += 32) {
    const bool h = e >= 49;
    const int x = h ? (e - 49) / 5 : e / 7, y = h ? (e - 49) % 5 : e % 7;
    double v = 0.0;
    if (x + y < (h ? 5 : 7)) {
      const double cub = kx * (P(x + 3, y) + P(x + 1, y + 2)) + ky * (P(x + 2, y + 1) + P(x, y + 3));
      const double lin = kx * P(x + 1, y) + ky * P(x, y + 1);
      v = h ? RT * c0 * P(x, y) + al * cub - be * lin : P(x, y) - 4.0 * lin + i2 * cub;
    }
    A.scr[(FS_G8 + e) * n + i] = v;
  }
}

// Shakhov model times the eight-term correction factor (model_eval's operation order for the
// model itself, then the factor).
template <class T>
__device__ __forceinline__ void u_model_eval8(const MP<T>& p, const T* b8, T xix, T xiy, T c0, T twoK, T& g,
                                              T& h) {
  using N = Num<T>;
  const T cx = N::sub(xix, p.ux), cy = N::sub(xiy, p.uy);
  const T geq = maxwell_sep<T, 2>(p, cx, cy);
  const T cc = N::fma(cy, cy, N::mul(cx, cx));
  const T cq = N::fma(p.kqy, cy, N::mul(p.kqx, cx));
  const T t = N::mul(N::mul(T(2), p.inv2RT), cc);
  const T gs = N::mul(geq, N::fma(cq, N::sub(t, T(4)), T(1)));
  const T hs = N::mul(N::mul(p.RT, geq), N::fma(cq, N::fma(N::sub(t, T(2)), c0, -twoK), c0));
  T corr = N::fma(p.b3, cc, N::fma(p.b2, cy, N::fma(p.b1, cx, p.b0)));
  corr = N::fma(N::mul(b8[0], cc), cx, corr);
  corr = N::fma(N::mul(b8[1], cc), cy, corr);
  corr = N::fma(b8[2], N::fma(cx, cx, -N::mul(cy, cy)), corr);
  corr = N::fma(N::mul(b8[3], cx), cy, corr);
  g = N::fma(gs, corr, gs);
  h = N::fma(hs, corr, hs);
}

// Model parameters of a point with state (rho, u, T, q), before the correction.
template <class T, int D>
__device__ inline void point_params(const GasDev& g, double rho, double ux, double uy, double Tm, double qx,
                                    double qy, MP<T>& mp) {
  const double RT = g.R * Tm;
  const double p = rho * RT;
  const double kap = (1.0 - g.Pr) / (5.0 * p * RT);
  mp.ux = T(ux); mp.uy = T(uy);
  mp.lnh = T((log(rho) - 0.5 * D * log(2.0 * 3.14159265358979323846 * RT)) / D);
  mp.inv2RT = T(0.5 / RT);
  mp.kqx = T(kap * qx); mp.kqy = T(kap * qy);
  mp.RT = T(RT);
  mp.b0 = T(0); mp.b1 = T(0); mp.b2 = T(0); mp.b3 = T(0);
}

// The four-moment compatibility correction (b0..b3 of mp) from the model moments.
template <class T, int D>
__device__ inline bool point_correct(const GasDev& g, double rho, double ux, double uy, double Tm,
                                     const double G[5][5], const double H[3][3], MP<T>& mp) {
  const double RT = g.R * Tm;
  // rows: (g, c_x g, c_y g, (|c|^2 g + h)/2); columns: basis (1, c_x, c_y, |c|^2)
  double M[4][4], b[4];
  M[0][0] = G[0][0]; M[0][1] = G[1][0]; M[0][2] = G[0][1]; M[0][3] = G[2][0] + G[0][2];
  M[1][0] = G[1][0]; M[1][1] = G[2][0]; M[1][2] = G[1][1]; M[1][3] = G[3][0] + G[1][2];
  M[2][0] = G[0][1]; M[2][1] = G[1][1]; M[2][2] = G[0][2]; M[2][3] = G[2][1] + G[0][3];
  M[3][0] = 0.5 * (G[2][0] + G[0][2] + H[0][0]);
  M[3][1] = 0.5 * (G[3][0] + G[1][2] + H[1][0]);
  M[3][2] = 0.5 * (G[2][1] + G[0][3] + H[0][1]);
  M[3][3] = 0.5 * (G[4][0] + 2.0 * G[2][2] + G[0][4] + H[2][0] + H[0][2]);
  const double dux = ux - (double)mp.ux, duy = (D == 2) ? uy - (double)mp.uy : 0.0;
  const double rhoe = 0.5 * (3.0 + g.K) * rho * RT + 0.5 * rho * (dux * dux + duy * duy);
  b[0] = rho - M[0][0];
  b[1] = rho * dux - M[1][0];
  b[2] = rho * duy - M[2][0];
  b[3] = rhoe - M[3][0];
  const int idx2[4] = {0, 1, 2, 3}, idx1[3] = {0, 1, 3};
  if (!solve_small(M, b, D == 2 ? idx2 : idx1, D == 2 ? 4 : 3)) return false;
  mp.b0 = T(b[0]); mp.b1 = T(b[1]); mp.b2 = T(b[2]); mp.b3 = T(b[3]);
  return true;
}

// Model parameters of a point with state (rho, u, T, q), with the compatibility correction.
template <class T, int D>
__device__ inline bool point_model(const PointArgs& A, double rho, double ux, double uy, double Tm,
                                   double qx, double qy, MP<T>& mp) {
  point_params<T, D>(A.gas, rho, ux, uy, Tm, qx, qy, mp);
  if (!A.compat) return true;
  double G[5][5], H[3][3];
  if (A.k.nax > 0) axis_moments<T, D>(A, mp, G, H);
  else direct_moments<T, D, 1>(A, mp, 0, G, H);
  return point_correct<T, D>(A.gas, rho, ux, uy, Tm, G, H, mp);
}

template <class T>
__device__ __forceinline__ void store_mp(T* P, long n, long i, const MP<T>& m, T kind) {
  P[P_UX * n + i] = m.ux; P[P_UY * n + i] = m.uy; P[P_LNH * n + i] = m.lnh;
  P[P_INV2RT * n + i] = m.inv2RT; P[P_KQX * n + i] = m.kqx; P[P_KQY * n + i] = m.kqy;
  P[P_RT * n + i] = m.RT; P[P_B0 * n + i] = m.b0; P[P_B1 * n + i] = m.b1;
  P[P_B2 * n + i] = m.b2; P[P_B3 * n + i] = m.b3; P[P_C1 * n + i] = m.c1;
  P[P_C2 * n + i] = m.c2; P[P_KIND * n + i] = kind;
}

// Parameters of the unit-density wall Maxwellian (u_w, v_w, T_w).
template <class T>
__device__ __forceinline__ void wall_mp(double R, double uw, double vw, double Tw, MP<T>& mp) {
  const double RT = R * Tw;
  mp.ux = T(uw); mp.uy = T(vw);
  mp.lnh = T(-0.5 * log(2.0 * 3.14159265358979323846 * RT));
  mp.inv2RT = T(0.5 / RT); mp.RT = T(RT);
  mp.kqx = T(0); mp.kqy = T(0);
  mp.b0 = T(0); mp.b1 = T(0); mp.b2 = T(0); mp.b3 = T(0); mp.c1 = T(0); mp.c2 = T(0);
}

// Curvilinear walls: den = sum_{xi.n_in > 0} w (xi.n_in) g_w of every wall face (a warp per
// face), with xi.n formed as the tile kernels form it.  Constant in time; computed once.
template <class T, int D>
__global__ void k_wall_den_table(const StepConst k, GasDev gas, const T* __restrict__ vt,
                                 const T* __restrict__ fgeo, const double* __restrict__ wallv, double* __restrict__ out) {
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= k.nface) return;
  int side = -1;
  const int nxf = k.nfx * k.ny;
  if (f < nxf) {
    const int gi = f % k.nfx;
    if (!k.px && gi == 0 && k.bc[0] == BC_WALL) side = 0;
    if (!k.px && gi == k.nx && k.bc[1] == BC_WALL) side = 1;
  } else {
    const int gj = (f - nxf) / k.nx;
    if (!k.py && gj == 0 && k.bc[2] == BC_WALL) side = 2;
    if (!k.py && gj == k.ny && k.bc[3] == BC_WALL) side = 3;
  }
  if (side < 0) {
    if (lane == 0) out[f] = 0.0;
    return;
  }
  MP<T> mp;
  wall_mp<T>(gas.R, wallv[3 * side], wallv[3 * side + 1], wallv[3 * side + 2], mp);
  const T sgn = (side == 0 || side == 2) ? T(1) : T(-1);
  const T nx = fgeo[f], ny = fgeo[(long)k.nface + f];
  const int nv = k.nv;
  KSum<T> den;
  den.zero();
  for (int v = lane; v < nv; v += 32) {
    const T xx = vt[v], yy = vt[nv + v];
    const T xn = Num<T>::add(Num<T>::mul(xx, nx), Num<T>::mul(yy, ny));   // as the tile kernels form it
    const T xin = sgn * xn;
    if (xin > T(0)) {
      T gv, hv;
      model_eval<T, D>(mp, xx, yy, T(k.c0), T(k.twoK), gv, hv);
      den.add(vt[2 * nv + v] * (vt[3 * nv + v] * (xin * gv)));
    }
  }
  const double d = lane_sum<32>(den.val());
  if (lane == 0) out[f] = d;
}

__device__ __forceinline__ int wrap_or_clamp_h(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Normal mass flux of the unit-density wall Maxwellian over the velocities entering the
// domain: den = sum_{xi.n_in > 0} w (xi.n_in) g_w, with the tile kernels' evaluation.
template <class T, int D, int LANES>
__device__ inline double wall_den(const PointArgs& A, const MP<T>& mp, bool xdir, T sgn, int lane) {
  const StepConst& k = A.k;
  if (k.nax > 0) {
    const T* ax = reinterpret_cast<const T*>(A.ax);
    KSum<T> nrm, tan_;
    nrm.zero(); tan_.zero();
    const T un = xdir ? mp.ux : mp.uy, ut = xdir ? mp.uy : mp.ux;
    for (int i = 0; i < k.nax; ++i) {
      const T X = ax[i], Wt = ax[k.nax + i];
      const T xin = sgn * X;
      if (xin > T(0)) nrm.add(Wt * xin * Num<T>::gauss(X - un, mp.inv2RT, mp.lnh));
      if (D == 2) tan_.add(Wt * Num<T>::gauss(X - ut, mp.inv2RT, mp.lnh));
    }
    return D == 2 ? nrm.val() * tan_.val() : nrm.val();
  }
  const T* vt = reinterpret_cast<const T*>(A.vt);
  const int nv = k.nv;
  KSum<T> den;
  den.zero();
  for (int v = lane; v < nv; v += LANES) {
    const T xx = vt[v], yy = (D == 2) ? vt[nv + v] : T(0);
    const T xin = sgn * (xdir ? xx : yy);
    if (xin > T(0)) {
      T gv, hv;
      model_eval<T, D>(mp, xx, yy, T(k.c0), T(k.twoK), gv, hv);
      den.add(vt[2 * nv + v] * (vt[3 * nv + v] * (xin * gv)));
    }
  }
  return lane_sum<LANES>(den.val());
}

// Cells (is_face = 0): Eq. discrete_W, Eq. discrete_q, tau = mu(T)/p, blending of phi-bar-plus.
// Faces (is_face = 1): Eq. W_from_bar, q = 2 tau/(2 tau + s Pr) q-bar, Eq. recover_phi weights;
// wall faces: rho_w from the zero net normal mass flux.
// One thread per point.  PART 0: everything (tensor-product spaces); PART 1: k_fin_pre's
// share of the split path (state and uncorrected model into the parameters and scratch).
template <class T, int D, int PART>
__device__ __forceinline__ void finalize_point(const PointArgs& a, int i) {
  if (i >= a.nwork) return;
  if (a.pts) i = a.pts[i];
  if (a.is_face && a.frole && a.frole[i] != FR_NORMAL && a.frole[i] != FR_CROSS) return;
  const StepConst& k = a.k;
  const T* cp = reinterpret_cast<const T*>(a.cprm);
  const T* uc = reinterpret_cast<const T*>(a.ucell);
  T* po = reinterpret_cast<T*>(a.prm_out);
  const long nc = k.ncell;
  const GasDev& g = a.gas;
  double M[NMOM];
#pragma unroll
  for (int m = 0; m < NMOM; ++m) M[m] = 0.0;
  T shx = T(0), shy = T(0);
  int kind = FK_INTERIOR;
  int side = -1;
  {
    if (a.msum) {
#pragma unroll
      for (int m = 0; m < NMOM; ++m) M[m] = a.msum[(long)m * a.npt + i];
    } else {
      for (int c = 0; c < k.nchunk; ++c)
#pragma unroll
        for (int m = 0; m < NMOM; ++m) M[m] += a.part[((long)c * NMOM + m) * a.npt + i];
    }
    if (!a.is_face) {
      shx = cp[P_UX * (long)a.npt + i];
      shy = cp[P_UY * (long)a.npt + i];
    } else {
      int sL, sR;
      const int nxf = k.nfx * k.ny;
      if (i < nxf) {
        const int gj = i / k.nfx, gi = i % k.nfx;
        sL = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + wrap_or_clamp_h(gi - 1, k.nx, k.px);
        sR = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + wrap_or_clamp_h(gi, k.nx, k.px);
        if (!k.px && gi == 0 && k.bc[0] == BC_WALL) { kind = FK_WALL_LO; side = 0; }
        if (!k.px && gi == k.nx && k.bc[1] == BC_WALL) { kind = FK_WALL_HI; side = 1; }
        if (!k.px && gi == 0 && k.bc[0] == BC_FREE) { kind = FK_FREE_LO; side = 0; }
        if (!k.px && gi == k.nx && k.bc[1] == BC_FREE) { kind = FK_FREE_HI; side = 1; }
      } else {
        const int r = i - nxf;
        const int gj = r / k.nx, gi = r % k.nx;
        sL = wrap_or_clamp_h(gj - 1, k.ny, k.py) * k.nx + gi;
        sR = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + gi;
        if (!k.py && gj == 0 && k.bc[2] == BC_WALL) { kind = FK_WALL_LO; side = 2; }
        if (!k.py && gj == k.ny && k.bc[3] == BC_WALL) { kind = FK_WALL_HI; side = 3; }
        if (!k.py && gj == 0 && k.bc[2] == BC_FREE) { kind = FK_FREE_LO; side = 2; }
        if (!k.py && gj == k.ny && k.bc[3] == BC_FREE) { kind = FK_FREE_HI; side = 3; }
      }
      shx = T(0.5) * (uc[sL] + uc[sR]);
      shy = (D == 2) ? T(0.5) * (uc[nc + sL] + uc[nc + sR]) : T(0);
    }
  }
  // the state and the uncorrected model; need: 1 = wall density sum, 2 = model moments
  MP<T> mp;
  mp.ux = mp.uy = mp.lnh = mp.inv2RT = mp.kqx = mp.kqy = mp.RT = T(0);
  mp.b0 = mp.b1 = mp.b2 = mp.b3 = mp.c1 = mp.c2 = T(0);
  int need = 0;
  double rho = 0, ux = 0, uy = 0, Tm = 0, qx = 0, qy = 0, tau = 0;
  bool state_ok = false;
  const bool wall = kind == FK_WALL_LO || kind == FK_WALL_HI;
  const bool free_ = kind == FK_FREE_LO || kind == FK_FREE_HI;
  if (wall) {
    wall_mp<T>(g.R, a.wall[side][0], a.wall[side][1], a.wall[side][2], mp);
    need = 1;
  } else if (free_) {
    // freestream side: the model of the freestream state, entering with weight one
    rho = a.far[0];
    ux = a.far[1];
    uy = (D == 2) ? a.far[2] : 0.0;
    Tm = a.far[3];
    state_ok = true;
    point_params<T, D>(g, rho, ux, uy, Tm, 0.0, 0.0, mp);
    if (a.compat) need = 2;
  } else {
    rho = M[MO_0];
    const double upx = M[MO_X] / rho, upy = (D == 2) ? M[MO_Y] / rho : 0.0;
    const double u2 = upx * upx + upy * upy;
    ux = (double)shx + upx;
    uy = (D == 2) ? (double)shy + upy : 0.0;
    Tm = (M[MO_E] - rho * u2) / ((3.0 + g.K) * rho * g.R);
    // q = 1/2 [J - 2 u'.G - u' E' + 2 rho |u'|^2 u']  in the shifted frame
    qx = 0.5 * (M[MO_JX] - 2.0 * (upx * M[MO_GXX] + upy * M[MO_GXY]) - upx * M[MO_E] + 2.0 * rho * u2 * upx);
    qy = (D == 2) ? 0.5 * (M[MO_JY] - 2.0 * (upx * M[MO_GXY] + upy * M[MO_GYY]) - upy * M[MO_E] + 2.0 * rho * u2 * upy) : 0.0;
    const double p = rho * g.R * Tm;
    const double mu = g.mu_ref * pow(Tm / g.T_ref, g.omega);
    tau = mu / p;
    const double hdt = a.is_face ? 0.5 * k.dt : k.dt;    // dt at cells, s at faces
    const double qf = 2.0 * tau / (2.0 * tau + hdt * g.Pr);
    qx *= qf;
    qy *= qf;
    state_ok = isfinite(rho) && isfinite(Tm) && isfinite(ux) && isfinite(uy) && rho > 0.0 && Tm > 0.0;
    if (state_ok) {
      point_params<T, D>(g, rho, ux, uy, Tm, qx, qy, mp);
      if (a.compat) need = 2;
    }
  }
  if (PART == 1) {
    // split path: the uncorrected model and what k_fin_sums / k_fin_post need; need 3: the
    // eight-moment correction (cells and faces, not freestream sides), with its heat-flux
    // target (1 - Pr) q
    const bool c8s = D == 2 && a.prm8_out && need == 2 && !free_;
    a.need[i] = need == 1 ? 16 + 4 * side + kind : (c8s ? 3 : need);
    a.scr[FS_RHO * (long)a.npt + i] = wall ? M[MO_0] : rho;
    a.scr[FS_UX * (long)a.npt + i] = ux;
    a.scr[FS_UY * (long)a.npt + i] = uy;
    a.scr[FS_T * (long)a.npt + i] = Tm;
    if (c8s) {
      a.scr[FS_QX * (long)a.npt + i] = (1.0 - g.Pr) * qx;
      a.scr[FS_QY * (long)a.npt + i] = (1.0 - g.Pr) * qy;
    }
  }
  double den = 0.0;
  double G[5][5], H[3][3];
  // the eight-moment correction replaces the four-moment one at cells and faces (not on
  // freestream sides, which keep the four-moment correction)
  const bool c8 = D == 2 && PART == 0 && a.prm8_out && !free_ && !wall;
  T* p8 = reinterpret_cast<T*>(a.prm8_out);
  if (PART == 0) {
    if (need == 1)
      den = a.wden ? a.wden[i] : wall_den<T, D, 1>(a, mp, side < 2, (kind == FK_WALL_LO) ? T(1) : T(-1), 0);
    if (need == 2 && !c8) {
      if (k.nax > 0) axis_moments<T, D>(a, mp, G, H);
      else direct_moments<T, D, 1>(a, mp, 0, G, H);
    }
  }
  if (p8)   // nonzero only where the eight-moment correction is solved
    for (int m = 0; m < 4; ++m) p8[m * (long)a.npt + i] = T(0);
  if (wall) {
    if (PART == 1) {   // rho_w in k_fin_post
      store_mp<T>(po, a.npt, i, mp, T(kind));
      po[P_SHX * (long)a.npt + i] = shx;
      po[P_SHY * (long)a.npt + i] = shy;
      return;
    }
    // diffuse wall: unit-density wall Maxwellian, rho_w = -M_out / den
    const double rw = -M[MO_0] / den;
    // rho_w as an unevaluated sum hi + lo, so that its rounding leaves no net wall mass flux
    mp.c2 = T(rw);
    mp.c1 = T(rw - (double)mp.c2);
    store_mp<T>(po, a.npt, i, mp, T(kind));
    po[P_SHX * (long)a.npt + i] = shx;
    po[P_SHY * (long)a.npt + i] = shy;
    // rho_w follows from zero net mass flux even where a non-positive incident distribution
    // (a near-vacuum wall cell) makes it slightly negative; only a non-finite value is an error
    if (!isfinite(rw)) atomicOr(a.err, ERR_NONFINITE);
    return;
  }
  bool ok = true;
  if (PART == 0 && need == 2) {
    if constexpr (D == 2) {
      if (c8) {
        // heat-flux target: the Shakhov model's own heat flux (1 - Pr) q
        T b8[4];
        const double pr = 1.0 - g.Pr;
        ok = u_correct8<T>(a, rho, ux, uy, Tm, pr * qx, pr * qy, mp, b8);
        for (int m = 0; m < 4; ++m) p8[m * (long)a.npt + i] = b8[m];
      } else {
        ok = point_correct<T, D>(g, rho, ux, uy, Tm, G, H, mp);
      }
    } else {
      ok = point_correct<T, D>(g, rho, ux, uy, Tm, G, H, mp);
    }
  }
  const double s = 0.5 * k.dt;
  if (free_) {
    mp.c1 = T(1);
    mp.c2 = T(0);
  } else if (!a.is_face) {
    mp.c1 = T(3.0 * s / (2.0 * tau + k.dt));
    mp.c2 = T(4.0 * s / (2.0 * tau + k.dt));
  } else {
    mp.c1 = T(2.0 * tau / (2.0 * tau + s));
    mp.c2 = T(s / (2.0 * tau + s));
  }
  store_mp<T>(po, a.npt, i, mp, T(kind));
  po[P_SHX * (long)a.npt + i] = shx;
  po[P_SHY * (long)a.npt + i] = shy;
  if (a.W) {
    const long wi = a.ids ? a.ids[i] : i;   // global cell id of a cell point
    a.W[0 * nc + wi] = rho;
    a.W[1 * nc + wi] = ux;
    a.W[2 * nc + wi] = uy;
    a.W[3 * nc + wi] = Tm;
    a.W[4 * nc + wi] = qx;
    a.W[5 * nc + wi] = qy;
    a.W[6 * nc + wi] = rho * (0.5 * (ux * ux + uy * uy) + 0.5 * (3.0 + g.K) * g.R * Tm);
    a.W[7 * nc + wi] = tau;
    // stress deviator of phi: 2 tau/(2 tau + dt) (P~ - p I), P~ the central second moment of g~
    const double upx = M[MO_X] / rho, upy = (D == 2) ? M[MO_Y] / rho : 0.0;
    const double sf = 2.0 * tau / (2.0 * tau + k.dt), pr = rho * g.R * Tm;
    a.W[8 * nc + wi] = sf * (M[MO_GXX] - rho * upx * upx - pr);
    a.W[9 * nc + wi] = sf * (M[MO_GXY] - rho * upx * upy);
    a.W[10 * nc + wi] = (D == 2) ? sf * (M[MO_GYY] - rho * upy * upy - pr) : 0.0;
  }
  if (!ok) report_point(a.err, ERR_SINGULAR, i, a.is_face, rho, Tm);
  if (!isfinite(rho) || !isfinite(Tm) || !isfinite(ux) || !isfinite(uy))
    report_point(a.err, ERR_NONFINITE, i, a.is_face, rho, Tm);
  else if (!(rho > 0.0) || !(Tm > 0.0)) report_point(a.err, ERR_POSITIVITY, i, a.is_face, rho, Tm);
}

template <class T, int D>
__global__ void k_finalize(const PointArgs a) {
  finalize_point<T, D, 0>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <class T, int D>
__global__ void k_fin_pre(const PointArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nwork) return;
  a.need[a.pts ? a.pts[i] : i] = 0;
  finalize_point<T, D, 1>(a, i);
}

// Velocity sums of the split path, a warp per point (blockDim a multiple of 32).  C8: the form
// with the eight-moment correction's sums (need 3, spaces with row tables).
template <class T, int D, bool C8 = false>
__global__ void k_fin_sums(const PointArgs a) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= a.nwork) return;
  if (a.pts) i = a.pts[i];
  const int need = a.need[i];
  if (need == 0) return;
  const T* P = reinterpret_cast<const T*>(a.prm_out);
  MP<T> q;
  q.load(P, a.npt, i);
  q.b0 = q.b1 = q.b2 = q.b3 = T(0);
  const long n = a.npt;
  if (need >= 16) {
    if (a.wden) {
      if (lane == 0) a.scr[FS_DEN * n + i] = a.wden[i];
      return;
    }
    const int side = (need - 16) >> 2, kind = (need - 16) & 3;
    const double d = wall_den<T, D, 32>(a, q, side < 2, (kind == FK_WALL_LO) ? T(1) : T(-1), lane);
    if (lane == 0) a.scr[FS_DEN * n + i] = d;
    return;
  }
  if constexpr (C8 && D == 2) {
    if (need == 3) {
      if (!a.rows) {   // the host checks that the level's space has row tables
        if (lane == 0) atomicOr(a.err, ERR_SINGULAR);
        return;
      }
      extern __shared__ __align__(16) unsigned char fsm8[];
      T* wsm = reinterpret_cast<T*>(fsm8) + (size_t)(threadIdx.x >> 5) * row_smem_values(a.n1, 10);
      row_moments<T, 10>(a, q, lane, wsm);
      row_store_gh8<T>(a, q, lane, wsm, i);
      return;
    }
  }
  double G[5][5], H[3][3];
  if (a.k.nax > 0) {
    // tensor-product space: the one-axis sums over the lanes, combined on lane 0
    const T* ax = reinterpret_cast<const T*>(a.ax);
    double Sx[8], Sy[8];
    axis_sums_lanes<T, 32>(ax, a.k.nax, q.ux, q.inv2RT, q.lnh, lane, Sx);
    if (D == 2) {
      axis_sums_lanes<T, 32>(ax, a.k.nax, q.uy, q.inv2RT, q.lnh, lane, Sy);
    } else {
      Sy[0] = 1.0;
      for (int b = 1; b < 8; ++b) Sy[b] = 0.0;
    }
    if (lane != 0) return;
    axis_combine<T, D>(a, q, Sx, Sy, G, H);
  } else if (D == 2 && a.rows) {
    // a space that is not a tensor product, from its rows
    extern __shared__ __align__(16) unsigned char fsm[];
    T* wsm = reinterpret_cast<T*>(fsm) + (size_t)(threadIdx.x >> 5) * row_smem_values(a.n1, C8 ? 10 : 8);
    row_moments<T>(a, q, lane, wsm);
    row_store_gh<T, D>(a, q, lane, wsm, i);
    return;
  } else {
    direct_moments<T, D, 32>(a, q, lane, G, H);
  }
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < 25; ++r) a.scr[(FS_G + r) * n + i] = G[r / 5][r % 5];
#pragma unroll
    for (int r = 0; r < 9; ++r) a.scr[(FS_H + r) * n + i] = H[r / 3][r % 3];
  }
}

// Correction of the split path: wall densities and the four-moment solve (C8: the eight-moment
// solve of need-3 points as well).
template <class T, int D, bool C8 = false>
__global__ void k_fin_post(const PointArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nwork) return;
  if (a.pts) i = a.pts[i];
  const int need = a.need[i];
  if (need == 0) return;
  T* po = reinterpret_cast<T*>(a.prm_out);
  const long n = a.npt;
  if (need >= 16) {
    const double rw = -a.scr[FS_RHO * n + i] / a.scr[FS_DEN * n + i];
    const T hi = T(rw);
    po[P_C2 * n + i] = hi;
    po[P_C1 * n + i] = T(rw - (double)hi);
    if (!isfinite(rw)) atomicOr(a.err, ERR_NONFINITE);   // a negative rho_w is what the flux balance gives
    return;
  }
  MP<T> mp;
  mp.load(po, n, i);
  if constexpr (C8 && D == 2) {
    if (need == 3) {
      double G8[7][7], H8[5][5];
      for (int r = 0; r < 49; ++r) G8[r / 7][r % 7] = a.scr[(FS_G8 + r) * n + i];
      for (int r = 0; r < 25; ++r) H8[r / 5][r % 5] = a.scr[(FS_H8 + r) * n + i];
      T b8[4];
      const bool ok8 = u_solve8<T>(a.gas, a.scr[FS_RHO * n + i], a.scr[FS_UX * n + i], a.scr[FS_UY * n + i],
                                   a.scr[FS_T * n + i], a.scr[FS_QX * n + i], a.scr[FS_QY * n + i], G8, H8, mp, b8);
      po[P_B0 * n + i] = mp.b0;
      po[P_B1 * n + i] = mp.b1;
      po[P_B2 * n + i] = mp.b2;
      po[P_B3 * n + i] = mp.b3;
      T* p8 = reinterpret_cast<T*>(a.prm8_out);
      for (int m = 0; m < 4; ++m) p8[m * n + i] = b8[m];
      if (!ok8) atomicOr(a.err, ERR_SINGULAR);
      return;
    }
  }
  double G[5][5], H[3][3];
#pragma unroll
  for (int r = 0; r < 25; ++r) G[r / 5][r % 5] = a.scr[(FS_G + r) * n + i];
#pragma unroll
  for (int r = 0; r < 9; ++r) H[r / 3][r % 3] = a.scr[(FS_H + r) * n + i];
  const bool ok = point_correct<T, D>(a.gas, a.scr[FS_RHO * n + i], a.scr[FS_UX * n + i], a.scr[FS_UY * n + i],
                                      a.scr[FS_T * n + i], G, H, mp);
  po[P_B0 * n + i] = mp.b0;
  po[P_B1 * n + i] = mp.b1;
  po[P_B2 * n + i] = mp.b2;
  po[P_B3 * n + i] = mp.b3;
  if (!ok) atomicOr(a.err, ERR_SINGULAR);
}

// Sums of the velocity-chunk partials in chunk order, one thread per (moment, point): the
// same values a finalisation thread would form, with the FP64 chains spread over many warps.
// pts (null: every point) lists the nwork points to sum; npt is the stride of part and out.
static __global__ void k_sum_chunks(const double* __restrict__ part, int nchunk, int npt, const int* __restrict__ pts,
                                    int nwork, double* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)NMOM * nwork) return;
  const int m = (int)(t / nwork), w = (int)(t % nwork);
  const int i = pts ? pts[w] : w;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((long)c * NMOM + m) * npt + i];
  out[(long)m * npt + i] = s;
}

// Initial parameters from (rho, u, v, T) with q = 0 (phi~ = phi^eq at t = 0).
template <class T, int D>
__global__ void k_init_params(const PointArgs a, const double* W0 /* [ncell][4] */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.npt) return;
  T* po = reinterpret_cast<T*>(a.prm_out);
  const double rho = W0[4 * i], ux = W0[4 * i + 1], uy = (D == 2) ? W0[4 * i + 2] : 0.0, Tm = W0[4 * i + 3];
  MP<T> mp;
  bool ok = point_model<T, D>(a, rho, ux, uy, Tm, 0.0, 0.0, mp);
  mp.c1 = T(0); mp.c2 = T(0);
  store_mp<T>(po, a.npt, i, mp, T(0));
  po[P_SHX * (long)a.npt + i] = mp.ux;
  po[P_SHY * (long)a.npt + i] = mp.uy;
  if (!ok) atomicOr(a.err, ERR_SINGULAR);
}

// phi~ = corrected Maxwellian of the initial parameters.
template <class S, class T, int D>
__global__ void k_init_f(StepConst k, int n, const T* __restrict__ prm, const T* __restrict__ vt,
                         S* __restrict__ f) {
  const long nc = n;   // cells of the level
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  MP<T> m;
  m.load(prm, nc, c);
  const T c0 = T(k.c0), twoK = T(k.twoK);
  for (int v = blockIdx.y; v < k.nv; v += gridDim.y) {
    T g, h;
    model_eval<T, D>(m, vt[v], (D == 2) ? vt[k.nv + v] : T(0), c0, twoK, g, h);
    unsigned rb = 0;
    if constexpr (sizeof(S) == 2) rb = hash32(0x5bd1e995u ^ hash32((unsigned)c * 0x9e3779b1u + (unsigned)v));
    f[(long)v * nc + c] = Stored<S, T>::enc(g, rb);
    f[((long)k.nv + v) * nc + c] = Stored<S, T>::enc(h, rb >> 16);
  }
}

// Chunk partial moments of f in the frame of the cell velocity in prm (used after init).
template <class S, class T, int D>
__global__ void k_moments(StepConst k, int n, const T* __restrict__ prm, const T* __restrict__ vt,
                          const S* __restrict__ f, double* __restrict__ part) {
  const long nc = n;   // cells of the level
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int chunk = blockIdx.y;
  const int v0 = chunk * k.vpc, v1 = min(k.nv, v0 + k.vpc);
  const T ux = prm[P_UX * nc + c], uy = prm[P_UY * nc + c];
  KSum<T> a0, ax, ay, ae;
  a0.zero(); ax.zero(); ay.zero(); ae.zero();
  T gxx = 0, gxy = 0, gyy = 0, jx = 0, jy = 0;
  const long nv = k.nv;
  for (int v = v0; v < v1; ++v) {
    const T gq = ldf<S, T>(f + (long)v * nc + c), hq = ldf<S, T>(f + (nv + v) * nc + c);
    const T xp = vt[v] - ux, yp = (D == 2) ? vt[nv + v] - uy : T(0);
    const T wxv = vt[2 * nv + v], wyv = vt[3 * nv + v];
    const T wg = wxv * (wyv * gq);
    const T e = wxv * (wyv * ((xp * xp + yp * yp) * gq + hq));
    a0.add(wg); ax.add(wg * xp); ae.add(e);
    gxx += wg * xp * xp; jx += e * xp;
    if (D == 2) { ay.add(wg * yp); gxy += wg * xp * yp; gyy += wg * yp * yp; jy += e * yp; }
  }
  double* P = part + (long)chunk * NMOM * nc + c;
  P[MO_0 * nc] = a0.val(); P[MO_X * nc] = ax.val(); P[MO_Y * nc] = (D == 2) ? ay.val() : 0.0;
  P[MO_E * nc] = ae.val(); P[MO_GXX * nc] = gxx; P[MO_GXY * nc] = gxy; P[MO_GYY * nc] = gyy;
  P[MO_JX * nc] = jx; P[MO_JY * nc] = jy;
}

}  // namespace mlvs
