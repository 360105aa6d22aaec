// Velocity-space requirement of every cell (Sec. 3.2): one CTA per cell.
//
// The cell's (g~, h~) on its current space is read on the base grid by inheritance (every
// base node takes the g and H = h + |xi|^2 g of the point that covers it, Sec. 3.3.2).  Then
//   * per level-1 block b: S1(b) = sum_b w g and S2(b) = sum_b w H (FP64, in shared memory),
//     so that a candidate block's contributions (Eq. M1/M2) are sums of S1, S2 over its
//     level-1 blocks divided by the totals;
//   * I_B = max(sum_B M1, sum_B M2) (Eq. block-contribution-indicator) and the three-regime
//     rule with hysteresis (Eq. block-hysteresis-rule), with the transport-error test of
//     Eq. merge-transport-error / combined-merge-condition below C_merge when eps > 0;
//   * the hierarchical scan: a level-3 candidate block first, its level-2 children if it
//     does not merge, then their level-1 blocks; a merged block writes its level into kappa
//     of every level-1 block it holds, a level-1 block that does not merge writes 0.
// "Previous status" is the consistent coarsening index of the space the cell is on.
//
// FP64 throughout (the decisions compare sums with thresholds).  The transport test needs,
// per candidate block, sums of w xi_d m_r over the nodes on each side of xi_d = 0; a level-1
// block never straddles xi = 0 (the centre node is a group of its own), so these sums add up
// over level-1 blocks: the node pass stores seven more per-block sums (x g, y g, x^2 g,
// x y g, y^2 g, x H, y H) in shared memory when it holds them (tblk = 1), else in a global
// scratch slice per CTA (tblk = 2), and a candidate block adds its members' sums.  The scale
// S_r of the test uses per-point geometric sums of the cell's space (inherited values are
// constant on a point's rectangle).  A level-1 block inside one point of the cell's space takes its sums
// from that point's g and H times the block's geometric sums.  Thresholds are applied as
// products (s1 < C T1 for s1/T1 < C, |F - F~| <= eps S_r for the relative error), which is
// the same test up to rounding.
#pragma once
#include "mlvs_common.cuh"

namespace mlvs {

struct CritArgs {
  const int* sel;              // slots to evaluate, one CTA each (null: slot = CTA index)
  const void* f;               // [2][nv][ns] phi~ of the level (storage type)
  int ns, nv;
  const int* ids;              // [ns] global cell of every slot
  const int* owner;            // [n*n] point of this space covering base node (iy, ix)
  const double* xi;            // [2][nv] point coordinates
  const double* bx;            // [n] base nodes
  const double* bw;            // [n] base weights
  int n, N1;
  const int* g1;               // [N1+1] first base index of every level-1 group (+ n)
  const int* pstart;           // [4][N1+1] row L: first level-1 block of every level-L group
  const int* cstart;           // [4][N1+1] row L: first level-(L-1) group of every level-L group
  int ng[4];                   // groups per axis at level L
  const unsigned char* kprev;  // [N1*N1] consistent coarsening index of this space
  const double* W1;            // [N1] sum of w over every level-1 group
  const double* X1;            // [N1] sum of w x over every level-1 group
  const double* XX1;           // [N1] sum of w x^2 over every level-1 group
  const double* geo;           // [5][nv] per point: sum w|x|, sum w|y|, sum w x^2, sum w y^2, sum w|x||y|
  double C_split, C_merge, eps;
  int max_level;
  int tblk;                    // per-block transport sums: 0 none (the test walks the nodes),
                               // 1 in shared memory, 2 in global scratch (TBg)
  double* TBg;                 // tblk == 2: [gridDim.x][CB_N][N1*N1], one slice per CTA
  int sel0;                    // first entry of sel (or first slot) of this launch
  unsigned char* kout;         // [ncell][N1*N1]
};

enum { CB_XG = 0, CB_YG, CB_XXG, CB_XYG, CB_YYG, CB_XH, CB_YH, CB_N };

constexpr int CRIT_THREADS = 256;

struct CritCtx {
  const CritArgs* a;
  const double* S1;
  const double* S2;
  const double* TB;            // [CB_N][nb] when a->tblk != 0
  double T1, T2;
  double Sr[4];
  double epsSr[4];             // eps * S_r
  int slot;
  unsigned char* out;
};

template <class S> __device__ __forceinline__ double ld_d(const S* p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ double ld_d<__nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(__ldg(p));
}

template <class S>
__device__ __forceinline__ void crit_point(const CritArgs& a, int slot, int iy, int ix, double& g, double& H) {
  const S* f = reinterpret_cast<const S*>(a.f);
  const int k = a.owner[iy * a.n + ix];
  g = ld_d<S>(f + (long)k * a.ns + slot);
  const double h = ld_d<S>(f + ((long)a.nv + k) * a.ns + slot);
  const double x = a.xi[k], y = a.xi[a.nv + k];
  H = h + (x * x + y * y) * g;
}

// Eq. merge-transport-error on the base nodes of the candidate block, against the merged
// cell of the block (summed weight, weight-averaged coordinate, aggregated g and H).
template <class S>
__device__ bool crit_transport_ok(const CritCtx& c, int xa, int xb, int ya, int yb) {
  const CritArgs& a = *c.a;
  double wsum = 0, sxw = 0, syw = 0, sg = 0, sH = 0;
  double F[2][2][4];
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int r = 0; r < 4; ++r) F[d][s][r] = 0.0;
  for (int iy = ya; iy < yb; ++iy)
    for (int ix = xa; ix < xb; ++ix) {
      double g, H;
      crit_point<S>(a, c.slot, iy, ix, g, H);
      const double x = a.bx[ix], y = a.bx[iy], w = a.bw[iy] * a.bw[ix];
      const double x2 = x * x + y * y;
      const double hi = H - x2 * g;                 // h inherited at the base node
      const double m[4] = {g, x * g, y * g, 0.5 * (hi + x2 * g)};
      wsum += w; sxw += w * x; syw += w * y; sg += w * g; sH += w * (hi + x2 * g);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const double xd = d ? y : x;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (xd >= 0.0) F[d][0][r] += w * xd * m[r];
          if (xd <= 0.0) F[d][1][r] += w * xd * m[r];
        }
      }
    }
  const double xbar = sxw / wsum, ybar = syw / wsum;
  const double gb = sg / wsum, Hb = sH / wsum;
  const double xb2 = xbar * xbar + ybar * ybar;
  const double hb = Hb - xb2 * gb;
  const double mb[4] = {gb, xbar * gb, ybar * gb, 0.5 * (hb + xb2 * gb)};
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const double xd = d ? ybar : xbar;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const bool on = (s == 0) ? (xd >= 0.0) : (-xd >= 0.0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double Ft = on ? wsum * xd * mb[r] : 0.0;
        if (!(fabs(F[d][s][r] - Ft) <= c.epsSr[r])) return false;
      }
    }
  }
  return true;
}

// The same test from the per-block sums of the member blocks.  The centre node is a group of
// its own at every level, so a candidate block lies entirely on one side of xi_d = 0 in each
// axis or is the centre group: the one-sided sums of the test are the block's own sums (on the
// block's side, both sides for the centre group) or zero.  sum w and sum w xi_d are products
// of one-axis sums over the block's group ranges; sum w g and sum w H are the block's s1, s2.
__device__ inline bool crit_transport_blocks(const CritCtx& c, int bxa, int bxb, int bya, int byb, double s1,
                                             double s2) {
  const CritArgs& a = *c.a;
  const int nb = a.N1 * a.N1, mid = a.N1 / 2;   // the centre group has x = 0
  double w0x = 0, w1x = 0, w0y = 0, w1y = 0;
  for (int bx = bxa; bx < bxb; ++bx) { w0x += a.W1[bx]; w1x += a.X1[bx]; }
  for (int by = bya; by < byb; ++by) { w0y += a.W1[by]; w1y += a.X1[by]; }
  double t[CB_N];
#pragma unroll
  for (int r = 0; r < CB_N; ++r) t[r] = 0.0;
  for (int by = bya; by < byb; ++by)
    for (int bx = bxa; bx < bxb; ++bx) {
      const int b = by * a.N1 + bx;
#pragma unroll
      for (int r = 0; r < CB_N; ++r) t[r] += c.TB[r * nb + b];
    }
  const double wsum = w0x * w0y, sxw = w1x * w0y, syw = w0x * w1y;
  const double mx[4] = {t[CB_XG], t[CB_XXG], t[CB_XYG], 0.5 * t[CB_XH]};
  const double my[4] = {t[CB_YG], t[CB_XYG], t[CB_YYG], 0.5 * t[CB_YH]};
  // side s = 0 holds the members with xi_d >= 0 (group index >= mid), s = 1 those with xi_d <= 0
  const bool in[2][2] = {{bxb - 1 >= mid, bxa <= mid}, {byb - 1 >= mid, bya <= mid}};
  const double iw = 1.0 / wsum;
  const double xbar = sxw * iw, ybar = syw * iw;
  const double gb = s1 * iw, Hb = s2 * iw;
  const double xb2 = xbar * xbar + ybar * ybar;
  const double hb = Hb - xb2 * gb;
  const double mb[4] = {gb, xbar * gb, ybar * gb, 0.5 * (hb + xb2 * gb)};
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const double xd = d ? ybar : xbar;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const bool on = (s == 0) ? (xd >= 0.0) : (-xd >= 0.0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double F = in[d][s] ? (d ? my[r] : mx[r]) : 0.0;
        const double Ft = on ? wsum * xd * mb[r] : 0.0;
        if (!(fabs(F - Ft) <= c.epsSr[r])) return false;
      }
    }
  }
  return true;
}

template <class S>
__device__ bool crit_decide(const CritCtx& c, int L, int px, int py) {
  const CritArgs& a = *c.a;
  const int* P = a.pstart + L * (a.N1 + 1);
  const int bxa = P[px], bxb = P[px + 1], bya = P[py], byb = P[py + 1];
  double s1 = 0.0, s2 = 0.0;
  for (int by = bya; by < byb; ++by)
    for (int bx = bxa; bx < bxb; ++bx) {
      s1 += c.S1[by * a.N1 + bx];
      s2 += c.S2[by * a.N1 + bx];
    }
  // I_B = max(s1/T1, s2/T2) against the thresholds, as products
  if (s1 < a.C_merge * c.T1 && s2 < a.C_merge * c.T2) {
    if (!(a.eps > 0.0)) return true;
    if (a.tblk) return crit_transport_blocks(c, bxa, bxb, bya, byb, s1, s2);
    return crit_transport_ok<S>(c, a.g1[bxa], a.g1[bxb], a.g1[bya], a.g1[byb]);
  }
  if (s1 <= a.C_split * c.T1 && s2 <= a.C_split * c.T2) {
    for (int by = bya; by < byb; ++by)
      for (int bx = bxa; bx < bxb; ++bx)
        if (a.kprev[by * a.N1 + bx] < L) return false;
    return true;
  }
  return false;
}

__device__ __forceinline__ void crit_fill(const CritCtx& c, int L, int px, int py, unsigned char val) {
  const CritArgs& a = *c.a;
  const int* P = a.pstart + L * (a.N1 + 1);
  for (int by = P[py]; by < P[py + 1]; ++by)
    for (int bx = P[px]; bx < P[px + 1]; ++bx) c.out[by * a.N1 + bx] = val;
}

template <class S, int L>
__device__ void crit_scan(const CritCtx& c, int px, int py) {
  if (crit_decide<S>(c, L, px, py)) { crit_fill(c, L, px, py, (unsigned char)L); return; }
  if constexpr (L == 1) {
    crit_fill(c, 1, px, py, 0);
  } else {
    const int* C = c.a->cstart + L * (c.a->N1 + 1);
    for (int qy = C[py]; qy < C[py + 1]; ++qy)
      for (int qx = C[px]; qx < C[px + 1]; ++qx) crit_scan<S, L - 1>(c, qx, qy);
  }
}

template <class S>
__global__ void __launch_bounds__(CRIT_THREADS) k_criterion(const CritArgs a) {
  extern __shared__ __align__(16) double csm[];
  const int nb = a.N1 * a.N1;
  double* S1 = csm;
  double* S2 = csm + nb;
  __shared__ double red[10][CRIT_THREADS / 32];
  const int slot = a.sel ? a.sel[a.sel0 + blockIdx.x] : a.sel0 + (int)blockIdx.x;
  const int tid = threadIdx.x;
  // [CB_N][nb] per-block transport sums: shared memory, or this CTA's slice of the scratch
  double* TB = a.tblk == 2 ? a.TBg + (size_t)blockIdx.x * CB_N * nb : csm + 2 * nb;
  // level-1 block sums of w g and w H (and of the transport moments) on the base grid
  for (int b = tid; b < nb; b += CRIT_THREADS) {
    const int by = b / a.N1, bx = b % a.N1;
    double s1 = 0.0, s2 = 0.0;
    double t[CB_N];
#pragma unroll
    for (int r = 0; r < CB_N; ++r) t[r] = 0.0;
    const int ixa = a.g1[bx], ixb = a.g1[bx + 1] - 1, iya = a.g1[by], iyb = a.g1[by + 1] - 1;
    const int k0 = a.owner[iya * a.n + ixa];
    if (k0 == a.owner[iyb * a.n + ixb]) {
      // the block lies inside point k0: inherited g and H times the geometric sums
      double g, H;
      crit_point<S>(a, slot, iya, ixa, g, H);
      const double W = a.W1[bx] * a.W1[by];
      s1 = g * W;
      s2 = H * W;
      if (a.tblk) {
        const double xW = a.X1[bx] * a.W1[by], yW = a.W1[bx] * a.X1[by];
        t[CB_XG] = g * xW;
        t[CB_YG] = g * yW;
        t[CB_XXG] = g * (a.XX1[bx] * a.W1[by]);
        t[CB_XYG] = g * (a.X1[bx] * a.X1[by]);
        t[CB_YYG] = g * (a.W1[bx] * a.XX1[by]);
        t[CB_XH] = H * xW;
        t[CB_YH] = H * yW;
      }
    } else
    for (int iy = a.g1[by]; iy < a.g1[by + 1]; ++iy)
      for (int ix = a.g1[bx]; ix < a.g1[bx + 1]; ++ix) {
        double g, H;
        crit_point<S>(a, slot, iy, ix, g, H);
        const double w = a.bw[iy] * a.bw[ix];
        const double wg = w * g, wH = w * H;
        s1 += wg;
        s2 += wH;
        if (a.tblk) {
          const double x = a.bx[ix], y = a.bx[iy];
          t[CB_XG] += x * wg;
          t[CB_YG] += y * wg;
          t[CB_XXG] += x * x * wg;
          t[CB_XYG] += x * y * wg;
          t[CB_YYG] += y * y * wg;
          t[CB_XH] += x * wH;
          t[CB_YH] += y * wH;
        }
      }
    S1[b] = s1;
    S2[b] = s2;
    if (a.tblk)
#pragma unroll
      for (int r = 0; r < CB_N; ++r) TB[r * nb + b] = t[r];
  }
  __syncthreads();
  // totals, and S_r = max_d sum w |xi_d| |m_r| over the base grid for the transport test:
  // per point of the cell's space, |g| and |H| times the geometric sums of its rectangle
  double v[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) v[r] = 0.0;
  for (int b = tid; b < nb; b += CRIT_THREADS) { v[0] += S1[b]; v[1] += S2[b]; }
  if (a.eps > 0.0) {
    const S* f = reinterpret_cast<const S*>(a.f);
    for (int k = tid; k < a.nv; k += CRIT_THREADS) {
      const double g = ld_d<S>(f + (long)k * a.ns + slot);
      const double h = ld_d<S>(f + ((long)a.nv + k) * a.ns + slot);
      const double x = a.xi[k], y = a.xi[a.nv + k];
      const double ag = fabs(g), aH = fabs(h + (x * x + y * y) * g);
      const double Ax = a.geo[k], Ay = a.geo[a.nv + k], Bx = a.geo[2 * a.nv + k];
      const double By = a.geo[3 * a.nv + k], Cxy = a.geo[4 * a.nv + k];
      v[2] += ag * Ax;  v[3] += ag * Bx;  v[4] += ag * Cxy; v[5] += 0.5 * aH * Ax;
      v[6] += ag * Ay;  v[7] += ag * Cxy; v[8] += ag * By;  v[9] += 0.5 * aH * Ay;
    }
  }
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    double x = v[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0) red[r][tid >> 5] = x;
  }
  __syncthreads();
  CritCtx c;
  c.a = &a;
  c.S1 = S1;
  c.S2 = S2;
  c.TB = TB;
  double tot[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    double x = 0.0;
    for (int w = 0; w < CRIT_THREADS / 32; ++w) x += red[r][w];
    tot[r] = x;
  }
  c.T1 = tot[0];
  c.T2 = tot[1];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    c.Sr[r] = fmax(tot[2 + r], tot[6 + r]);
    c.epsSr[r] = a.eps * c.Sr[r];
  }
  c.slot = slot;
  c.out = a.kout + (long)a.ids[slot] * nb;
  // hierarchical scan, one thread per top-level candidate block
  const int L = a.max_level;
  const int ngL = a.ng[L];
  for (int q = tid; q < ngL * ngL; q += CRIT_THREADS) {
    const int py = q / ngL, px = q % ngL;
    if (L == 3) crit_scan<S, 3>(c, px, py);
    else if (L == 2) crit_scan<S, 2>(c, px, py);
    else crit_scan<S, 1>(c, px, py);
  }
}

}  // namespace mlvs
