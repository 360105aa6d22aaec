// Tile kernels of one DUGKS step on a structured Cartesian mesh (Sec. 2.2).
//
// A CTA owns a TX x TY tile of cells and a contiguous chunk of velocities.  For each
// velocity it stages phi-bar-plus of the tile and a two-cell halo in shared memory
// (Sec. 2.2, derived conversion phi-bar-plus = C1 phi~ + C2 phi^S), limited slopes
// (Eq. reconstruction), and the face phi-bar of every face of the tile by the
// characteristic (Eq. bar_phi_transport).  MODE 0 accumulates the face moments over the
// chunk (input of Eq. W_from_bar); MODE 1 recovers the face phi (Eq. recover_phi), applies
// Eq. explicit_update to the tile's cells, stores phi~^{n+1} and accumulates the cell moments
// of the new phi~ (input of Eq. discrete_W / discrete_q of the next step).
//
// Velocity is uniform across the CTA inside the loop, so the upwind choice by sign(xi.n)
// is a uniform branch.  Halo sources are wrapped (periodic sides) or clamped (ghost copies
// of the boundary cell on the other sides).
#pragma once
#include "mlvs_common.cuh"

namespace mlvs {

struct TileArgs {
  StepConst k;
  const void* f_in;      // [2][nv][ncell]
  void* f_out;           // [2][nv][ncell] (MODE 1)
  const void* cparam;    // [NP][ncell]  type T
  const void* fparam;    // [NP][nface]  type T (MODE 1)
  const void* vt;        // [4][nv]      type T
  double* part;          // MODE 0: [nchunk][NMOM][nface], MODE 1: [nchunk][NMOM][ncell]
  int ntx, nty;          // tiles per axis
};

template <int TX, int TY, int D> struct TileGeom {
  static constexpr int NT = TX * TY;
  static constexpr int EW = TX + 4;
  static constexpr int EH = (D == 2) ? TY + 4 : 1;
  static constexpr int NEXT = EW * EH;
  static constexpr int NHALO = NEXT - NT;
  static constexpr int SW = TX + 2;
  static constexpr int SH = (D == 2) ? TY + 2 : 1;
  static constexpr int NSL = SW * SH;
  static constexpr int NFXL = (TX + 1) * TY;
  static constexpr int NFYL = (D == 2) ? TX * (TY + 1) : 0;
  // ext index of tile-local cell (x, y), x in [-2, TX+1], y in [-2, TY+1]
  static __device__ __forceinline__ int eidx(int x, int y) {
    return (D == 2) ? (y + 2) * EW + (x + 2) : (x + 2);
  }
  // slope index of tile-local cell (x, y), x in [-1, TX], y in [-1, TY]
  static __device__ __forceinline__ int sidx(int x, int y) {
    return (D == 2) ? (y + 1) * SW + (x + 1) : (x + 1);
  }
  // k-th halo position of the extended tile
  static __device__ __forceinline__ void halo_pos(int k, int& x, int& y) {
    if (D == 1) {
      const int cols[4] = {-2, -1, TX, TX + 1};
      x = cols[k];
      y = 0;
      return;
    }
    if (k < 2 * EW) { y = k / EW - 2; x = k % EW - 2; return; }
    k -= 2 * EW;
    if (k < 2 * EW) { y = TY + k / EW; x = k % EW - 2; return; }
    k -= 2 * EW;
    y = k / 4;
    const int c = k % 4;
    x = (c == 0) ? -2 : (c == 1) ? -1 : (c == 2) ? TX : TX + 1;
  }
};

__device__ __forceinline__ int wrap_or_clamp(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// van Leer limited slope (reading of Eq. reconstruction): 2ab/(a+b)/h for a, b of equal
// strict sign, else 0.  limiter == 1: central difference (a+b)/(2h).
template <class T>
__device__ __forceinline__ T limited(T a, T b, T inv_h, int limiter) {
  if (limiter) return T(0.5) * (a + b) * inv_h;
  const bool same = (a > T(0) && b > T(0)) || (a < T(0) && b < T(0));
  return same ? Num<T>::dv(T(2) * a * b, a + b) * inv_h : T(0);
}

// Face descriptor held per thread.
struct FaceRef {
  int dir;     // 0: x-face, 1: y-face, -1: none
  int li, lj;  // tile-local face coordinates
  int fid;     // global face index (param / partial row), -1: invalid
  int owned;   // MODE 0: accumulate into partials
  int kind;    // FK_*
};

template <class S, class T, int D, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY)
k_tile(const TileArgs a, int limiter) {
  using G = TileGeom<TX, TY, D>;
  static_assert(G::NHALO <= G::NT, "halo larger than the thread count");
  static_assert(G::NSL <= 2 * G::NT, "slope rectangle larger than two per thread");
  static_assert(TY + ((D == 2) ? TX : 0) <= G::NT, "edge faces larger than the thread count");
  const StepConst& k = a.k;
  __shared__ T sPg[2][G::NEXT];
  __shared__ T sPh[2][G::NEXT];
  __shared__ T sSxg[G::NSL], sSxh[G::NSL];
  __shared__ T sSyg[(D == 2) ? G::NSL : 1], sSyh[(D == 2) ? G::NSL : 1];
  __shared__ T sFxg[(MODE == 1) ? G::NFXL : 1], sFxh[(MODE == 1) ? G::NFXL : 1];
  __shared__ T sFyg[(MODE == 1 && D == 2) ? G::NFYL : 1], sFyh[(MODE == 1 && D == 2) ? G::NFYL : 1];

  const S* __restrict__ fin = reinterpret_cast<const S*>(a.f_in);
  const T* __restrict__ cp = reinterpret_cast<const T*>(a.cparam);
  const T* __restrict__ fp = reinterpret_cast<const T*>(a.fparam);
  const T* __restrict__ vt = reinterpret_cast<const T*>(a.vt);
  const long nc = k.ncell;
  const long nv = k.nv;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int bx = blockIdx.x % a.ntx, by = blockIdx.x / a.ntx;
  const int x0 = bx * TX, y0 = by * TY;
  const int chunk = blockIdx.y;
  const int v0 = chunk * k.vpc;
  const int v1 = min(k.nv, v0 + k.vpc);

  // ---- extended positions handled by this thread: own cell + at most one halo cell
  const int ex0 = tx, ey0 = (D == 2) ? ty : 0;
  const int src0 = wrap_or_clamp(y0 + ey0, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + ex0, k.nx, k.px);
  const bool own_active = (x0 + tx < k.nx) && (D == 1 || y0 + ty < k.ny);
  const int own_cell = own_active ? (y0 + ty) * k.nx + (x0 + tx) : -1;
  int ex1 = 0, ey1 = 0, src1 = -1;
  if (tid < G::NHALO) {
    G::halo_pos(tid, ex1, ey1);
    src1 = wrap_or_clamp(y0 + ey1, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + ex1, k.nx, k.px);
  }
  MP<T> m0, m1;
  m0.load(cp, nc, src0);
  if (src1 >= 0) m1.load(cp, nc, src1);
  const int e0 = G::eidx(ex0, ey0);
  const int e1 = (src1 >= 0) ? G::eidx(ex1, ey1) : 0;

  // ---- slope positions: (TX+2) x (TY+2) rectangle from (-1,-1)
  int sl_n = 0;
  int sl_e[2], sl_s[2];
  for (int q = tid; q < G::NSL; q += G::NT) {
    const int sx = q % G::SW - 1, sy = (D == 2) ? q / G::SW - 1 : 0;
    sl_e[sl_n] = G::eidx(sx, sy);
    sl_s[sl_n] = q;
    ++sl_n;
  }

  // ---- faces handled by this thread
  FaceRef fr[3];
  int nfr = 0;
  {
    auto xface = [&](int li, int lj) {
      FaceRef r;
      r.dir = 0; r.li = li; r.lj = lj;
      const int gi = x0 + li, gj = y0 + lj;
      const bool valid = (gi <= k.nx) && (D == 1 || gj < k.ny);
      r.fid = -1; r.owned = 0; r.kind = FK_INTERIOR;
      if (valid) {
        const int pi = (k.px && gi == k.nx) ? 0 : gi;
        r.fid = ((D == 2) ? gj : 0) * k.nfx + pi;
        r.owned = (gi < k.nx) ? (li < TX) : !k.px;
        if (!k.px && gi == 0 && k.bc[0] == BC_WALL) r.kind = FK_WALL_LO;
        if (!k.px && gi == k.nx && k.bc[1] == BC_WALL) r.kind = FK_WALL_HI;
      }
      return r;
    };
    auto yface = [&](int li, int lj) {
      FaceRef r;
      r.dir = 1; r.li = li; r.lj = lj;
      const int gi = x0 + li, gj = y0 + lj;
      const bool valid = (gi < k.nx) && (gj <= k.ny);
      r.fid = -1; r.owned = 0; r.kind = FK_INTERIOR;
      if (valid) {
        const int pj = (k.py && gj == k.ny) ? 0 : gj;
        r.fid = k.nfx * k.ny + pj * k.nx + gi;
        r.owned = (gj < k.ny) ? (lj < TY) : !k.py;
        if (!k.py && gj == 0 && k.bc[2] == BC_WALL) r.kind = FK_WALL_LO;
        if (!k.py && gj == k.ny && k.bc[3] == BC_WALL) r.kind = FK_WALL_HI;
      }
      return r;
    };
    fr[nfr++] = xface(tx, ty);
    if (D == 2) fr[nfr++] = yface(tx, ty);
    if (tid < TY) fr[nfr++] = xface(TX, tid);
    else if (D == 2 && tid < TY + TX) fr[nfr++] = yface(tid - TY, TY);
  }
  // per-face data: shift (MODE 0) or model parameters (MODE 1)
  T fsx[3], fsy[3];
  MP<T> fm[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    fsx[q] = T(0); fsy[q] = T(0);
    if (q < nfr && fr[q].fid >= 0) {
      if (MODE == 0) {
        // shift = mean velocity of the two adjacent cells (sources as in the halo)
        int li = fr[q].li, lj = fr[q].lj;
        int xl = (fr[q].dir == 0) ? li - 1 : li, yl = (fr[q].dir == 0) ? lj : lj - 1;
        int sL = wrap_or_clamp(y0 + yl, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + xl, k.nx, k.px);
        int sR = wrap_or_clamp(y0 + lj, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + li, k.nx, k.px);
        fsx[q] = T(0.5) * (cp[P_UX * nc + sL] + cp[P_UX * nc + sR]);
        if (D == 2) fsy[q] = T(0.5) * (cp[P_UY * nc + sL] + cp[P_UY * nc + sR]);
      } else {
        fm[q].load(fp, k.nface, fr[q].fid);
      }
    }
  }

  // ---- accumulators
  KSum<T> acc0[3], accX[3], accY[3], accE[3];
  T acc[3][5];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    acc0[q].zero(); accX[q].zero(); accY[q].zero(); accE[q].zero();
#pragma unroll
    for (int r = 0; r < 5; ++r) acc[q][r] = T(0);
  }

  const T c0 = T(k.c0), twoK = T(k.twoK);
  const T s = T(0.5 * k.dt);
  const T hdx = T(0.5 * k.dx), hdy = T(0.5 * k.dy);
  const T idx_ = T(1.0 / k.dx), idy_ = T(1.0 / k.dy);
  const T lamx = T(k.dt / k.dx), lamy = T(k.dt / k.dy);
  S* __restrict__ fout = reinterpret_cast<S*>(a.f_out);

  // prefetch registers
  T g0n = T(0), h0n = T(0), g1n = T(0), h1n = T(0);
  if (v0 < v1) {
    g0n = ldf<S, T>(fin + (long)v0 * nc + src0);
    h0n = ldf<S, T>(fin + (nv + v0) * nc + src0);
    if (src1 >= 0) {
      g1n = ldf<S, T>(fin + (long)v0 * nc + src1);
      h1n = ldf<S, T>(fin + (nv + v0) * nc + src1);
    }
  }

  int par = 0;
  for (int v = v0; v < v1; ++v) {
    const T xix = vt[v], xiy = (D == 2) ? vt[nv + v] : T(0), wxv = vt[2 * nv + v], wyv = vt[3 * nv + v];
    const T g0 = g0n, h0 = h0n, g1 = g1n, h1 = h1n;
    if (v + 1 < v1) {
      g0n = ldf<S, T>(fin + (long)(v + 1) * nc + src0);
      h0n = ldf<S, T>(fin + (nv + v + 1) * nc + src0);
      if (src1 >= 0) {
        g1n = ldf<S, T>(fin + (long)(v + 1) * nc + src1);
        h1n = ldf<S, T>(fin + (nv + v + 1) * nc + src1);
      }
    }
    // ---- phase 1: phi-bar-plus on the extended tile
    // Written as phi~ + b (phi^S - phi~) so that the two blending weights sum to one exactly
    // whatever their rounding: the collision then conserves the moments of phi~.
    T dg0, dh0;
    {
      T gs, hs;
      model_eval<T, D>(m0, xix, xiy, c0, twoK, gs, hs);
      dg0 = gs - g0;
      dh0 = hs - h0;
      sPg[par][e0] = g0 + m0.c1 * dg0;
      sPh[par][e0] = h0 + m0.c1 * dh0;
      if (src1 >= 0) {
        model_eval<T, D>(m1, xix, xiy, c0, twoK, gs, hs);
        sPg[par][e1] = g1 + m1.c1 * (gs - g1);
        sPh[par][e1] = h1 + m1.c1 * (hs - h1);
      }
    }
    __syncthreads();
    // ---- phase 2: limited slopes
    for (int q = 0; q < sl_n; ++q) {
      const int e = sl_e[q], si = sl_s[q];
      const T* Pg = sPg[par];
      const T* Ph = sPh[par];
      sSxg[si] = limited(Pg[e + 1] - Pg[e], Pg[e] - Pg[e - 1], idx_, limiter);
      sSxh[si] = limited(Ph[e + 1] - Ph[e], Ph[e] - Ph[e - 1], idx_, limiter);
      if (D == 2) {
        sSyg[si] = limited(Pg[e + G::EW] - Pg[e], Pg[e] - Pg[e - G::EW], idy_, limiter);
        sSyh[si] = limited(Ph[e + G::EW] - Ph[e], Ph[e] - Ph[e - G::EW], idy_, limiter);
      }
    }
    __syncthreads();
    // ---- phase 3: faces
    {
      const T* Pg = sPg[par];
      const T* Ph = sPh[par];
      const T bx_ = -xix * s, by_ = -xiy * s;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= nfr || fr[q].fid < 0) continue;
        const int li = fr[q].li, lj = fr[q].lj;
        T gb, hb, xn;
        if (fr[q].dir == 0) {
          xn = xix;
          // left cell (li-1, lj), right cell (li, lj)
          const int eL = G::eidx(li - 1, lj), eR = G::eidx(li, lj);
          const int sL = G::sidx(li - 1, lj), sR = G::sidx(li, lj);
          T gL = Pg[eL] + (hdx + bx_) * sSxg[sL];
          T hL = Ph[eL] + (hdx + bx_) * sSxh[sL];
          T gR = Pg[eR] + (-hdx + bx_) * sSxg[sR];
          T hR = Ph[eR] + (-hdx + bx_) * sSxh[sR];
          if (D == 2) {
            gL += by_ * sSyg[sL]; hL += by_ * sSyh[sL];
            gR += by_ * sSyg[sR]; hR += by_ * sSyh[sR];
          }
          if (xix > T(0)) { gb = gL; hb = hL; }
          else if (xix < T(0)) { gb = gR; hb = hR; }
          else { gb = T(0.5) * (gL + gR); hb = T(0.5) * (hL + hR); }
        } else {
          xn = xiy;
          const int eS = G::eidx(li, lj - 1), eN = G::eidx(li, lj);
          const int sS = G::sidx(li, lj - 1), sN = G::sidx(li, lj);
          T gS_ = Pg[eS] + bx_ * sSxg[sS] + (hdy + by_) * sSyg[sS];
          T hS_ = Ph[eS] + bx_ * sSxh[sS] + (hdy + by_) * sSyh[sS];
          T gN = Pg[eN] + bx_ * sSxg[sN] + (-hdy + by_) * sSyg[sN];
          T hN = Ph[eN] + bx_ * sSxh[sN] + (-hdy + by_) * sSyh[sN];
          if (xiy > T(0)) { gb = gS_; hb = hS_; }
          else if (xiy < T(0)) { gb = gN; hb = hN; }
          else { gb = T(0.5) * (gS_ + gN); hb = T(0.5) * (hS_ + hN); }
        }
        if (MODE == 0) {
          if (!fr[q].owned) continue;
          if (fr[q].kind == FK_INTERIOR) {
            const T xp = xix - fsx[q], yp = (D == 2) ? xiy - fsy[q] : T(0);
            const T wg = wxv * (wyv * gb);
            const T e = wxv * (wyv * ((xp * xp + yp * yp) * gb + hb));
            acc0[q].add(wg);
            accX[q].add(wg * xp);
            accE[q].add(e);
            acc[q][0] += wg * xp * xp;
            acc[q][3] += e * xp;
            if (D == 2) {
              accY[q].add(wg * yp);
              acc[q][1] += wg * xp * yp;
              acc[q][2] += wg * yp * yp;
              acc[q][4] += e * yp;
            }
          } else {
            // wall: outgoing normal mass flux sum_{xi.n_in <= 0} w (xi.n_in) g-bar
            const T xin = (fr[q].kind == FK_WALL_LO) ? xn : -xn;
            if (xin <= T(0)) acc0[q].add(wxv * (wyv * (xin * gb)));
          }
        } else {
          T gf, hf;
          if (fr[q].kind == FK_INTERIOR) {
            T gs, hs;
            model_eval<T, D>(fm[q], xix, xiy, c0, twoK, gs, hs);
            gf = gb + fm[q].c2 * (gs - gb);     // Eq. recover_phi, weights summing to one
            hf = hb + fm[q].c2 * (hs - hb);
          } else {
            const T xin = (fr[q].kind == FK_WALL_LO) ? xn : -xn;
            if (xin > T(0)) {
              T gs, hs;
              model_eval<T, D>(fm[q], xix, xiy, c0, twoK, gs, hs);
              gf = fm[q].c2 * gs;
              hf = fm[q].c2 * hs;
            } else {
              gf = gb;
              hf = hb;
            }
          }
          if (fr[q].dir == 0) {
            sFxg[lj * (TX + 1) + li] = gf;
            sFxh[lj * (TX + 1) + li] = hf;
          } else {
            sFyg[lj * TX + li] = gf;
            sFyh[lj * TX + li] = hf;
          }
        }
      }
    }
    if (MODE == 1) {
      __syncthreads();
      // ---- phase 4: update of the tile's cells (Eq. explicit_update)
      if (own_active) {
        const int w_ = (D == 2) ? ty * (TX + 1) + tx : tx;
        // phi~+ = 4/3 phi-bar-plus - 1/3 phi~ = phi~ + (4/3) b (phi^S - phi~)
        T gn = g0 + m0.c2 * dg0 - lamx * xix * (sFxg[w_ + 1] - sFxg[w_]);
        T hn = h0 + m0.c2 * dh0 - lamx * xix * (sFxh[w_ + 1] - sFxh[w_]);
        if (D == 2) {
          const int sI = ty * TX + tx;
          gn -= lamy * xiy * (sFyg[sI + TX] - sFyg[sI]);
          hn -= lamy * xiy * (sFyh[sI + TX] - sFyh[sI]);
        }
        stf<S, T>(fout + (long)v * nc + own_cell, gn);
        stf<S, T>(fout + (nv + v) * nc + own_cell, hn);
        // moments of the stored value
        const T gq = ldf_round<S, T>(gn), hq = ldf_round<S, T>(hn);
        const T xp = xix - m0.ux, yp = (D == 2) ? xiy - m0.uy : T(0);
        const T wg = wxv * (wyv * gq);
        const T e = wxv * (wyv * ((xp * xp + yp * yp) * gq + hq));
        acc0[0].add(wg);
        accX[0].add(wg * xp);
        accE[0].add(e);
        acc[0][0] += wg * xp * xp;
        acc[0][3] += e * xp;
        if (D == 2) {
          accY[0].add(wg * yp);
          acc[0][1] += wg * xp * yp;
          acc[0][2] += wg * yp * yp;
          acc[0][4] += e * yp;
        }
      }
    } else {
      par ^= 1;
    }
  }

  // ---- write partial moments of this chunk
  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= nfr || fr[q].fid < 0 || !fr[q].owned) continue;
      double* P = a.part + (long)chunk * NMOM * k.nface + fr[q].fid;
      const long st = k.nface;
      P[MO_0 * st] = acc0[q].val();
      P[MO_X * st] = accX[q].val();
      P[MO_Y * st] = (D == 2) ? accY[q].val() : 0.0;
      P[MO_E * st] = accE[q].val();
      P[MO_GXX * st] = (double)acc[q][0];
      P[MO_GXY * st] = (double)acc[q][1];
      P[MO_GYY * st] = (double)acc[q][2];
      P[MO_JX * st] = (double)acc[q][3];
      P[MO_JY * st] = (double)acc[q][4];
    }
  } else if (own_active) {
    double* P = a.part + (long)chunk * NMOM * nc + own_cell;
    P[MO_0 * nc] = acc0[0].val();
    P[MO_X * nc] = accX[0].val();
    P[MO_Y * nc] = (D == 2) ? accY[0].val() : 0.0;
    P[MO_E * nc] = accE[0].val();
    P[MO_GXX * nc] = (double)acc[0][0];
    P[MO_GXY * nc] = (double)acc[0][1];
    P[MO_GYY * nc] = (double)acc[0][2];
    P[MO_JX * nc] = (double)acc[0][3];
    P[MO_JY * nc] = (double)acc[0][4];
  }
}

}  // namespace mlvs
