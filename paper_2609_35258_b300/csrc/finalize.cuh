// Point finalisation: from velocity-chunk partial moments to the model parameters of a cell
// or a face, including the four-moment compatibility correction (Sec. 3.3.1).
//
// One warp per point.  The chunk partials are summed in chunk order (deterministic), the
// macroscopic state follows Eq. discrete_W / discrete_q (cells) or Eq. W_from_bar (faces),
// and the correction sums of Eq. joint_gh_correction_matrix / Eq. linear_moment_defect run
// over the velocities with the same per-velocity evaluation (model_eval, compute type T)
// that the tile kernels use, so the corrected model distribution they evaluate carries the
// target moments up to the rounding of its own arithmetic.
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
  int npt;              // number of points
  int is_face;          // 0: cells, 1: faces
  const void* cprm;     // [NP][ncell] current cell params (T): shift source
  void* prm_out;        // [NP][npt] (T)
  double* W;            // cells: [8][ncell] rho,u,v,T,qx,qy,rhoE,tau (may be null for faces)
  const void* vt;       // [4][nv] (T)
  int compat;
  double wall[4][3];    // (u_w, v_w, T_w)
  int* err;             // device error bits
};

enum { ERR_NONFINITE = 1, ERR_POSITIVITY = 2, ERR_SINGULAR = 4 };

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Gaussian elimination with partial pivoting, n <= 4.  Returns false if singular.
__device__ inline bool solve_small(double A[4][4], double b[4], int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(A[c][c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > best) { best = fabs(A[r][c]); p = r; }
    if (!(best > 1e-300)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
      double t = b[c]; b[c] = b[p]; b[p] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r][c] / A[c][c];
      for (int j = c; j < n; ++j) A[r][j] -= f * A[c][j];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int j = c + 1; j < n; ++j) s -= A[c][j] * b[j];
    b[c] = s / A[c][c];
  }
  return true;
}

// Model parameters of a point with state (rho, u, T, q) and compatibility coefficients.
// All lanes of the warp call this with identical arguments; every lane returns the same mp.
template <class T, int D>
__device__ inline bool point_model(const PointArgs& a, double rho, double ux, double uy, double Tm,
                                   double qx, double qy, MP<T>& mp) {
  const GasDev& g = a.gas;
  const double RT = g.R * Tm;
  const double p = rho * RT;
  const double kap = (1.0 - g.Pr) / (5.0 * p * RT);
  mp.ux = T(ux); mp.uy = T(uy);
  mp.lnn = T(log(rho) - 0.5 * D * log(2.0 * 3.14159265358979323846 * RT));
  mp.inv2RT = T(0.5 / RT);
  mp.kqx = T(kap * qx); mp.kqy = T(kap * qy);
  mp.RT = T(RT);
  mp.p0 = T(1); mp.a1 = T(0); mp.a2 = T(0); mp.p3 = T(0);
  if (!a.compat) return true;
  // correction sums (Eq. joint_gh_correction_matrix and Eq. linear_moment_defect)
  const T* vt = reinterpret_cast<const T*>(a.vt);
  const int nv = a.k.nv;
  const T c0 = T(a.k.c0), twoK = T(a.k.twoK);
  KSum<T> s0, s1, s2, e3;        // sum w g, w xi_x g, w xi_y g, 1/2 w (xi^2 g + h)
  s0.zero(); s1.zero(); s2.zero(); e3.zero();
  T sg[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // indices 3..9 used
  T sh[4] = {0, 0, 0, 0};                     // indices 1..3 used
  const int lane = threadIdx.x & 31;
  for (int v = lane; v < nv; v += 32) {
    const T xx = vt[v], yy = (D == 2) ? vt[nv + v] : T(0), w = vt[2 * nv + v], x2 = vt[3 * nv + v];
    T gv, hv;
    model_eval<T, D>(mp, xx, yy, x2, c0, twoK, gv, hv);
    const T wg = w * gv, wh = w * hv;
    s0.add(wg);
    s1.add(wg * xx);
    s2.add(wg * yy);
    e3.add(T(0.5) * (x2 * wg + wh));
    sg[3] += wg * x2;
    sg[4] += wg * xx * xx;
    sg[5] += wg * xx * yy;
    sg[6] += wg * yy * yy;
    sg[7] += wg * xx * x2;
    sg[8] += wg * yy * x2;
    sg[9] += wg * x2 * x2;
    sh[1] += wh * xx;
    sh[2] += wh * yy;
    sh[3] += wh * x2;
  }
  double S0 = warp_sum(s0.val()), S1 = warp_sum(s1.val()), S2 = warp_sum(s2.val());
  double E3 = warp_sum(e3.val());
  double G[10], H[4];
  for (int i = 3; i < 10; ++i) G[i] = warp_sum((double)sg[i]);
  for (int i = 1; i < 4; ++i) H[i] = warp_sum((double)sh[i]);
  const double hc = 0.5 * a.k.c0 * RT;   // 1/2 (3-D+K) R T of E_xi
  // rows: kernels (g, xi_x g, xi_y g, 1/2(xi^2 g + h)); columns: basis (1, xi_x, xi_y, E_xi)
  double A[4][4], b[4];
  const double rhoE = rho * (0.5 * (ux * ux + uy * uy) + 0.5 * (3.0 + g.K) * g.R * Tm);
  if (D == 2) {
    A[0][0] = S0; A[0][1] = S1;   A[0][2] = S2;   A[0][3] = hc * S0 + 0.5 * G[3];
    A[1][0] = S1; A[1][1] = G[4]; A[1][2] = G[5]; A[1][3] = hc * S1 + 0.5 * G[7];
    A[2][0] = S2; A[2][1] = G[5]; A[2][2] = G[6]; A[2][3] = hc * S2 + 0.5 * G[8];
    A[3][0] = E3; A[3][1] = 0.5 * (G[7] + H[1]); A[3][2] = 0.5 * (G[8] + H[2]);
    A[3][3] = hc * E3 + 0.25 * (G[9] + H[3]);
    b[0] = rho - S0; b[1] = rho * ux - S1; b[2] = rho * uy - S2; b[3] = rhoE - E3;
    if (!solve_small(A, b, 4)) return false;
    mp.p0 = T(1.0 + b[0] + b[3] * hc);
    mp.a1 = T(b[1]); mp.a2 = T(b[2]); mp.p3 = T(0.5 * b[3]);
  } else {
    A[0][0] = S0; A[0][1] = S1;   A[0][2] = hc * S0 + 0.5 * G[3];
    A[1][0] = S1; A[1][1] = G[4]; A[1][2] = hc * S1 + 0.5 * G[7];
    A[2][0] = E3; A[2][1] = 0.5 * (G[7] + H[1]); A[2][2] = hc * E3 + 0.25 * (G[9] + H[3]);
    b[0] = rho - S0; b[1] = rho * ux - S1; b[2] = rhoE - E3;
    if (!solve_small(A, b, 3)) return false;
    mp.p0 = T(1.0 + b[0] + b[2] * hc);
    mp.a1 = T(b[1]); mp.a2 = T(0); mp.p3 = T(0.5 * b[2]);
  }
  return true;
}

template <class T>
__device__ __forceinline__ void store_mp(T* P, long n, long i, const MP<T>& m, T kind) {
  P[P_UX * n + i] = m.ux; P[P_UY * n + i] = m.uy; P[P_LNN * n + i] = m.lnn;
  P[P_INV2RT * n + i] = m.inv2RT; P[P_KQX * n + i] = m.kqx; P[P_KQY * n + i] = m.kqy;
  P[P_RT * n + i] = m.RT; P[P_P0 * n + i] = m.p0; P[P_A1 * n + i] = m.a1;
  P[P_A2 * n + i] = m.a2; P[P_P3 * n + i] = m.p3; P[P_C1 * n + i] = m.c1;
  P[P_C2 * n + i] = m.c2; P[P_KIND * n + i] = kind;
}

__device__ __forceinline__ int wrap_or_clamp_h(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Cells (is_face = 0): Eq. discrete_W, Eq. discrete_q, tau = mu(T)/p, blending of phi-bar-plus.
// Faces (is_face = 1): Eq. W_from_bar, q = 2 tau/(2 tau + s Pr) q-bar, Eq. recover_phi weights;
// wall faces: rho_w from the zero net normal mass flux.
template <class T, int D>
__global__ void k_finalize(const PointArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const StepConst& k = a.k;
  const T* cp = reinterpret_cast<const T*>(a.cprm);
  T* po = reinterpret_cast<T*>(a.prm_out);
  const long nc = k.ncell;
  for (int i = warp; i < a.npt; i += nwarps) {
    // chunk sums in chunk order: lane m sums moment m
    double mom = 0.0;
    if (lane < NMOM)
      for (int c = 0; c < k.nchunk; ++c) mom += a.part[((long)c * NMOM + lane) * a.npt + i];
    double M[NMOM];
#pragma unroll
    for (int m = 0; m < NMOM; ++m) M[m] = __shfl_sync(0xffffffffu, mom, m);

    // shift and face kind
    T shx, shy;
    int kind = FK_INTERIOR;
    int side = -1;
    if (!a.is_face) {
      shx = cp[P_UX * nc + i];
      shy = cp[P_UY * nc + i];
    } else {
      int sL, sR;
      const int nxf = k.nfx * k.ny;
      if (i < nxf) {
        const int gj = i / k.nfx, gi = i % k.nfx;
        sL = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + wrap_or_clamp_h(gi - 1, k.nx, k.px);
        sR = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + wrap_or_clamp_h(gi, k.nx, k.px);
        if (!k.px && gi == 0 && k.bc[0] == BC_WALL) { kind = FK_WALL_LO; side = 0; }
        if (!k.px && gi == k.nx && k.bc[1] == BC_WALL) { kind = FK_WALL_HI; side = 1; }
      } else {
        const int r = i - nxf;
        const int gj = r / k.nx, gi = r % k.nx;
        sL = wrap_or_clamp_h(gj - 1, k.ny, k.py) * k.nx + gi;
        sR = wrap_or_clamp_h(gj, k.ny, k.py) * k.nx + gi;
        if (!k.py && gj == 0 && k.bc[2] == BC_WALL) { kind = FK_WALL_LO; side = 2; }
        if (!k.py && gj == k.ny && k.bc[3] == BC_WALL) { kind = FK_WALL_HI; side = 3; }
      }
      shx = T(0.5) * (cp[P_UX * nc + sL] + cp[P_UX * nc + sR]);
      shy = (D == 2) ? T(0.5) * (cp[P_UY * nc + sL] + cp[P_UY * nc + sR]) : T(0);
    }
    const GasDev& g = a.gas;
    MP<T> mp;
    if (kind != FK_INTERIOR) {
      // diffuse wall: unit-density wall Maxwellian, rho_w = -M_out / den
      const double uw = a.wall[side][0], vw = a.wall[side][1], Tw = a.wall[side][2];
      const double RT = g.R * Tw;
      mp.ux = T(uw); mp.uy = T(vw);
      mp.lnn = T(-0.5 * D * log(2.0 * 3.14159265358979323846 * RT));
      mp.inv2RT = T(0.5 / RT); mp.kqx = T(0); mp.kqy = T(0); mp.RT = T(RT);
      mp.p0 = T(1); mp.a1 = T(0); mp.a2 = T(0); mp.p3 = T(0);
      const T* vt = reinterpret_cast<const T*>(a.vt);
      const int nv = k.nv;
      const bool xdir = (side < 2);
      const T sgn = (kind == FK_WALL_LO) ? T(1) : T(-1);
      KSum<T> den;
      den.zero();
      for (int v = lane; v < nv; v += 32) {
        const T xx = vt[v], yy = (D == 2) ? vt[nv + v] : T(0);
        const T xin = sgn * (xdir ? xx : yy);
        if (xin > T(0)) {
          T gv, hv;
          model_eval<T, D>(mp, xx, yy, vt[3 * nv + v], T(k.c0), T(k.twoK), gv, hv);
          den.add(vt[2 * nv + v] * xin * gv);
        }
      }
      const double dsum = warp_sum(den.val());
      const double rw = -M[MO_0] / dsum;
      mp.c1 = T(0);
      mp.c2 = T(rw);
      if (lane == 0) {
        store_mp<T>(po, a.npt, i, mp, T(kind));
        po[P_SHX * (long)a.npt + i] = shx;
        po[P_SHY * (long)a.npt + i] = shy;
        if (!(rw >= 0.0) || !isfinite(rw)) atomicOr(a.err, ERR_POSITIVITY);
      }
      continue;
    }
    const double rho = M[MO_0];
    const double upx = M[MO_X] / rho, upy = (D == 2) ? M[MO_Y] / rho : 0.0;
    const double u2 = upx * upx + upy * upy;
    const double ux = (double)shx + upx, uy = (D == 2) ? (double)shy + upy : 0.0;
    const double Tm = (M[MO_E] - rho * u2) / ((3.0 + g.K) * rho * g.R);
    // q = 1/2 [J - 2 u'.G - u' E' + 2 rho |u'|^2 u']  in the shifted frame
    double qx = 0.5 * (M[MO_JX] - 2.0 * (upx * M[MO_GXX] + upy * M[MO_GXY]) - upx * M[MO_E] + 2.0 * rho * u2 * upx);
    double qy = (D == 2) ? 0.5 * (M[MO_JY] - 2.0 * (upx * M[MO_GXY] + upy * M[MO_GYY]) - upy * M[MO_E] + 2.0 * rho * u2 * upy) : 0.0;
    const double p = rho * g.R * Tm;
    const double mu = g.mu_ref * pow(Tm / g.T_ref, g.omega);
    const double tau = mu / p;
    const double hdt = a.is_face ? 0.5 * k.dt : k.dt;    // dt at cells, s at faces
    const double qf = 2.0 * tau / (2.0 * tau + hdt * g.Pr);
    qx *= qf;
    qy *= qf;
    bool ok = point_model<T, D>(a, rho, ux, uy, Tm, qx, qy, mp);
    const double s = 0.5 * k.dt;
    if (!a.is_face) {
      mp.c1 = T((2.0 * tau - s) / (2.0 * tau + k.dt));
      mp.c2 = T(3.0 * s / (2.0 * tau + k.dt));
    } else {
      mp.c1 = T(2.0 * tau / (2.0 * tau + s));
      mp.c2 = T(s / (2.0 * tau + s));
    }
    if (lane == 0) {
      store_mp<T>(po, a.npt, i, mp, T(kind));
      po[P_SHX * (long)a.npt + i] = shx;
      po[P_SHY * (long)a.npt + i] = shy;
      if (a.W) {
        a.W[0 * nc + i] = rho;
        a.W[1 * nc + i] = ux;
        a.W[2 * nc + i] = uy;
        a.W[3 * nc + i] = Tm;
        a.W[4 * nc + i] = qx;
        a.W[5 * nc + i] = qy;
        a.W[6 * nc + i] = rho * (0.5 * (ux * ux + uy * uy) + 0.5 * (3.0 + g.K) * g.R * Tm);
        a.W[7 * nc + i] = tau;
      }
      if (!ok) atomicOr(a.err, ERR_SINGULAR);
      if (!isfinite(rho) || !isfinite(Tm) || !isfinite(ux) || !isfinite(uy)) atomicOr(a.err, ERR_NONFINITE);
      else if (!(rho > 0.0) || !(Tm > 0.0)) atomicOr(a.err, ERR_POSITIVITY);
    }
  }
}

// Initial parameters from (rho, u, v, T) with q = 0 (phi~ = phi^eq at t = 0).
template <class T, int D>
__global__ void k_init_params(const PointArgs a, const double* W0 /* [ncell][4] */) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  T* po = reinterpret_cast<T*>(a.prm_out);
  for (int i = warp; i < a.npt; i += nwarps) {
    const double rho = W0[4 * i], ux = W0[4 * i + 1], uy = (D == 2) ? W0[4 * i + 2] : 0.0, Tm = W0[4 * i + 3];
    MP<T> mp;
    bool ok = point_model<T, D>(a, rho, ux, uy, Tm, 0.0, 0.0, mp);
    mp.c1 = T(1); mp.c2 = T(0);
    if (lane == 0) {
      store_mp<T>(po, a.npt, i, mp, T(0));
      if (!ok) atomicOr(a.err, ERR_SINGULAR);
    }
  }
}

// phi~ = corrected Maxwellian of the initial parameters, and the chunk partial moments.
template <class S, class T, int D>
__global__ void k_init_f(StepConst k, const T* __restrict__ prm, const T* __restrict__ vt,
                         S* __restrict__ f) {
  const long nc = k.ncell;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  MP<T> m;
  m.load(prm, nc, c);
  const T c0 = T(k.c0), twoK = T(k.twoK);
  for (int v = blockIdx.y; v < k.nv; v += gridDim.y) {
    T g, h;
    model_eval<T, D>(m, vt[v], (D == 2) ? vt[k.nv + v] : T(0), vt[3 * k.nv + v], c0, twoK, g, h);
    stf<S, T>(f + (long)v * nc + c, g);
    stf<S, T>(f + ((long)k.nv + v) * nc + c, h);
  }
}

// Chunk partial moments of f in the frame of the cell velocity in prm (used after init).
template <class S, class T, int D>
__global__ void k_moments(StepConst k, const T* __restrict__ prm, const T* __restrict__ vt,
                          const S* __restrict__ f, double* __restrict__ part) {
  const long nc = k.ncell;
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
    const T wv = vt[2 * nv + v];
    const T wg = wv * gq;
    const T e = wv * ((xp * xp + yp * yp) * gq + hq);
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
