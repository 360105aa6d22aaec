// Shared device definitions of the MLVS-DUGKS library (sm_103a).
//
// Layouts (device memory, per instance and level):
//   f      [comp in {g~, h~}][v][cell]        storage type S (double | float | bf16), cells row-major
//   params [NP][point]                        compute type T, one point = a cell or a face
//   part   [chunk][NMOM][point]               double, per-velocity-chunk partial moments
//   vt     [4][v] = (xi_x, xi_y, w_x, w_y)    compute type T; the weight is w = w_x w_y and
//                                             every velocity sum forms w_x (w_y x), so the
//                                             rounding of the weight product never repeats
//                                             systematically over the velocities
//   ax     [2][n_axis] = (X, W)                compute type T, 1-D axis of a tensor-product space
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mlvs {

// Per-point parameters of the model distribution (Eq. g_h_eq_Pr with the compatibility
// correction of Eq. gh_model_correction folded in) plus two blending coefficients:
//   cells: C1 = b = 3 s/(2 tau + dt), C2 = 4 b / 3, with
//          phi-bar-plus = phi~ + b (phi^S - phi~),  phi~+ = phi~ + (4/3) b (phi^S - phi~)
//          (the derived conversions of Sec. 2.2 with their weights summing to one)
//   faces: C1 = 2 tau/(2 tau + s), C2 = s/(2 tau + s):  phi = phi-bar + C2 (phi^S - phi-bar)
//          (Eq. recover_phi)
//   wall faces: C2 + C1 = rho_w (high and low parts) multiplies the unit-density wall
//          Maxwellian.
// The correction factor is 1 + B0 + B1 c_x + B2 c_y + B3 |c|^2 with c = xi - u: the span of
// the basis of Eq. eq_four_basis {1, xi_x, xi_y, E_xi} written in peculiar velocity.
enum {
  P_UX = 0, P_UY, P_LNH, P_INV2RT, P_KQX, P_KQY, P_RT, P_B0, P_B1, P_B2, P_B3, P_C1, P_C2,
  P_KIND, P_SHX, P_SHY, NP
};
// face kinds
enum { FK_INTERIOR = 0, FK_WALL_LO = 1, FK_WALL_HI = 2, FK_FREE_LO = 3, FK_FREE_HI = 4 };
// the domain lies on the +normal side of a low-side boundary face
__host__ __device__ __forceinline__ bool fk_low(int kind) { return kind == FK_WALL_LO || kind == FK_FREE_LO; }
// moments accumulated per point, in the frame shifted by a reference velocity xi' = xi - u_ref
//   M0 = sum w g, MX/MY = sum w xi' g, E = sum w (|xi'|^2 g + h), G = sum w xi' xi' g,
//   J = sum w xi' (|xi'|^2 g + h)
enum { MO_0 = 0, MO_X, MO_Y, MO_E, MO_GXX, MO_GXY, MO_GYY, MO_JX, MO_JY, NMOM };
// Role of a face on a level: evaluated here between two cells of this level (or a wall of a
// cell of this level), evaluated here as a cross-level face on its common refinement
// (V^int, Sec. 3.4) with the flux exported, or received as a mapped flux.
enum { FR_NONE = 0, FR_NORMAL = 1, FR_CROSS = 2, FR_RECV = 3 };
// boundary kinds (match mlvs.h)
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_WALL = 2, BC_FREE = 3 };

template <class T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
  // exp(l - c^2 k) with the operation order pinned (no contraction freedom), so every
  // kernel that evaluates this factor gets the same bits for the same inputs.
  static __device__ __forceinline__ float gauss(float c, float k, float l) {
    return __expf(__fmaf_rn(__fmul_rn(c, c), -k, l));
  }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
  static __device__ __forceinline__ double gauss(double c, double k, double l) {
    return exp(__fma_rn(__dmul_rn(c, c), -k, l));
  }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

template <class S, class T> __device__ __forceinline__ T ldf(const S* p);
template <> __device__ __forceinline__ float ldf<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ double ldf<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <class S, class T> __device__ __forceinline__ void stf(S* p, T v);
template <> __device__ __forceinline__ void stf<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void stf<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void stf<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

// 32-bit integer hash (the "lowbias32" xorshift-multiply finaliser).
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Rounding of an updated value into the storage type.  BF16 rounds stochastically with
// 16 random bits r: the float's low 16 bits plus r carry into the kept bits with probability
// (low bits)/2^16, so the stored value is unbiased and the rounding errors of successive
// steps are independent (round to nearest repeats the same error on a slowly changing
// state, and that error then accumulates step after step).
template <class S, class T> struct Stored {
  static __device__ __forceinline__ S enc(T v, unsigned) { return v; }
  static __device__ __forceinline__ T dec(S s) { return s; }
};
template <> struct Stored<__nv_bfloat16, float> {
  static __device__ __forceinline__ __nv_bfloat16 enc(float v, unsigned r) {
    const unsigned u = __float_as_uint(v);
    __nv_bfloat16_raw raw;
    raw.x = (unsigned short)((u + (r & 0xffffu)) >> 16);
    return __nv_bfloat16(raw);
  }
  static __device__ __forceinline__ float dec(__nv_bfloat16 s) { return __bfloat162float(s); }
};

// Value as stored (round trip through the storage type).
template <class S, class T> __device__ __forceinline__ T ldf_round(T v) { return v; }
template <> __device__ __forceinline__ float ldf_round<__nv_bfloat16, float>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Model parameters of one point, held in registers.
template <class T> struct MP {
  T ux, uy, lnh, inv2RT, kqx, kqy, RT, b0, b1, b2, b3, c1, c2;
  __device__ __forceinline__ void load(const T* __restrict__ P, long n, long i) {
    ux = P[P_UX * n + i];     uy = P[P_UY * n + i];   lnh = P[P_LNH * n + i];
    inv2RT = P[P_INV2RT * n + i]; kqx = P[P_KQX * n + i]; kqy = P[P_KQY * n + i];
    RT = P[P_RT * n + i];     b0 = P[P_B0 * n + i];   b1 = P[P_B1 * n + i];
    b2 = P[P_B2 * n + i];     b3 = P[P_B3 * n + i];   c1 = P[P_C1 * n + i];
    c2 = P[P_C2 * n + i];
  }
  __device__ __forceinline__ void zero() {
    ux = uy = lnh = inv2RT = kqx = kqy = RT = b0 = b1 = b2 = b3 = c1 = c2 = T(0);
  }
};

// Maxwellian of a point as a product of one factor per axis (D = 2) or one factor (D = 1):
//   g^eq = rho/(2 pi R T)^{D/2} exp(-|c|^2/(2RT)) = exp(lnh - c_x^2/(2RT)) exp(lnh - c_y^2/(2RT))
// with lnh = ln(rho/(2 pi R T)^{D/2}) / D  (Eq. g_h_eq_Pr, first line).
template <class T, int D>
__device__ __forceinline__ T maxwell_sep(const MP<T>& p, T cx, T cy) {
  const T ex = Num<T>::gauss(cx, p.inv2RT, p.lnh);
  if (D == 1) return ex;
  const T ey = Num<T>::gauss(cy, p.inv2RT, p.lnh);
  return Num<T>::mul(ex, ey);
}

// Shakhov model distribution times the compatibility factor at velocity xi:
//   g^S = g^eq [1 + kq.c (|c|^2/RT - D - 2)]
//   h^S = RT g^eq [c0 + kq.c ((|c|^2/RT - D) c0 - 2K)],  c0 = K + 3 - D, kq = (1-Pr) q/(5 p RT)
//   (Eq. g_h_eq_Pr), then multiplied by 1 + B0 + B1 c_x + B2 c_y + B3 |c|^2.
// Every operation is an explicitly rounded intrinsic, so each kernel that evaluates the model
// (face sums, update, finalisation) obtains the same bits for the same inputs.
template <class T, int D>
__device__ __forceinline__ void model_eval(const MP<T>& p, T xix, T xiy, T c0, T twoK, T& g, T& h) {
  using N = Num<T>;
  const T cx = N::sub(xix, p.ux);
  const T cy = (D == 2) ? N::sub(xiy, p.uy) : T(0);
  const T geq = maxwell_sep<T, D>(p, cx, cy);
  const T cc = N::fma(cy, cy, N::mul(cx, cx));
  const T cq = N::fma(p.kqy, cy, N::mul(p.kqx, cx));
  const T t = N::mul(N::mul(T(2), p.inv2RT), cc);
  const T gs = N::mul(geq, N::fma(cq, N::sub(t, T(D + 2)), T(1)));
  const T hs = N::mul(N::mul(p.RT, geq), N::fma(cq, N::fma(N::sub(t, T(D)), c0, -twoK), c0));
  const T corr = N::fma(p.b3, cc, N::fma(p.b2, cy, N::fma(p.b1, cx, p.b0)));
  g = N::fma(gs, corr, gs);
  h = N::fma(hs, corr, hs);
}

// A pair of lanes: two velocities processed together by one thread.  Every lane operation is
// the explicitly rounded operation of Num<T> on that lane (a - b as a + (-b), the same IEEE
// result), so a pair gives the same bits as two scalar evaluations.  FP32 pairs use the
// packed two-lane FP32 instructions of sm_100 and later (one instruction per lane pair).
template <class T> struct Pk;
template <> struct Pk<float> {
  using V = float2;
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V splat(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ float ex(float a) { return __expf(a); }
};
template <> struct Pk<double> {
  using V = double2;
  static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ V splat(double a) { return make_double2(a, a); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
  }
  static __device__ __forceinline__ double ex(double a) { return exp(a); }
};
template <class T> using V2 = typename Pk<T>::V;

// model_eval on a pair of velocities: the same operations, lane by lane.
template <class T, int D>
__device__ __forceinline__ void model_eval2(const MP<T>& p, V2<T> xix, V2<T> xiy, T c0, T twoK, V2<T>& g,
                                            V2<T>& h) {
  using P = Pk<T>;
  using N = Num<T>;
  const V2<T> cx = P::sub(xix, P::splat(p.ux));
  const V2<T> cy = (D == 2) ? P::sub(xiy, P::splat(p.uy)) : P::splat(T(0));
  const V2<T> cx2 = P::mul(cx, cx);
  const V2<T> ax = P::fma(cx2, P::splat(-p.inv2RT), P::splat(p.lnh));
  V2<T> geq = P::mk(P::ex(ax.x), P::ex(ax.y));
  if (D == 2) {
    const V2<T> ay = P::fma(P::mul(cy, cy), P::splat(-p.inv2RT), P::splat(p.lnh));
    geq = P::mul(geq, P::mk(P::ex(ay.x), P::ex(ay.y)));
  }
  const V2<T> cc = P::fma(cy, cy, cx2);
  const V2<T> cq = P::fma(P::splat(p.kqy), cy, P::mul(P::splat(p.kqx), cx));
  const V2<T> t = P::mul(P::splat(N::mul(T(2), p.inv2RT)), cc);
  const V2<T> gs = P::mul(geq, P::fma(cq, P::sub(t, P::splat(T(D + 2))), P::splat(T(1))));
  const V2<T> hs = P::mul(P::mul(P::splat(p.RT), geq),
                          P::fma(cq, P::fma(P::sub(t, P::splat(T(D))), P::splat(c0), P::splat(-twoK)), P::splat(c0)));
  const V2<T> corr = P::fma(P::splat(p.b3), cc, P::fma(P::splat(p.b2), cy, P::fma(P::splat(p.b1), cx, P::splat(p.b0))));
  g = P::fma(gs, corr, gs);
  h = P::fma(hs, corr, hs);
}

// model_eval2 with the eight-term correction factor 1 + b0 + b1 c_x + b2 c_y + b3 |c|^2 + b4 |c|^2 c_x
// + b5 |c|^2 c_y + b6 (c_x^2 - c_y^2) + b7 c_x c_y (2-D; b8 = b4..b7), the factor formed in the
// order of the scalar eight-moment evaluation.
template <class T>
__device__ __forceinline__ void model_eval2c8(const MP<T>& p, const T b8[4], V2<T> xix, V2<T> xiy, T c0, T twoK,
                                              V2<T>& g, V2<T>& h) {
  using P = Pk<T>;
  using N = Num<T>;
  const V2<T> cx = P::sub(xix, P::splat(p.ux));
  const V2<T> cy = P::sub(xiy, P::splat(p.uy));
  const V2<T> cx2 = P::mul(cx, cx);
  const V2<T> ax = P::fma(cx2, P::splat(-p.inv2RT), P::splat(p.lnh));
  const V2<T> ay = P::fma(P::mul(cy, cy), P::splat(-p.inv2RT), P::splat(p.lnh));
  const V2<T> geq = P::mul(P::mk(P::ex(ax.x), P::ex(ax.y)), P::mk(P::ex(ay.x), P::ex(ay.y)));
  const V2<T> cc = P::fma(cy, cy, cx2);
  const V2<T> cq = P::fma(P::splat(p.kqy), cy, P::mul(P::splat(p.kqx), cx));
  const V2<T> t = P::mul(P::splat(N::mul(T(2), p.inv2RT)), cc);
  const V2<T> gs = P::mul(geq, P::fma(cq, P::sub(t, P::splat(T(4))), P::splat(T(1))));
  const V2<T> hs = P::mul(P::mul(P::splat(p.RT), geq),
                          P::fma(cq, P::fma(P::sub(t, P::splat(T(2))), P::splat(c0), P::splat(-twoK)), P::splat(c0)));
  V2<T> corr = P::fma(P::splat(p.b3), cc, P::fma(P::splat(p.b2), cy, P::fma(P::splat(p.b1), cx, P::splat(p.b0))));
  corr = P::fma(P::mul(P::splat(b8[0]), cc), cx, corr);
  corr = P::fma(P::mul(P::splat(b8[1]), cc), cy, corr);
  const V2<T> cyy = P::mul(cy, cy);
  corr = P::fma(P::splat(b8[2]), P::fma(cx, cx, P::mk(-cyy.x, -cyy.y)), corr);
  corr = P::fma(P::mul(P::splat(b8[3]), cx), cy, corr);
  g = P::fma(gs, corr, gs);
  h = P::fma(hs, corr, hs);
}

// a + b rounded stochastically to FP32 with 16 random bits r (FP32 storage of phi~^{n+1}):
// given s = RN(a + b) and its rounding error e, the neighbour of s towards the
// exact sum is taken with probability |e| / gap, so the stored value is unbiased: near a
// steady state the increments below half an ulp are not lost step after step, and the
// rounding errors of successive steps are independent.
__device__ __forceinline__ float sr_pick(float s, float e, unsigned r) {
  const unsigned us = __float_as_uint(s);
  const float sn = __uint_as_float(((s > 0.0f) == (e > 0.0f)) ? us + 1u : us - 1u);
  const float gap = fabsf(__fsub_rn(sn, s));
  const float u = __fmul_rn(__uint2float_rn(r & 0xffffu) + 0.5f, 1.0f / 65536.0f);
  return (e != 0.0f && s != 0.0f && __fmul_rn(u, gap) < fabsf(e)) ? sn : s;
}
// a + b for a pair of lanes, a the stored value and b its increment: the rounding error by
// Dekker's Fast2Sum, e = b - (s - a), exact whenever |a| >= |b| (every value that does not
// more than double in a step), in packed arithmetic
__device__ __forceinline__ float2 sr_add2(float2 a, float2 b, unsigned r0, unsigned r1) {
  using P = Pk<float>;
  const float2 s = P::add(a, b);
  const float2 e = P::sub(b, P::sub(s, a));
  return make_float2(sr_pick(s.x, e.x, r0), sr_pick(s.y, e.y, r1));
}

// Compensated (Kahan) accumulation for sums that must keep FP64-level accuracy in FP32.
template <class T> struct KSum {
  T s, c;
  __device__ __forceinline__ void zero() { s = T(0); c = T(0); }
  __device__ __forceinline__ void add(T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double val() const { return (double)s - (double)c; }
};
template <> struct KSum<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double val() const { return s; }
};

// Per-level step constants.
struct StepConst {
  int nx, ny, nfx, nfy, ncell, nface;
  int px, py;          // periodic flags
  int bc[4];
  int nv, vpc, nchunk;  // velocities, velocities per chunk, chunks
  int nax;             // > 0: the space is the tensor product of one axis of nax points
  double dx, dy, dt;
  double c0, twoK;      // K + 3 - D, 2K
};

}  // namespace mlvs
