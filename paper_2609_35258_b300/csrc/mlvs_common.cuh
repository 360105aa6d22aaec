// Shared device definitions of the MLVS-DUGKS library (sm_103a).
//
// Layouts (device memory, per instance and level):
//   f      [comp in {g~, h~}][v][cell]        storage type S (double | float | bf16), cells row-major
//   params [NP][point]                        compute type T, one point = a cell or a face
//   part   [chunk][NMOM][point]               double, per-velocity-chunk partial moments
//   vt     [4][v] = (xi_x, xi_y, w, |xi|^2)    compute type T (and a double copy)
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mlvs {

// Per-point parameters of the model distribution (Eq. g_h_eq_Pr with the compatibility
// factor of Eq. gh_model_correction folded in) plus two blending coefficients:
//   cells: C1 = (2 tau - s)/(2 tau + dt), C2 = 3 s/(2 tau + dt)  (phi-bar-plus from phi~, phi^S)
//   faces: C1 = 2 tau/(2 tau + s),       C2 = s/(2 tau + s)      (Eq. recover_phi)
//   wall faces: C2 = rho_w multiplies the unit-density wall Maxwellian.
enum {
  P_UX = 0, P_UY, P_LNN, P_INV2RT, P_KQX, P_KQY, P_RT, P_P0, P_A1, P_A2, P_P3, P_C1, P_C2,
  P_KIND, P_SHX, P_SHY, NP
};
// face kinds
enum { FK_INTERIOR = 0, FK_WALL_LO = 1, FK_WALL_HI = 2 };
// moments accumulated per point, in the frame shifted by a reference velocity xi' = xi - u_ref
//   M0 = sum w g, MX/MY = sum w xi' g, E = sum w (|xi'|^2 g + h), G = sum w xi' xi' g,
//   J = sum w xi' (|xi'|^2 g + h)
enum { MO_0 = 0, MO_X, MO_Y, MO_E, MO_GXX, MO_GXY, MO_GYY, MO_JX, MO_JY, NMOM };
// boundary kinds (match mlvs.h)
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_WALL = 2 };

template <class T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float ex(float x) { return __expf(x); }
  static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
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

// Value as stored (round trip through the storage type).
template <class S, class T> __device__ __forceinline__ T ldf_round(T v) { return v; }
template <> __device__ __forceinline__ float ldf_round<__nv_bfloat16, float>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Model parameters of one point, held in registers.
template <class T> struct MP {
  T ux, uy, lnn, inv2RT, kqx, kqy, RT, p0, a1, a2, p3, c1, c2;
  __device__ __forceinline__ void load(const T* __restrict__ P, long n, long i) {
    ux = P[P_UX * n + i];     uy = P[P_UY * n + i];   lnn = P[P_LNN * n + i];
    inv2RT = P[P_INV2RT * n + i]; kqx = P[P_KQX * n + i]; kqy = P[P_KQY * n + i];
    RT = P[P_RT * n + i];     p0 = P[P_P0 * n + i];   a1 = P[P_A1 * n + i];
    a2 = P[P_A2 * n + i];     p3 = P[P_P3 * n + i];   c1 = P[P_C1 * n + i];
    c2 = P[P_C2 * n + i];
  }
};

// Shakhov model distribution times the compatibility factor at velocity xi:
//   g^eq = exp(lnn - |c|^2/(2RT)),  c = xi - u                          (Eq. g_h_eq_Pr)
//   g^S  = g^eq [1 + kq.c (|c|^2/RT - D - 2)]
//   h^S  = RT g^eq [c0 + kq.c ((|c|^2/RT - D) c0 - 2K)],  c0 = K + 3 - D, kq = (1-Pr) q/(5 p RT)
//   factor = 1 + sum_m a_m phi_m(xi) = p0 + a1 xi_x + a2 xi_y + p3 |xi|^2   (Eq. eq_four_basis)
template <class T, int D>
__device__ __forceinline__ void model_eval(const MP<T>& p, T xix, T xiy, T xi2, T c0, T twoK,
                                           T& g, T& h) {
  T cx = xix - p.ux;
  T cy = (D == 2) ? (xiy - p.uy) : T(0);
  T cc = cx * cx + cy * cy;
  T geq = Num<T>::ex(p.lnn - cc * p.inv2RT);
  T cq = p.kqx * cx + p.kqy * cy;
  T t = T(2) * p.inv2RT * cc;
  T gs = geq * (T(1) + cq * (t - T(D + 2)));
  T hs = p.RT * geq * (c0 + cq * ((t - T(D)) * c0 - twoK));
  T fac = p.p0 + p.a1 * xix + p.a2 * xiy + p.p3 * xi2;
  g = gs * fac;
  h = hs * fac;
}

// Compensated (Kahan) accumulation for the conserved-moment sums in FP32; plain in FP64.
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
  double dx, dy, dt;
  double c0, twoK;      // K + 3 - D, 2K
};

}  // namespace mlvs
