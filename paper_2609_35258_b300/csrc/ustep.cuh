// DUGKS step on an unstructured mesh of polygonal cells, one velocity space (Sec. 2.2 on
// general polygons; the two-cavity expansion of Sec. 4.5 runs on unstructured cells).
//
// Every pass is a per-element function u_elem<E>(args, i) over a flat index; the CUDA kernel
// of a pass is a grid-stride loop over it, so the step's arithmetic and indexing are one
// piece of code whatever runs the loop.  Passes of one step, in order:
//   U_CELL_FIN   cell           Eqs. discrete_W, discrete_q, tau, model + compatibility
//                               correction (Sec. 3.3.1), blending weights, from the
//                               velocity-chunk partial moments of phi~ in the cell's frame
//   U_BARP       (v, cell)      phi-bar-plus = phi~ + b (phi^S - phi~)
//   U_GRAD       (v, cell)      least-squares gradient of phi-bar-plus over the face
//                               neighbours (a boundary face adds the cell reflected through it,
//                               a zero difference), Venkatakrishnan-limited
//   U_FACE_BAR   (face, chunk)  Eq. reconstruction from the upwind side (a boundary face's
//                               ghost: the cell's own data at the reflected centroid) over the
//                               chunk's velocities, and their face moments (Eq. W_from_bar), or
//                               on a wall face their outgoing normal mass flux
//   U_FACE_FIN   face           face state, model + correction, Eq. recover_phi weights; on a
//                               wall face rho_w from zero net mass flux
//   U_FLUX       (v, face)      (xi.n) |f| phi_face (a wall face emits rho_w g_w inward)
//   U_UPDATE     (cell, chunk)  Eq. explicit_update: phi~+ - dt/|V| sum_faces flux over the
//                               chunk's velocities, and the partial moments of the new phi~
//                               that the next step's U_CELL_FIN sums
// U_CELL_SUMS forms those partial moments once after the initial state.  A (face, chunk) or
// (cell, chunk) pass takes consecutive faces or cells on consecutive threads, so at each
// velocity of its loop a warp's loads and stores stay coalesced.
// Layouts (flat, cells and faces contiguous within a velocity plane):
//   f, barp  [comp][v][cell];  grad [comp][dir][v][cell];  fbar, flux [comp][v][face]
//   part_c [chunk][NMOM][cell], part_f [chunk][NMOM][face] (double)
//   cprm [NP][cell], fprm [NP][face]; cgeo [UC_N][cell]; fgeo [UF_N][face]
#pragma once
#include "mlvs_common.cuh"
#include "finalize.cuh"

namespace mlvs {

enum { U_CELL_SUMS = 0, U_CELL_FIN, U_BARP, U_GRAD, U_FACE_BAR, U_FACE_FIN, U_FLUX, U_UPDATE,
       U_INIT_PARAMS, U_INIT_F, U_WALL_DEN, U_NPASS };
// per-cell geometry rows: area, centroid, inverse least-squares normal matrix, area^{3/2}
enum { UC_AREA = 0, UC_CX, UC_CY, UC_MXX, UC_MXY, UC_MYY, UC_H3, UC_N };
// per-face geometry rows: unit normal out of L, length, midpoint
enum { UF_NX = 0, UF_NY, UF_LEN, UF_MX, UF_MY, UF_N };
enum { ULIM_NONE = 0, ULIM_VENKAT = 1 };

template <class T> struct UArgs {
  PointArgs pa;         // velocity tables, gas, constants (k.nv, k.nax, k.dt, k.c0, k.twoK), err
  int nc, nf, nv, vpc, nchunk, limiter, compat_face;
  int compat8;          // 1: the eight-moment correction at cells and faces (compat flags on)
  double dt;
  double wall[8][3];    // (u_w, v_w, T_w) per wall index
  const T* cgeo;        // [UC_N][nc]
  const T* fgeo;        // [UF_N][nf]
  const int* fcell;     // [2][nf] L, R (-1: boundary)
  const int* fwall;     // [nf] wall index of a boundary face, -1 inside
  const int* cf_ptr;    // [nc + 1]
  const int* cf;        // signed faces of every cell (f: the cell is L; -f - 1: it is R)
  const double* W0;     // [nc][4] initial (rho, u, v, T)
  T* f;
  T* barp;
  T* grad;
  T* fbar;
  T* flux;
  double* part_c;
  double* part_f;
  T* cprm;
  T* fprm;
  T* cprm8;             // [4][nc] eight-moment coefficients b4..b7 (zero without it)
  T* fprm8;             // [4][nf]
  double* W;            // [11][nc] cell state at the start of the step
  double* wden;         // [nf] sum_{xi.n_in > 0} w (xi.n_in) g_w of the unit-density wall Maxwellian
};

template <class T>
__device__ __forceinline__ T u_xi(const UArgs<T>& a, int v, int d) {
  return reinterpret_cast<const T*>(a.pa.vt)[(long)d * a.nv + v];
}

// Partial moments of one point's values over a run of velocities, in the frame (ux, uy):
// M0 = sum w g, M_x, M_y = sum w c g, E = sum w (|c|^2 g + h), G = sum w c c g,
// J = sum w c (|c|^2 g + h) (compensated where the finalisation subtracts large terms).
template <class T> struct UMom {
  KSum<T> a0, ax, ay, ae;
  T gxx, gxy, gyy, jx, jy;
  __device__ __forceinline__ void zero() {
    a0.zero(); ax.zero(); ay.zero(); ae.zero();
    gxx = gxy = gyy = jx = jy = T(0);
  }
  __device__ __forceinline__ void add(const UArgs<T>& a, int v, T gq, T hq, T ux, T uy) {
    const T xp = u_xi(a, v, 0) - ux, yp = u_xi(a, v, 1) - uy;
    const T wxv = u_xi(a, v, 2), wyv = u_xi(a, v, 3);
    const T wg = wxv * (wyv * gq);
    const T e = wxv * (wyv * ((xp * xp + yp * yp) * gq + hq));
    a0.add(wg); ax.add(wg * xp); ay.add(wg * yp); ae.add(e);
    gxx += wg * xp * xp; gxy += wg * xp * yp; gyy += wg * yp * yp;
    jx += e * xp; jy += e * yp;
  }
  __device__ __forceinline__ void store(double* out, long stride) const {
    out[MO_0 * stride] = a0.val(); out[MO_X * stride] = ax.val(); out[MO_Y * stride] = ay.val();
    out[MO_E * stride] = ae.val(); out[MO_GXX * stride] = gxx; out[MO_GXY * stride] = gxy;
    out[MO_GYY * stride] = gyy; out[MO_JX * stride] = jx; out[MO_JY * stride] = jy;
  }
};

// frame of a face's moments: the mean of its cells' velocities (its only cell on a boundary)
template <class T>
__device__ __forceinline__ void u_face_shift(const UArgs<T>& a, int fi, T& sx, T& sy) {
  const int L = a.fcell[fi], R = a.fcell[a.nf + fi] >= 0 ? a.fcell[a.nf + fi] : L;
  sx = T(0.5) * (a.cprm[P_UX * (long)a.nc + L] + a.cprm[P_UX * (long)a.nc + R]);
  sy = T(0.5) * (a.cprm[P_UY * (long)a.nc + L] + a.cprm[P_UY * (long)a.nc + R]);
}

// phi-bar-plus reconstructed at (ox, oy) from the centroid of cell c, moved back by xi s
template <class T>
__device__ __forceinline__ T u_recon(const UArgs<T>& a, int comp, int v, int c, T ox, T oy, T xs, T ys) {
  const long nc = a.nc, nv = a.nv;
  const T P = a.barp[((long)comp * nv + v) * nc + c];
  const T gx = a.grad[(((long)comp * 2 + 0) * nv + v) * nc + c];
  const T gy = a.grad[(((long)comp * 2 + 1) * nv + v) * nc + c];
  return P + (ox - xs) * gx + (oy - ys) * gy;
}

// the model of point i with parameters P[NP][n] and, in eight-moment mode, P8[4][n]
template <class T>
__device__ __forceinline__ void u_model(const UArgs<T>& a, const MP<T>& m, const T* P8, long n, long i, T xx, T yy,
                                        T& g, T& h) {
  if (a.compat8) {
    const T b8[4] = {P8[i], P8[n + i], P8[2 * n + i], P8[3 * n + i]};
    u_model_eval8<T>(m, b8, xx, yy, T(a.pa.k.c0), T(a.pa.k.twoK), g, h);
  } else {
    model_eval<T, 2>(m, xx, yy, T(a.pa.k.c0), T(a.pa.k.twoK), g, h);
  }
}

template <int E, class T>
__device__ inline void u_elem(const UArgs<T>& a, long i) {
  const long nc = a.nc, nf = a.nf, nv = a.nv;
  using N = Num<T>;
  if constexpr (E == U_CELL_SUMS) {
    const int c = (int)(i % nc), chunk = (int)(i / nc);
    const int v0 = chunk * a.vpc, v1 = min(a.nv, v0 + a.vpc);
    const T ux = a.cprm[P_UX * nc + c], uy = a.cprm[P_UY * nc + c];
    UMom<T> acc;
    acc.zero();
    for (int v = v0; v < v1; ++v) acc.add(a, v, a.f[(long)v * nc + c], a.f[(nv + v) * nc + c], ux, uy);
    acc.store(a.part_c + (long)chunk * NMOM * nc + c, nc);
  } else if constexpr (E == U_CELL_FIN) {
    finalize_point<T, 2, 0>(a.pa, (int)i);
    if (a.compat8 && a.pa.compat) {
      const double* W = a.W;
      const double rho = W[i], ux = W[nc + i], uy = W[2 * nc + i], Tm = W[3 * nc + i];
      if (!(rho > 0.0) || !(Tm > 0.0) || !isfinite(rho) || !isfinite(Tm)) return;   // flagged already
      MP<T> mp;
      mp.load(a.cprm, nc, i);
      const T c1 = mp.c1, c2 = mp.c2;
      point_params<T, 2>(a.pa.gas, rho, ux, uy, Tm, W[4 * nc + i], W[5 * nc + i], mp);
      T b8[4];
      const double pr = 1.0 - a.pa.gas.Pr;
      if (!u_correct8<T>(a.pa, rho, ux, uy, Tm, pr * W[4 * nc + i], pr * W[5 * nc + i], mp, b8))
        atomicOr(a.pa.err, ERR_SINGULAR);
      mp.c1 = c1;
      mp.c2 = c2;
      store_mp<T>(a.cprm, nc, i, mp, T(0));
      for (int m = 0; m < 4; ++m) a.cprm8[m * nc + i] = b8[m];
    }
  } else if constexpr (E == U_BARP) {
    const int c = (int)(i % nc), v = (int)(i / nc);
    MP<T> m;
    m.load(a.cprm, nc, c);
    T gS, hS;
    u_model<T>(a, m, a.cprm8, nc, c, u_xi(a, v, 0), u_xi(a, v, 1), gS, hS);
    const T gt = a.f[(long)v * nc + c], ht = a.f[(nv + v) * nc + c];
    a.barp[(long)v * nc + c] = N::fma(m.c1, N::sub(gS, gt), gt);
    a.barp[(nv + v) * nc + c] = N::fma(m.c1, N::sub(hS, ht), ht);
  } else if constexpr (E == U_GRAD) {
    const int c = (int)(i % nc), v = (int)(i / nc);
    const T cx = a.cgeo[UC_CX * nc + c], cy = a.cgeo[UC_CY * nc + c];
    for (int comp = 0; comp < 2; ++comp) {
      const T* P = a.barp + (long)comp * nv * nc + (long)v * nc;
      const T pc = P[c];
      T rx = T(0), ry = T(0), umax = pc, umin = pc;
      for (int k = a.cf_ptr[c]; k < a.cf_ptr[c + 1]; ++k) {
        const int s = a.cf[k], fi = s >= 0 ? s : -s - 1;
        const int o = s >= 0 ? a.fcell[nf + fi] : a.fcell[fi];
        if (o < 0) continue;                     // the reflected ghost: a zero difference
        const T po = P[o], du = po - pc;
        rx += du * (a.cgeo[UC_CX * nc + o] - cx);
        ry += du * (a.cgeo[UC_CY * nc + o] - cy);
        umax = po > umax ? po : umax;
        umin = po < umin ? po : umin;
      }
      T gx = a.cgeo[UC_MXX * nc + c] * rx + a.cgeo[UC_MXY * nc + c] * ry;
      T gy = a.cgeo[UC_MXY * nc + c] * rx + a.cgeo[UC_MYY * nc + c] * ry;
      if (a.limiter == ULIM_VENKAT) {
        const T dmax = umax - pc, dmin = umin - pc;
        const T eps2 = a.cgeo[UC_H3 * nc + c] * pc * pc;
        T phi = T(1);
        for (int k = a.cf_ptr[c]; k < a.cf_ptr[c + 1]; ++k) {
          const int s = a.cf[k], fi = s >= 0 ? s : -s - 1;
          const T d2 = gx * (a.fgeo[UF_MX * nf + fi] - cx) + gy * (a.fgeo[UF_MY * nf + fi] - cy);
          if (d2 == T(0)) continue;
          const T d1 = d2 > T(0) ? dmax : dmin;
          const T num = (d1 * d1 + eps2) * d2 + T(2) * d2 * d2 * d1;
          const T den = d1 * d1 + T(2) * d2 * d2 + d1 * d2 + eps2;
          const T r = num / den / d2;
          phi = r < phi ? r : phi;
        }
        gx *= phi;
        gy *= phi;
      }
      a.grad[(((long)comp * 2 + 0) * nv + v) * nc + c] = gx;
      a.grad[(((long)comp * 2 + 1) * nv + v) * nc + c] = gy;
    }
  } else if constexpr (E == U_FACE_BAR) {
    const int fi = (int)(i % nf), chunk = (int)(i / nf);
    const int v0 = chunk * a.vpc, v1 = min(a.nv, v0 + a.vpc);
    const T s = T(0.5 * a.dt);
    const T nx = a.fgeo[UF_NX * nf + fi], ny = a.fgeo[UF_NY * nf + fi];
    const T mx = a.fgeo[UF_MX * nf + fi], my = a.fgeo[UF_MY * nf + fi];
    const int L = a.fcell[fi], R = a.fcell[nf + fi];
    const T oxL = mx - a.cgeo[UC_CX * nc + L], oyL = my - a.cgeo[UC_CY * nc + L];
    const T oxR = R >= 0 ? mx - a.cgeo[UC_CX * nc + R] : -oxL, oyR = R >= 0 ? my - a.cgeo[UC_CY * nc + R] : -oyL;
    const int Rc = R >= 0 ? R : L;                  // a boundary face's ghost carries L's data
    const bool wall = a.fwall[fi] >= 0;
    T sx = T(0), sy = T(0);
    if (!wall) u_face_shift<T>(a, fi, sx, sy);
    UMom<T> acc;
    acc.zero();
    KSum<T> out0;                                   // wall: sum_{xi.n_in <= 0} w (xi.n_in) phi-bar_g
    out0.zero();
    for (int v = v0; v < v1; ++v) {
      const T xx = u_xi(a, v, 0), yy = u_xi(a, v, 1);
      // two rounded products and a rounded sum (no contraction): a velocity tangential to
      // the face gives an exact zero, as in the oracle, and takes the mean of both sides
      const T xn = N::add(N::mul(nx, xx), N::mul(ny, yy));
      T bar[2];
      for (int comp = 0; comp < 2; ++comp) {
        const T vL = u_recon<T>(a, comp, v, L, oxL, oyL, xx * s, yy * s);
        const T vR = u_recon<T>(a, comp, v, Rc, oxR, oyR, xx * s, yy * s);
        bar[comp] = xn > T(0) ? vL : (xn < T(0) ? vR : T(0.5) * (vL + vR));
        a.fbar[((long)comp * nv + v) * nf + fi] = bar[comp];
      }
      if (wall) {
        const T xin = -xn;
        if (xin <= T(0)) out0.add(u_xi(a, v, 2) * (u_xi(a, v, 3) * (xin * bar[0])));
      } else {
        acc.add(a, v, bar[0], bar[1], sx, sy);
      }
    }
    double* out = a.part_f + (long)chunk * NMOM * nf + fi;
    if (wall) {
      out[MO_0 * nf] = out0.val();
      for (int m = 1; m < NMOM; ++m) out[m * nf] = 0.0;
    } else {
      acc.store(out, nf);
    }
  } else if constexpr (E == U_FACE_FIN) {
    const int fi = (int)i;
    double M[NMOM];
    for (int m = 0; m < NMOM; ++m) M[m] = 0.0;
    for (int c = 0; c < a.nchunk; ++c)
      for (int m = 0; m < NMOM; ++m) M[m] += a.part_f[((long)c * NMOM + m) * nf + fi];
    const GasDev& g = a.pa.gas;
    MP<T> mp;
    const int wi = a.fwall[fi];
    if (wi >= 0) {
      wall_mp<T>(g.R, a.wall[wi][0], a.wall[wi][1], a.wall[wi][2], mp);
      const double rw = -M[MO_0] / a.wden[fi];
      mp.c2 = T(rw);                            // rho_w as hi + lo
      mp.c1 = T(rw - (double)mp.c2);
      store_mp<T>(a.fprm, nf, fi, mp, T(FK_WALL_LO));
      if (!isfinite(rw)) atomicOr(a.pa.err, ERR_NONFINITE);
      return;
    }
    T sx, sy;
    u_face_shift<T>(a, fi, sx, sy);
    const double rho = M[MO_0];
    const double upx = M[MO_X] / rho, upy = M[MO_Y] / rho, u2 = upx * upx + upy * upy;
    const double ux = (double)sx + upx, uy = (double)sy + upy;
    const double Tm = (M[MO_E] - rho * u2) / ((3.0 + g.K) * rho * g.R);
    double qx = 0.5 * (M[MO_JX] - 2.0 * (upx * M[MO_GXX] + upy * M[MO_GXY]) - upx * M[MO_E] + 2.0 * rho * u2 * upx);
    double qy = 0.5 * (M[MO_JY] - 2.0 * (upx * M[MO_GXY] + upy * M[MO_GYY]) - upy * M[MO_E] + 2.0 * rho * u2 * upy);
    const double s = 0.5 * a.dt;
    const double tau = g.mu_ref * pow(Tm / g.T_ref, g.omega) / (rho * g.R * Tm);
    const double qf = 2.0 * tau / (2.0 * tau + s * g.Pr);
    qx *= qf;
    qy *= qf;
    const bool finite = isfinite(rho) && isfinite(Tm) && isfinite(ux) && isfinite(uy);
    if (!finite || !(rho > 0.0) || !(Tm > 0.0)) {
      atomicOr(a.pa.err, finite ? ERR_POSITIVITY : ERR_NONFINITE);
      return;
    }
    PointArgs pf = a.pa;
    pf.compat = a.compat_face;
    bool ok;
    if (a.compat8 && a.compat_face) {
      point_params<T, 2>(pf.gas, rho, ux, uy, Tm, qx, qy, mp);
      T b8[4];
      const double pr = 1.0 - g.Pr;
      ok = u_correct8<T>(pf, rho, ux, uy, Tm, pr * qx, pr * qy, mp, b8);
      for (int m = 0; m < 4; ++m) a.fprm8[m * nf + fi] = b8[m];
    } else {
      ok = point_model<T, 2>(pf, rho, ux, uy, Tm, qx, qy, mp);
    }
    mp.c1 = T(2.0 * tau / (2.0 * tau + s));
    mp.c2 = T(s / (2.0 * tau + s));
    store_mp<T>(a.fprm, nf, fi, mp, T(FK_INTERIOR));
    if (!ok) atomicOr(a.pa.err, ERR_SINGULAR);
  } else if constexpr (E == U_FLUX) {
    const int fi = (int)(i % nf), v = (int)(i / nf);
    MP<T> m;
    m.load(a.fprm, nf, fi);
    const T xx = u_xi(a, v, 0), yy = u_xi(a, v, 1);
    const T xn = N::add(N::mul(a.fgeo[UF_NX * nf + fi], xx), N::mul(a.fgeo[UF_NY * nf + fi], yy));
    const T scale = xn * a.fgeo[UF_LEN * nf + fi];
    T gS, hS;
    if (a.fwall[fi] >= 0) model_eval<T, 2>(m, xx, yy, T(a.pa.k.c0), T(a.pa.k.twoK), gS, hS);
    else u_model<T>(a, m, a.fprm8, nf, fi, xx, yy, gS, hS);
    const T gb = a.fbar[(long)v * nf + fi], hb = a.fbar[(nv + v) * nf + fi];
    T gp, hp;
    if (a.fwall[fi] >= 0) {
      if (-xn > T(0)) {                          // entering the domain: rho_w g_w
        gp = N::fma(m.c1, gS, N::mul(m.c2, gS));
        hp = N::fma(m.c1, hS, N::mul(m.c2, hS));
      } else {
        gp = gb;
        hp = hb;
      }
    } else {
      gp = N::fma(m.c2, N::sub(gS, gb), gb);
      hp = N::fma(m.c2, N::sub(hS, hb), hb);
    }
    a.flux[(long)v * nf + fi] = scale * gp;
    a.flux[(nv + v) * nf + fi] = scale * hp;
  } else if constexpr (E == U_UPDATE) {
    const int c = (int)(i % nc), chunk = (int)(i / nc);
    const int v0 = chunk * a.vpc, v1 = min(a.nv, v0 + a.vpc);
    const T dtA = T(a.dt / (double)a.cgeo[UC_AREA * nc + c]);
    const T ux = a.cprm[P_UX * nc + c], uy = a.cprm[P_UY * nc + c];   // the next step's frame
    const int k0 = a.cf_ptr[c], k1 = a.cf_ptr[c + 1];
    UMom<T> acc;
    acc.zero();
    for (int v = v0; v < v1; ++v) {
      T nw[2];
      for (int comp = 0; comp < 2; ++comp) {
        const long at = ((long)comp * nv + v) * nc + c;
        const T t = a.f[at], bp = a.barp[at];
        T div = T(0);
        for (int k = k0; k < k1; ++k) {
          const int sg = a.cf[k];
          const T F = a.flux[((long)comp * nv + v) * nf + (sg >= 0 ? sg : -sg - 1)];
          div = sg >= 0 ? div + F : div - F;
        }
        const T tp = t + T(4.0 / 3.0) * (bp - t);   // phi~+ = 4/3 phi-bar-plus - 1/3 phi~
        nw[comp] = tp - dtA * div;
        a.f[at] = nw[comp];
      }
      acc.add(a, v, nw[0], nw[1], ux, uy);
    }
    acc.store(a.part_c + (long)chunk * NMOM * nc + c, nc);
  } else if constexpr (E == U_INIT_PARAMS) {
    const int c = (int)i;
    const double* w = a.W0 + 4 * (long)c;
    MP<T> mp;
    const bool ok = point_model<T, 2>(a.pa, w[0], w[1], w[2], w[3], 0.0, 0.0, mp);
    mp.c1 = T(0);
    mp.c2 = T(0);
    store_mp<T>(a.cprm, nc, c, mp, T(0));
    a.cprm[P_SHX * nc + c] = mp.ux;
    a.cprm[P_SHY * nc + c] = mp.uy;
    if (!ok) atomicOr(a.pa.err, ERR_SINGULAR);
  } else if constexpr (E == U_INIT_F) {
    const int c = (int)(i % nc), v = (int)(i / nc);
    MP<T> m;
    m.load(a.cprm, nc, c);
    T g, h;
    model_eval<T, 2>(m, u_xi(a, v, 0), u_xi(a, v, 1), T(a.pa.k.c0), T(a.pa.k.twoK), g, h);
    a.f[(long)v * nc + c] = g;
    a.f[(nv + v) * nc + c] = h;
  } else if constexpr (E == U_WALL_DEN) {
    const int fi = (int)i;
    const int wi = a.fwall[fi];
    if (wi < 0) {
      a.wden[fi] = 0.0;
      return;
    }
    MP<T> m;
    wall_mp<T>(a.pa.gas.R, a.wall[wi][0], a.wall[wi][1], a.wall[wi][2], m);
    const T nx = a.fgeo[UF_NX * nf + fi], ny = a.fgeo[UF_NY * nf + fi];
    double den = 0.0;
    for (int v = 0; v < a.nv; ++v) {
      const T xx = u_xi(a, v, 0), yy = u_xi(a, v, 1);
      const T xin = -N::add(N::mul(nx, xx), N::mul(ny, yy));
      if (!(xin > T(0))) continue;
      T g, h;
      model_eval<T, 2>(m, xx, yy, T(a.pa.k.c0), T(a.pa.k.twoK), g, h);
      den += (double)(u_xi(a, v, 2) * (u_xi(a, v, 3) * (xin * g)));
    }
    a.wden[fi] = den;
  }
}

// Flat extent of a pass.
template <class T>
inline long u_extent(const UArgs<T>& a, int E) {
  switch (E) {
    case U_CELL_SUMS: case U_UPDATE: return (long)a.nc * a.nchunk;
    case U_CELL_FIN: case U_INIT_PARAMS: return a.nc;
    case U_BARP: case U_GRAD: case U_INIT_F: return (long)a.nv * a.nc;
    case U_FLUX: return (long)a.nv * a.nf;
    case U_FACE_BAR: return (long)a.nf * a.nchunk;
    case U_FACE_FIN: case U_WALL_DEN: return a.nf;
  }
  return 0;
}

// One time step as its sequence of passes; run.template pass<E>(n) executes pass E over n
// elements (a kernel launch, or a loop).
template <class T, class Run>
inline void u_step_sequence(Run& run, const UArgs<T>& a) {
  run.template pass<U_CELL_FIN>(u_extent(a, U_CELL_FIN));
  run.template pass<U_BARP>(u_extent(a, U_BARP));
  run.template pass<U_GRAD>(u_extent(a, U_GRAD));
  run.template pass<U_FACE_BAR>(u_extent(a, U_FACE_BAR));
  run.template pass<U_FACE_FIN>(u_extent(a, U_FACE_FIN));
  run.template pass<U_FLUX>(u_extent(a, U_FLUX));
  run.template pass<U_UPDATE>(u_extent(a, U_UPDATE));
}

// Initial state phi~ = corrected Maxwellian of W0, its partial moments, and the wall
// normalisations.
template <class T, class Run>
inline void u_init_sequence(Run& run, const UArgs<T>& a) {
  run.template pass<U_INIT_PARAMS>(u_extent(a, U_INIT_PARAMS));
  run.template pass<U_INIT_F>(u_extent(a, U_INIT_F));
  run.template pass<U_CELL_SUMS>(u_extent(a, U_CELL_SUMS));
  run.template pass<U_WALL_DEN>(u_extent(a, U_WALL_DEN));
}

}  // namespace mlvs
