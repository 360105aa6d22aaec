// DUGKS step on an unstructured mesh of polygonal cells, one velocity space (Sec. 2.2 on
// general polygons; the two-cavity expansion of Sec. 4.5 runs on unstructured cells).
//
// Every pass is a per-element function u_elem<E>(args, i) over a flat index; the CUDA kernel
// of a pass is a grid-stride loop over it, so the step's arithmetic and indexing are one
// piece of code whatever runs the loop.  Passes of one step, in order:
//   U_CELL_SUMS  (cell, chunk)  velocity-chunk partial moments of phi~ in the cell's frame
//   U_CELL_FIN   cell           Eqs. discrete_W, discrete_q, tau, model + compatibility
//                               correction (Sec. 3.3.1), blending weights
//   U_BARP       (v, cell)      phi-bar-plus = phi~ + b (phi^S - phi~)
//   U_GRAD       (v, cell)      least-squares gradient of phi-bar-plus over the face
//                               neighbours (a boundary face adds the cell reflected through it,
//                               a zero difference), Venkatakrishnan-limited
//   U_FACE_BAR   (v, face)      Eq. reconstruction from the upwind side (a boundary face's
//                               ghost: the cell's own data at the reflected centroid)
//   U_FACE_SUMS  (face, chunk)  face moments of phi-bar (Eq. W_from_bar), or on a wall face
//                               the outgoing normal mass flux
//   U_FACE_FIN   face           face state, model + correction, Eq. recover_phi weights; on a
//                               wall face rho_w from zero net mass flux
//   U_FLUX       (v, face)      (xi.n) |f| phi_face (a wall face emits rho_w g_w inward)
//   U_UPDATE     (v, cell)      Eq. explicit_update: phi~+ - dt/|V| sum_faces flux
// Layouts (flat, cells and faces contiguous within a velocity plane):
//   f, barp  [comp][v][cell];  grad [comp][dir][v][cell];  fbar, flux [comp][v][face]
//   part_c [chunk][NMOM][cell], part_f [chunk][NMOM][face] (double)
//   cprm [NP][cell], fprm [NP][face]; cgeo [UC_N][cell]; fgeo [UF_N][face]
#pragma once
#include "mlvs_common.cuh"
#include "finalize.cuh"

namespace mlvs {

enum { U_CELL_SUMS = 0, U_CELL_FIN, U_BARP, U_GRAD, U_FACE_BAR, U_FACE_SUMS, U_FACE_FIN, U_FLUX, U_UPDATE,
       U_INIT_PARAMS, U_INIT_F, U_WALL_DEN, U_NPASS };
// per-cell geometry rows: area, centroid, inverse least-squares normal matrix, area^{3/2}
enum { UC_AREA = 0, UC_CX, UC_CY, UC_MXX, UC_MXY, UC_MYY, UC_H3, UC_N };
// per-face geometry rows: unit normal out of L, length, midpoint
enum { UF_NX = 0, UF_NY, UF_LEN, UF_MX, UF_MY, UF_N };
enum { ULIM_NONE = 0, ULIM_VENKAT = 1 };

template <class T> struct UArgs {
  PointArgs pa;         // velocity tables, gas, constants (k.nv, k.nax, k.dt, k.c0, k.twoK), err
  int nc, nf, nv, vpc, nchunk, limiter, compat_face;
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
  double* W;            // [11][nc] cell state at the start of the step
  double* wden;         // [nf] sum_{xi.n_in > 0} w (xi.n_in) g_w of the unit-density wall Maxwellian
};

template <class T>
__device__ __forceinline__ T u_xi(const UArgs<T>& a, int v, int d) {
  return reinterpret_cast<const T*>(a.pa.vt)[(long)d * a.nv + v];
}

// chunk partial moments of the phi-bar data of one point over [v0, v1), in the frame (ux, uy)
template <class T>
__device__ inline void u_chunk_moments(const UArgs<T>& a, const T* src, long n, long i, int v0, int v1, T ux,
                                       T uy, double* out, long stride) {
  KSum<T> a0, ax, ay, ae;
  a0.zero(); ax.zero(); ay.zero(); ae.zero();
  T gxx = 0, gxy = 0, gyy = 0, jx = 0, jy = 0;
  const long nv = a.nv;
  for (int v = v0; v < v1; ++v) {
    const T gq = src[(long)v * n + i], hq = src[(nv + v) * n + i];
    const T xp = u_xi(a, v, 0) - ux, yp = u_xi(a, v, 1) - uy;
    const T wxv = u_xi(a, v, 2), wyv = u_xi(a, v, 3);
    const T wg = wxv * (wyv * gq);
    const T e = wxv * (wyv * ((xp * xp + yp * yp) * gq + hq));
    a0.add(wg); ax.add(wg * xp); ay.add(wg * yp); ae.add(e);
    gxx += wg * xp * xp; gxy += wg * xp * yp; gyy += wg * yp * yp;
    jx += e * xp; jy += e * yp;
  }
  out[MO_0 * stride] = a0.val(); out[MO_X * stride] = ax.val(); out[MO_Y * stride] = ay.val();
  out[MO_E * stride] = ae.val(); out[MO_GXX * stride] = gxx; out[MO_GXY * stride] = gxy;
  out[MO_GYY * stride] = gyy; out[MO_JX * stride] = jx; out[MO_JY * stride] = jy;
}

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

template <int E, class T>
__device__ inline void u_elem(const UArgs<T>& a, long i) {
  const long nc = a.nc, nf = a.nf, nv = a.nv;
  using N = Num<T>;
  if constexpr (E == U_CELL_SUMS) {
    const int c = (int)(i % nc), chunk = (int)(i / nc);
    const int v0 = chunk * a.vpc, v1 = min(a.nv, v0 + a.vpc);
    u_chunk_moments<T>(a, a.f, nc, c, v0, v1, a.cprm[P_UX * nc + c], a.cprm[P_UY * nc + c],
                       a.part_c + (long)chunk * NMOM * nc + c, nc);
  } else if constexpr (E == U_CELL_FIN) {
    finalize_point<T, 2, 0>(a.pa, (int)i);
  } else if constexpr (E == U_BARP) {
    const int c = (int)(i % nc), v = (int)(i / nc);
    MP<T> m;
    m.load(a.cprm, nc, c);
    T gS, hS;
    model_eval<T, 2>(m, u_xi(a, v, 0), u_xi(a, v, 1), T(a.pa.k.c0), T(a.pa.k.twoK), gS, hS);
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
    const int fi = (int)(i % nf), v = (int)(i / nf);
    const T s = T(0.5 * a.dt);
    const T xx = u_xi(a, v, 0), yy = u_xi(a, v, 1);
    const T xn = a.fgeo[UF_NX * nf + fi] * xx + a.fgeo[UF_NY * nf + fi] * yy;
    const T mx = a.fgeo[UF_MX * nf + fi], my = a.fgeo[UF_MY * nf + fi];
    const int L = a.fcell[fi], R = a.fcell[nf + fi];
    const T oxL = mx - a.cgeo[UC_CX * nc + L], oyL = my - a.cgeo[UC_CY * nc + L];
    for (int comp = 0; comp < 2; ++comp) {
      const T vL = u_recon<T>(a, comp, v, L, oxL, oyL, xx * s, yy * s);
      const T vR = R >= 0 ? u_recon<T>(a, comp, v, R, mx - a.cgeo[UC_CX * nc + R], my - a.cgeo[UC_CY * nc + R],
                                       xx * s, yy * s)
                          : u_recon<T>(a, comp, v, L, -oxL, -oyL, xx * s, yy * s);
      a.fbar[((long)comp * nv + v) * nf + fi] = xn > T(0) ? vL : (xn < T(0) ? vR : T(0.5) * (vL + vR));
    }
  } else if constexpr (E == U_FACE_SUMS) {
    const int fi = (int)(i % nf), chunk = (int)(i / nf);
    const int v0 = chunk * a.vpc, v1 = min(a.nv, v0 + a.vpc);
    double* out = a.part_f + (long)chunk * NMOM * nf + fi;
    if (a.fwall[fi] >= 0) {
      // outgoing normal mass flux sum_{xi.n_in <= 0} w (xi.n_in) phi-bar_g (xi.n_in = -xi.n)
      KSum<T> m0;
      m0.zero();
      const T nx = a.fgeo[UF_NX * nf + fi], ny = a.fgeo[UF_NY * nf + fi];
      for (int v = v0; v < v1; ++v) {
        const T xin = -(nx * u_xi(a, v, 0) + ny * u_xi(a, v, 1));
        if (xin <= T(0)) m0.add(u_xi(a, v, 2) * (u_xi(a, v, 3) * (xin * a.fbar[(long)v * nf + fi])));
      }
      out[MO_0 * nf] = m0.val();
      for (int m = 1; m < NMOM; ++m) out[m * nf] = 0.0;
      return;
    }
    T sx, sy;
    u_face_shift<T>(a, fi, sx, sy);
    u_chunk_moments<T>(a, a.fbar, nf, fi, v0, v1, sx, sy, out, nf);
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
    const bool ok = point_model<T, 2>(pf, rho, ux, uy, Tm, qx, qy, mp);
    mp.c1 = T(2.0 * tau / (2.0 * tau + s));
    mp.c2 = T(s / (2.0 * tau + s));
    store_mp<T>(a.fprm, nf, fi, mp, T(FK_INTERIOR));
    if (!ok) atomicOr(a.pa.err, ERR_SINGULAR);
  } else if constexpr (E == U_FLUX) {
    const int fi = (int)(i % nf), v = (int)(i / nf);
    MP<T> m;
    m.load(a.fprm, nf, fi);
    const T xx = u_xi(a, v, 0), yy = u_xi(a, v, 1);
    const T xn = a.fgeo[UF_NX * nf + fi] * xx + a.fgeo[UF_NY * nf + fi] * yy;
    const T scale = xn * a.fgeo[UF_LEN * nf + fi];
    T gS, hS;
    model_eval<T, 2>(m, xx, yy, T(a.pa.k.c0), T(a.pa.k.twoK), gS, hS);
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
    const int c = (int)(i % nc), v = (int)(i / nc);
    const T dtA = T(a.dt / (double)a.cgeo[UC_AREA * nc + c]);
    for (int comp = 0; comp < 2; ++comp) {
      const long at = ((long)comp * nv + v) * nc + c;
      const T t = a.f[at], bp = a.barp[at];
      T div = T(0);
      for (int k = a.cf_ptr[c]; k < a.cf_ptr[c + 1]; ++k) {
        const int s = a.cf[k];
        const T F = a.flux[((long)comp * nv + v) * nf + (s >= 0 ? s : -s - 1)];
        div = s >= 0 ? div + F : div - F;
      }
      const T tp = t + T(4.0 / 3.0) * (bp - t);   // phi~+ = 4/3 phi-bar-plus - 1/3 phi~
      a.f[at] = tp - dtA * div;
    }
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
      const T xin = -(nx * xx + ny * yy);
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
    case U_CELL_SUMS: return (long)a.nc * a.nchunk;
    case U_CELL_FIN: case U_INIT_PARAMS: return a.nc;
    case U_BARP: case U_GRAD: case U_UPDATE: case U_INIT_F: return (long)a.nv * a.nc;
    case U_FACE_BAR: case U_FLUX: return (long)a.nv * a.nf;
    case U_FACE_SUMS: return (long)a.nf * a.nchunk;
    case U_FACE_FIN: case U_WALL_DEN: return a.nf;
  }
  return 0;
}

// One time step as its sequence of passes; run.template pass<E>(n) executes pass E over n
// elements (a kernel launch, or a loop).
template <class T, class Run>
inline void u_step_sequence(Run& run, const UArgs<T>& a) {
  run.template pass<U_CELL_SUMS>(u_extent(a, U_CELL_SUMS));
  run.template pass<U_CELL_FIN>(u_extent(a, U_CELL_FIN));
  run.template pass<U_BARP>(u_extent(a, U_BARP));
  run.template pass<U_GRAD>(u_extent(a, U_GRAD));
  run.template pass<U_FACE_BAR>(u_extent(a, U_FACE_BAR));
  run.template pass<U_FACE_SUMS>(u_extent(a, U_FACE_SUMS));
  run.template pass<U_FACE_FIN>(u_extent(a, U_FACE_FIN));
  run.template pass<U_FLUX>(u_extent(a, U_FLUX));
  run.template pass<U_UPDATE>(u_extent(a, U_UPDATE));
}

// Initial state phi~ = corrected Maxwellian of W0, and the wall normalisations.
template <class T, class Run>
inline void u_init_sequence(Run& run, const UArgs<T>& a) {
  run.template pass<U_INIT_PARAMS>(u_extent(a, U_INIT_PARAMS));
  run.template pass<U_INIT_F>(u_extent(a, U_INIT_F));
  run.template pass<U_WALL_DEN>(u_extent(a, U_WALL_DEN));
}

}  // namespace mlvs
