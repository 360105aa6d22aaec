// Host-side setup of the unstructured step (the arrays its passes read), shared by the CUDA
// handle and by any other runner of the same passes.
//
//  * geometry from build_umesh: per cell area, centroid, inverse least-squares normal matrix,
//    area^{3/2} (the Venkatakrishnan threshold eps^2 = (K h)^3 P_c^2 with K = 1, h = sqrt(area));
//    per face unit normal, length, midpoint, cells, wall index (boundary faces are diffuse
//    walls: every boundary edge names one of the walls);
//  * velocity space: the tensor product of a Newton-Cotes base axis (Sec. 2.3), point
//    v = iy * n + ix, tables (xi_x, xi_y, w_x, w_y) and the axis (X, W);
//  * dt = cfl * min(area / longest edge) / max |xi|_inf unless a fixed dt is given.
#pragma once
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mlvs.h"
#include "gas_host.hpp"
#include "umesh_host.hpp"
#include "ustep.cuh"
#include "vspace_host.hpp"

namespace mlvs {

struct UHostConfig {
  double R, K, Pr, omega, mu_ref, T_ref;
  double cfl, dt;                 // dt > 0: fixed
  int compat_cell, compat_face, limiter;
  int compat_moments;             // 4 or 8
  int n_base, quadrature;
  double umin, umax;
  int n_wall;
  double wall[8][3];
  int vpc;                        // velocities per chunk of the moment sums
};

struct UHost {
  int nc = 0, nf = 0, nv = 0, nax = 0, vpc = 0, nchunk = 0;
  double dt = 0.0;
  std::vector<double> cgeo, fgeo;           // [7][nc], [5][nf]
  std::vector<int> fcell, fwall, cf_ptr, cf;  // [2][nf], [nf], [nc + 1], [cf_ptr[nc]]
  std::vector<double> vt, ax;               // [4][nv], [2][nax]
};

// The host configuration of a C-ABI configuration; returns "" or what is wrong.
inline std::string u_config(const mlvs_uconfig& c, UHostConfig& u) {
  if (c.storage != MLVS_F64 && c.storage != MLVS_F32) return "storage must be MLVS_F64 or MLVS_F32";
  if (c.limiter != MLVS_LIMITER_VENKAT && c.limiter != MLVS_LIMITER_NONE)
    return "limiter must be MLVS_LIMITER_VENKAT or MLVS_LIMITER_NONE";
  u.R = c.R; u.K = c.K_internal; u.Pr = c.Pr; u.omega = c.omega; u.T_ref = c.T_ref;
  u.mu_ref = c.mu_ref > 0 ? c.mu_ref : (c.Kn > 0 ? vhs_mu_ref(c.Kn, c.omega, 1.0, c.R, c.T_ref, 1.0) : 0.0);
  u.cfl = c.cfl; u.dt = c.dt;
  u.compat_cell = c.compat_cell != 0;
  u.compat_face = c.compat_face != 0;
  u.limiter = c.limiter == MLVS_LIMITER_VENKAT ? 1 : 0;
  if (c.compat_moments != 0 && c.compat_moments != 4 && c.compat_moments != 8)
    return "compat_moments must be 4 or 8 (0: 4)";
  u.compat_moments = c.compat_moments == 8 ? 8 : 4;
  u.n_base = c.n_base; u.quadrature = c.quadrature; u.umin = c.umin; u.umax = c.umax;
  u.n_wall = c.n_wall;
  for (int w = 0; w < 8; ++w)
    for (int j = 0; j < 3; ++j) u.wall[w][j] = c.wall[w][j];
  if (c.vpc < 0) return "vpc must be >= 0 (0: 64)";
  u.vpc = c.vpc > 0 ? c.vpc : 64;
  return "";
}

inline std::string u_build_host(int n_node, const double* xy, int n_cell, const int* cell_ptr,
                                const int* cell_nodes, const int* edge_wall, const UHostConfig& c, UHost& u) {
  if (!(c.R > 0) || !(c.Pr > 0) || c.K < 0 || !(c.mu_ref > 0) || !(c.T_ref > 0)) return "bad gas constants";
  if (!(c.umax > c.umin)) return "umax must exceed umin";
  if (c.n_wall < 1 || c.n_wall > 8) return "n_wall must be 1..8";
  if (!(c.dt > 0) && !(c.cfl > 0)) return "need cfl > 0 or dt > 0";
  if (c.limiter < 0 || c.limiter > 1) return "unknown limiter";
  if (c.vpc < 1) return "vpc must be >= 1";
  for (int w = 0; w < c.n_wall; ++w)
    if (!(c.wall[w][2] > 0)) return "wall temperatures must be > 0";
  UMeshGeo g;
  const std::string why = build_umesh(n_node, xy, n_cell, cell_ptr, cell_nodes, g);
  if (!why.empty()) return why;
  Base1D b;
  try {
    b = make_base_1d(c.n_base, c.umin, c.umax, c.quadrature);
  } catch (const std::exception& e) {
    return e.what();
  }
  const int nc = n_cell, nf = (int)g.fL.size(), n = c.n_base;
  u.nc = nc;
  u.nf = nf;
  u.nax = n;
  u.nv = n * n;
  u.vpc = c.vpc;
  u.nchunk = (u.nv + c.vpc - 1) / c.vpc;
  u.cgeo.assign((size_t)7 * nc, 0.0);
  for (int i = 0; i < nc; ++i) {
    u.cgeo[0 * (size_t)nc + i] = g.area[i];
    u.cgeo[1 * (size_t)nc + i] = g.cx[i];
    u.cgeo[2 * (size_t)nc + i] = g.cy[i];
    u.cgeo[3 * (size_t)nc + i] = g.mxx[i];
    u.cgeo[4 * (size_t)nc + i] = g.mxy[i];
    u.cgeo[5 * (size_t)nc + i] = g.myy[i];
    u.cgeo[6 * (size_t)nc + i] = g.area[i] * std::sqrt(g.area[i]);
  }
  u.fgeo.assign((size_t)5 * nf, 0.0);
  u.fcell.assign((size_t)2 * nf, -1);
  u.fwall.assign(nf, -1);
  for (int f = 0; f < nf; ++f) {
    u.fgeo[0 * (size_t)nf + f] = g.nx[f];
    u.fgeo[1 * (size_t)nf + f] = g.ny[f];
    u.fgeo[2 * (size_t)nf + f] = g.len[f];
    u.fgeo[3 * (size_t)nf + f] = g.midx[f];
    u.fgeo[4 * (size_t)nf + f] = g.midy[f];
    u.fcell[f] = g.fL[f];
    u.fcell[(size_t)nf + f] = g.fR[f];
  }
  u.cf_ptr = g.cf_ptr;
  u.cf = g.cf;
  // wall index of every boundary face, from the edge of its cell
  for (int cell = 0; cell < nc; ++cell)
    for (int k = cell_ptr[cell]; k < cell_ptr[cell + 1]; ++k) {
      const int s = g.cf[k];
      if (s < 0 || g.fR[s] >= 0) continue;
      const int w = edge_wall ? edge_wall[k] : 0;
      if (w < 0 || w >= c.n_wall) return "boundary edge of cell " + std::to_string(cell) + " names no wall";
      u.fwall[s] = w;
    }
  u.vt.assign((size_t)4 * u.nv, 0.0);
  u.ax.assign((size_t)2 * n, 0.0);
  double xmax = 0.0;
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix) {
      const size_t v = (size_t)iy * n + ix;
      u.vt[v] = b.x[ix];
      u.vt[(size_t)u.nv + v] = b.x[iy];
      u.vt[(size_t)2 * u.nv + v] = b.w[ix];
      u.vt[(size_t)3 * u.nv + v] = b.w[iy];
    }
  for (int i = 0; i < n; ++i) {
    u.ax[i] = b.x[i];
    u.ax[(size_t)n + i] = b.w[i];
    xmax = std::max(xmax, std::fabs(b.x[i]));
  }
  if (c.dt > 0) {
    u.dt = c.dt;
  } else {
    double wmin = g.width[0];
    for (int i = 1; i < nc; ++i) wmin = std::min(wmin, g.width[i]);
    u.dt = c.cfl * wmin / xmax;
  }
  return "";
}

// Buffers of the step: type (0 = compute type T, 1 = int, 2 = double) and element count.
enum { UB_CGEO = 0, UB_FGEO, UB_VT, UB_AX, UB_FCELL, UB_FWALL, UB_CFPTR, UB_CF, UB_W0, UB_F, UB_BARP, UB_GRAD,
       UB_FBAR, UB_FLUX, UB_PARTC, UB_PARTF, UB_CPRM, UB_FPRM, UB_W, UB_WDEN, UB_ERR, UB_CPRM8, UB_FPRM8,
       UB_N };

inline void u_buffer(const UHost& u, int b, int& type, size_t& count) {
  const size_t nc = u.nc, nf = u.nf, nv = u.nv, ch = u.nchunk;
  switch (b) {
    case UB_CGEO: type = 0; count = 7 * nc; return;
    case UB_FGEO: type = 0; count = 5 * nf; return;
    case UB_VT: type = 0; count = 4 * nv; return;
    case UB_AX: type = 0; count = 2 * (size_t)u.nax; return;
    case UB_FCELL: type = 1; count = 2 * nf; return;
    case UB_FWALL: type = 1; count = nf; return;
    case UB_CFPTR: type = 1; count = nc + 1; return;
    case UB_CF: type = 1; count = u.cf.size(); return;
    case UB_W0: type = 2; count = 4 * nc; return;
    case UB_F: case UB_BARP: type = 0; count = 2 * nv * nc; return;
    case UB_GRAD: type = 0; count = 4 * nv * nc; return;
    case UB_FBAR: case UB_FLUX: type = 0; count = 2 * nv * nf; return;
    case UB_PARTC: type = 2; count = ch * NMOM * nc; return;
    case UB_PARTF: type = 2; count = ch * NMOM * nf; return;
    case UB_CPRM: type = 0; count = (size_t)NP * nc; return;
    case UB_FPRM: type = 0; count = (size_t)NP * nf; return;
    case UB_W: type = 2; count = 11 * nc; return;
    case UB_WDEN: type = 2; count = nf; return;
    case UB_ERR: type = 1; count = ERR_WORDS; return;   // error bits and the first failing point
    case UB_CPRM8: type = 0; count = 4 * nc; return;
    case UB_FPRM8: type = 0; count = 4 * nf; return;
  }
  type = 0;
  count = 0;
}

// The passes' arguments over buffers p[UB_N] (all of one address space).
template <class T>
inline UArgs<T> u_wire(const UHost& u, const UHostConfig& c, void* const* p) {
  UArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  PointArgs& pa = a.pa;
  pa.k.ncell = u.nc;
  pa.k.nv = u.nv;
  pa.k.vpc = u.vpc;
  pa.k.nchunk = u.nchunk;
  pa.k.nax = u.nax;
  pa.k.dt = u.dt;
  pa.k.c0 = c.K + 3.0 - 2.0;
  pa.k.twoK = 2.0 * c.K;
  pa.gas = GasDev{c.R, c.K, c.Pr, c.omega, c.mu_ref, c.T_ref};
  pa.part = static_cast<const double*>(p[UB_PARTC]);
  pa.npt = u.nc;
  pa.nwork = u.nc;
  pa.cprm = p[UB_CPRM];
  pa.prm_out = p[UB_CPRM];
  pa.W = static_cast<double*>(p[UB_W]);
  pa.vt = p[UB_VT];
  pa.ax = p[UB_AX];
  pa.compat = c.compat_cell;
  pa.err = static_cast<int*>(p[UB_ERR]);
  a.compat_face = c.compat_face;
  a.compat8 = c.compat_moments == 8;
  a.nc = u.nc;
  a.nf = u.nf;
  a.nv = u.nv;
  a.vpc = u.vpc;
  a.nchunk = u.nchunk;
  a.limiter = c.limiter;
  a.dt = u.dt;
  for (int w = 0; w < 8; ++w)
    for (int j = 0; j < 3; ++j) a.wall[w][j] = c.wall[w][j];
  a.cgeo = static_cast<const T*>(p[UB_CGEO]);
  a.fgeo = static_cast<const T*>(p[UB_FGEO]);
  a.fcell = static_cast<const int*>(p[UB_FCELL]);
  a.fwall = static_cast<const int*>(p[UB_FWALL]);
  a.cf_ptr = static_cast<const int*>(p[UB_CFPTR]);
  a.cf = static_cast<const int*>(p[UB_CF]);
  a.W0 = static_cast<const double*>(p[UB_W0]);
  a.f = static_cast<T*>(p[UB_F]);
  a.barp = static_cast<T*>(p[UB_BARP]);
  a.grad = static_cast<T*>(p[UB_GRAD]);
  a.fbar = static_cast<T*>(p[UB_FBAR]);
  a.flux = static_cast<T*>(p[UB_FLUX]);
  a.part_c = static_cast<double*>(p[UB_PARTC]);
  a.part_f = static_cast<double*>(p[UB_PARTF]);
  a.cprm = static_cast<T*>(p[UB_CPRM]);
  a.fprm = static_cast<T*>(p[UB_FPRM]);
  a.cprm8 = static_cast<T*>(p[UB_CPRM8]);
  a.fprm8 = static_cast<T*>(p[UB_FPRM8]);
  a.W = static_cast<double*>(p[UB_W]);
  a.wden = static_cast<double*>(p[UB_WDEN]);
  return a;
}

// Host contents of the constant buffers, in the compute type where the buffer has it.
template <class T>
inline void u_constant(const UHost& u, int b, std::vector<T>& tv, std::vector<int>& iv) {
  const std::vector<double>* d = b == UB_CGEO ? &u.cgeo : b == UB_FGEO ? &u.fgeo : b == UB_VT ? &u.vt
                                 : b == UB_AX ? &u.ax : nullptr;
  if (d) tv.assign(d->begin(), d->end());
  const std::vector<int>* i = b == UB_FCELL ? &u.fcell : b == UB_FWALL ? &u.fwall : b == UB_CFPTR ? &u.cf_ptr
                              : b == UB_CF ? &u.cf : nullptr;
  if (i) iv = *i;
}

}  // namespace mlvs
