// Cell features of the level selector, one thread per cell, from the cell moments W.
//   0 log rho   1 u/sqrt(R T_ref)   2 v/sqrt(R T_ref)   3 log(T/T_ref)
//   4, 5 q/(rho (RT)^1.5)   6 dx|grad rho|/rho   7 dx|grad T|/T   8 dx|grad u|/sqrt(RT)
//   9 log10(lambda/L_ref), lambda = (mu/p) sqrt(pi R T/2)
// Gradients by central differences, neighbours wrapped (periodic sides) or clamped (others).
#pragma once

namespace mlvs {

struct FeatArgs {
  const double* W;       // [11][ncell]: rho, u, v, T, qx, qy, ...
  const double* geo;     // curvilinear: [5][ncell] J^{-T} (row-major) and the width |V|/max|S|; or null
  int nx, ny, px, py;
  double dx, dy, R, T_ref, mu_ref, omega, L_ref;
  float* out;            // [ncell][10]
};

__device__ __forceinline__ int feat_nb(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

__global__ void k_features(const FeatArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = a.nx * a.ny;
  if (c >= nc) return;
  const int i = c % a.nx, j = c / a.nx;
  const int ie = j * a.nx + feat_nb(i + 1, a.nx, a.px), iw = j * a.nx + feat_nb(i - 1, a.nx, a.px);
  const int jn = feat_nb(j + 1, a.ny, a.py) * a.nx + i, js = feat_nb(j - 1, a.ny, a.py) * a.nx + i;
  const double* rho = a.W;
  const double* u = a.W + nc;
  const double* v = a.W + 2 * (long)nc;
  const double* T = a.W + 3 * (long)nc;
  const double* qx = a.W + 4 * (long)nc;
  const double* qy = a.W + 5 * (long)nc;
  const bool two = a.ny > 1;
  auto grad = [&](const double* f, double& gx, double& gy) {
    if (a.geo) {   // index central differences through J^{-T}
      const double di = 0.5 * (f[ie] - f[iw]), dj = 0.5 * (f[jn] - f[js]);
      gx = a.geo[c] * di + a.geo[nc + c] * dj;
      gy = a.geo[2 * (long)nc + c] * di + a.geo[3 * (long)nc + c] * dj;
      return;
    }
    gx = (f[ie] - f[iw]) / (2.0 * a.dx);
    gy = two ? (f[jn] - f[js]) / (2.0 * a.dy) : 0.0;
  };
  const double h = a.geo ? a.geo[4 * (long)nc + c] : (two ? fmin(a.dx, a.dy) : a.dx);
  const double r = rho[c], t = T[c], RT = a.R * t;
  double gx, gy, gx2, gy2;
  grad(rho, gx, gy);
  const double grho = hypot(gx, gy);
  grad(T, gx, gy);
  const double gT = hypot(gx, gy);
  grad(u, gx, gy);
  grad(v, gx2, gy2);
  const double gu = sqrt(gx * gx + gy * gy + gx2 * gx2 + gy2 * gy2);
  const double mu = a.mu_ref * pow(t / a.T_ref, a.omega);
  const double lam = mu / (r * RT) * sqrt(3.14159265358979323846 * RT / 2.0);
  const double cs = sqrt(a.R * a.T_ref), q3 = r * RT * sqrt(RT);
  float* o = a.out + (long)c * 10;
  o[0] = (float)log(r);
  o[1] = (float)(u[c] / cs);
  o[2] = (float)(v[c] / cs);
  o[3] = (float)log(t / a.T_ref);
  o[4] = (float)(qx[c] / q3);
  o[5] = (float)(qy[c] / q3);
  o[6] = (float)(h * grho / r);
  o[7] = (float)(h * gT / t);
  o[8] = (float)(h * gu / sqrt(RT));
  o[9] = (float)log10(lam / a.L_ref);
}

}  // namespace mlvs
