// Host construction of the velocity spaces (Sec. 2.3, 3.1-3.2).
//
// Base grid: uniform nodes on [umin, umax] with composite Newton--Cotes weights (Boole by
// default, Simpson, trapezoid).  Level L groups one axis as follows: the centre node stays
// alone and the nodes on each side are grouped outward from the centre in runs of 2^L, the
// remainder joining the outermost group.  A merged cell has the summed weight and the
// weight-averaged coordinate (the relations under Eq. hierarchical_projection_operator).
#pragma once
#include <utility>
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <vector>

namespace mlvs {

struct Base1D {
  std::vector<double> x, w;
};

inline Base1D make_base_1d(int n, double umin, double umax, int rule) {
  if (n < 3 || (n % 2) == 0) throw std::invalid_argument("base size must be odd and >= 3");
  Base1D b;
  b.x.resize(n);
  b.w.assign(n, 0.0);
  const double h = (umax - umin) / (n - 1);
  for (int i = 0; i < n; ++i) b.x[i] = umin + h * i;
  if (rule == 0) {  // Boole: panels of four intervals
    if ((n - 1) % 4) throw std::invalid_argument("Boole rule needs 4k+1 nodes");
    const double c[5] = {7.0, 32.0, 12.0, 32.0, 7.0};
    for (int p = 0; p < (n - 1) / 4; ++p)
      for (int j = 0; j < 5; ++j) b.w[4 * p + j] += c[j] * 2.0 * h / 45.0;
  } else if (rule == 1) {  // Simpson
    for (int p = 0; p < (n - 1) / 2; ++p) {
      b.w[2 * p] += h / 3.0;
      b.w[2 * p + 1] += 4.0 * h / 3.0;
      b.w[2 * p + 2] += h / 3.0;
    }
  } else if (rule == 2) {  // trapezoid
    for (int i = 0; i < n; ++i) b.w[i] = (i == 0 || i == n - 1) ? 0.5 * h : h;
  } else {
    throw std::invalid_argument("unknown quadrature rule");
  }
  return b;
}

// Groups of one axis at level L: ranges [lo, hi) of base indices, ascending.
inline std::vector<std::pair<int, int>> groups_1d(int n, int L) {
  std::vector<std::pair<int, int>> out;
  if (L == 0) {
    for (int i = 0; i < n; ++i) out.push_back({i, i + 1});
    return out;
  }
  const int c = (n - 1) / 2;
  const int run = 1 << L;
  int ng = c / run;
  if (ng < 1) ng = 1;
  std::vector<std::pair<int, int>> right;
  for (int g = 0; g < ng; ++g) {
    const int lo = c + 1 + g * run;
    const int hi = (g == ng - 1) ? n : c + 1 + (g + 1) * run;
    right.push_back({lo, hi});
  }
  for (int g = ng - 1; g >= 0; --g) out.push_back({2 * c + 1 - right[g].second, 2 * c + 1 - right[g].first});
  out.push_back({c, c + 1});
  for (auto& r : right) out.push_back(r);
  return out;
}

// A velocity space: points with coordinates and weights, and the base rectangle each covers.
struct VSpace {
  int D = 2;
  std::vector<double> xix, xiy, w;
  std::vector<double> wx, wy;  // w = wx * wy: every merged cell is a product of axis ranges
  std::vector<int> rect;  // 4 per point: x0, x1, y0, y1 (D = 1: y0 = 0, y1 = 1)
  int nv() const { return (int)w.size(); }
};

inline void merged(const Base1D& b, int lo, int hi, double& X, double& W) {
  double sw = 0.0, sx = 0.0;
  for (int i = lo; i < hi; ++i) { sw += b.w[i]; sx += b.w[i] * b.x[i]; }
  W = sw;
  X = sx / sw;
}

// Tensor-product space with both axes grouped at level L.
inline VSpace uniform_vspace(const Base1D& b, int D, int L) {
  VSpace s;
  s.D = D;
  const int n = (int)b.x.size();
  auto gr = groups_1d(n, L);
  std::vector<double> X(gr.size()), W(gr.size());
  for (size_t g = 0; g < gr.size(); ++g) merged(b, gr[g].first, gr[g].second, X[g], W[g]);
  if (D == 1) {
    for (size_t g = 0; g < gr.size(); ++g) {
      s.xix.push_back(X[g]); s.xiy.push_back(0.0); s.w.push_back(W[g]);
      s.wx.push_back(W[g]); s.wy.push_back(1.0);
      s.rect.insert(s.rect.end(), {gr[g].first, gr[g].second, 0, 1});
    }
    return s;
  }
  for (size_t gy = 0; gy < gr.size(); ++gy)
    for (size_t gx = 0; gx < gr.size(); ++gx) {
      s.xix.push_back(X[gx]); s.xiy.push_back(X[gy]); s.w.push_back(W[gx] * W[gy]);
      s.wx.push_back(W[gx]); s.wy.push_back(W[gy]);
      s.rect.insert(s.rect.end(), {gr[gx].first, gr[gx].second, gr[gy].first, gr[gy].second});
    }
  return s;
}

// Level-L group index of every level-1 group of one axis.
inline std::vector<int> level1_parent(int n, int L) {
  auto g1 = groups_1d(n, 1);
  auto gL = groups_1d(n, L);
  std::vector<int> out(g1.size());
  for (size_t b = 0; b < g1.size(); ++b)
    for (size_t q = 0; q < gL.size(); ++q)
      if (g1[b].first >= gL[q].first && g1[b].first < gL[q].second) { out[b] = (int)q; break; }
  return out;
}

// Parent-child consistency of a block coarsening index (Sec. 3.2): kappa_eff(b) is the
// largest L <= kappa(b) such that every level-1 block of b's level-L parent has kappa >= L.
// kappa is [N1*N1] (row by, column bx) in 2-D or [N1] in 1-D, values 0..3.
inline std::vector<int> enforce_consistency(const std::vector<int>& kappa, int n, int D) {
  const int N1 = (int)groups_1d(n, 1).size();
  std::vector<std::vector<int>> par(4), pmin(4);
  std::vector<int> ng(4, 0);
  for (int L = 1; L <= 3; ++L) {
    par[L] = level1_parent(n, L);
    ng[L] = (int)groups_1d(n, L).size();
    pmin[L].assign(D == 2 ? ng[L] * ng[L] : ng[L], 1 << 30);
  }
  auto parent = [&](int L, int b) {
    return D == 2 ? par[L][b / N1] * ng[L] + par[L][b % N1] : par[L][b];
  };
  const int nb = D == 2 ? N1 * N1 : N1;
  for (int L = 1; L <= 3; ++L)
    for (int b = 0; b < nb; ++b) {
      int& m = pmin[L][parent(L, b)];
      m = std::min(m, kappa[b]);
    }
  std::vector<int> out(kappa.size(), 0);
  for (int b = 0; b < nb; ++b) {
    int best = 0;
    for (int L = 1; L <= std::min(kappa[b], 3); ++L)
      if (pmin[L][parent(L, b)] >= L) best = L;
    out[b] = best;
  }
  return out;
}

// Space of a (consistent) coarsening index: one point per merged cell, ordered by the
// lower-left base index (y major, x minor); the merged cell carries the summed weight and the
// weight-averaged coordinate.  Also fills owner[iy * n + ix] (2-D) or owner[ix] (1-D).
inline VSpace kappa_vspace(const Base1D& b, int D, const std::vector<int>& keff, std::vector<int>& owner) {
  const int n = (int)b.x.size();
  auto g1 = groups_1d(n, 1);
  const int N1 = (int)g1.size();
  std::vector<std::vector<std::pair<int, int>>> gl(4);
  std::vector<std::vector<int>> par(4);
  for (int L = 0; L <= 3; ++L) gl[L] = groups_1d(n, L);
  for (int L = 1; L <= 3; ++L) par[L] = level1_parent(n, L);
  struct Cell { int y0, x0, xa, xb, ya, yb; };
  std::vector<Cell> cells;
  if (D == 1) {
    std::vector<char> seen(4 * N1, 0);
    for (int bx = 0; bx < N1; ++bx) {
      const int L = keff[bx];
      if (L == 0) {
        for (int i = g1[bx].first; i < g1[bx].second; ++i) cells.push_back({0, i, i, i + 1, 0, 1});
      } else {
        const int p = par[L][bx];
        if (seen[L * N1 + p]) continue;
        seen[L * N1 + p] = 1;
        cells.push_back({0, gl[L][p].first, gl[L][p].first, gl[L][p].second, 0, 1});
      }
    }
  } else {
    std::vector<char> seen(4 * N1 * N1, 0);
    for (int by = 0; by < N1; ++by)
      for (int bx = 0; bx < N1; ++bx) {
        const int L = keff[by * N1 + bx];
        if (L == 0) {
          for (int iy = g1[by].first; iy < g1[by].second; ++iy)
            for (int ix = g1[bx].first; ix < g1[bx].second; ++ix) cells.push_back({iy, ix, ix, ix + 1, iy, iy + 1});
        } else {
          const int px = par[L][bx], py = par[L][by];
          const int key = (L * N1 + py) * N1 + px;
          if (seen[key]) continue;
          seen[key] = 1;
          cells.push_back({gl[L][py].first, gl[L][px].first, gl[L][px].first, gl[L][px].second,
                           gl[L][py].first, gl[L][py].second});
        }
      }
  }
  std::sort(cells.begin(), cells.end(), [](const Cell& a, const Cell& c) {
    return a.y0 != c.y0 ? a.y0 < c.y0 : a.x0 < c.x0;
  });
  VSpace s;
  s.D = D;
  owner.assign(D == 2 ? n * n : n, -1);
  for (size_t k = 0; k < cells.size(); ++k) {
    const Cell& c = cells[k];
    double X, WX, Y = 0.0, WY = 1.0;
    merged(b, c.xa, c.xb, X, WX);
    if (D == 2) merged(b, c.ya, c.yb, Y, WY);
    s.xix.push_back(X); s.xiy.push_back(Y); s.w.push_back(WX * WY);
    s.wx.push_back(WX); s.wy.push_back(WY);
    s.rect.insert(s.rect.end(), {c.xa, c.xb, c.ya, c.yb});
    for (int iy = c.ya; iy < c.yb; ++iy)
      for (int ix = c.xa; ix < c.xb; ++ix) owner[(D == 2 ? iy * n : 0) + ix] = (int)k;
  }
  return s;
}

// Inverse of the T-independent four-moment mapping matrix of a space (raw basis, unit
// weighting): rows (sum w phi, sum w xi_x phi, sum w xi_y phi, 1/2 sum w xi^2 phi),
// phi = (1, xi_x, xi_y, xi^2).  In 1-D the y row/column is the identity.
inline bool mapping_inverse(const VSpace& vs, int D, double inv[16]) {
  double A[4][4] = {{0}};
  for (int v = 0; v < vs.nv(); ++v) {
    const double w = vs.wx[v] * vs.wy[v], x = vs.xix[v], y = vs.xiy[v], x2 = x * x + y * y;
    const double phi[4] = {1.0, x, y, x2};
    const double psi[4] = {1.0, x, y, 0.5 * x2};
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) A[r][c] += w * psi[r] * phi[c];
  }
  if (D == 1) {
    for (int c = 0; c < 4; ++c) { A[2][c] = 0.0; A[c][2] = 0.0; }
    A[2][2] = 1.0;
  }
  double M[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) M[r][c] = (c < 4) ? A[r][c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
    if (!(std::fabs(M[p][c]) > 1e-300)) return false;
    for (int j = 0; j < 8; ++j) std::swap(M[c][j], M[p][j]);
    const double d = M[c][c];
    for (int j = 0; j < 8; ++j) M[c][j] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = M[r][c];
        for (int j = 0; j < 8; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) inv[4 * r + c] = M[r][4 + c];
  return true;
}

}  // namespace mlvs
