// Geometry of an unstructured mesh of polygonal cells, host side: what the finite-volume
// update of Eq. explicit_update and the reconstruction of Eq. reconstruction need on general
// polygons (the two-cavity expansion of Sec. 4.5 runs on unstructured cells).
//
//  * cells are counter-clockwise node lists (CSR: cell_ptr, cell_nodes); area and centroid by
//    the shoelace formula;
//  * a face is an edge used by one cell (a boundary face) or by two cells traversing it in
//    opposite directions; faces are numbered by (smaller node, larger node); L is the first
//    cell (in cell order) using the edge, the unit normal points out of L, R is the other
//    cell or -1;
//  * each cell lists its faces in edge order, as f (the cell is L, outward normal +n) or
//    ~f = -f - 1 (the cell is R, outward normal -n);
//  * the least-squares normal matrix of a cell sums d d^T over its faces, d the centroid of
//    the cell across the face minus the cell's, or for a boundary face twice the midpoint
//    minus the centroid (the cell reflected through the face); its inverse is stored (three
//    entries of a symmetric 2 x 2) so that a gradient is that inverse times sum d (P_o - P_c);
//  * width = area / longest edge (the cell size in the time-step bound).
//
// hilbert_order sorts cells along a Hilbert curve through the bounding box of their
// centroids (16 bits per axis), so that a block of consecutive cells is spatially compact
// and its face neighbours mostly fall in the same or nearby blocks.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

namespace mlvs {

struct UMeshGeo {
  std::vector<double> area, cx, cy, width, mxx, mxy, myy;   // per cell; m = inverse normal matrix
  std::vector<int> fL, fR, fn0, fn1;                        // per face (fn0 -> fn1 as L traverses it)
  std::vector<double> nx, ny, len, midx, midy;              // per face
  std::vector<int> cf_ptr, cf;                              // per cell CSR of signed faces
};

// Builds g from the mesh; returns "" or a description of the first defect found.
inline std::string build_umesh(int n_node, const double* xy, int n_cell, const int* cell_ptr,
                               const int* cell_nodes, UMeshGeo& g) {
  if (n_node < 3 || n_cell < 1) return "need at least three nodes and one cell";
  if (cell_ptr[0] != 0) return "cell_ptr[0] must be 0";
  for (int c = 0; c < n_cell; ++c)
    if (cell_ptr[c + 1] - cell_ptr[c] < 3) return "cell " + std::to_string(c) + " has fewer than three nodes";
  const long nent = cell_ptr[n_cell];
  for (long k = 0; k < nent; ++k)
    if (cell_nodes[k] < 0 || cell_nodes[k] >= n_node) return "node index out of range";
  const auto X = [&](int n) { return xy[2 * (size_t)n]; };
  const auto Y = [&](int n) { return xy[2 * (size_t)n + 1]; };

  g.area.assign(n_cell, 0.0);
  g.cx.assign(n_cell, 0.0);
  g.cy.assign(n_cell, 0.0);
  g.width.assign(n_cell, 0.0);
  // every edge use: key (min node, max node), cell, position in the cell, direction
  struct Use { int64_t key; int cell; int pos; int n0, n1; };
  std::vector<Use> uses;
  uses.reserve(nent);
  for (int c = 0; c < n_cell; ++c) {
    const int b = cell_ptr[c], m = cell_ptr[c + 1] - b;
    double a = 0.0, sx = 0.0, sy = 0.0, longest = 0.0;
    for (int k = 0; k < m; ++k) {
      const int p = cell_nodes[b + k], q = cell_nodes[b + (k + 1) % m];
      if (p == q) return "cell " + std::to_string(c) + " repeats a node on an edge";
      const double cr = X(p) * Y(q) - X(q) * Y(p);
      a += cr;
      sx += (X(p) + X(q)) * cr;
      sy += (Y(p) + Y(q)) * cr;
      longest = std::max(longest, std::hypot(X(q) - X(p), Y(q) - Y(p)));
      uses.push_back({(int64_t)std::min(p, q) * n_node + std::max(p, q), c, k, p, q});
    }
    a *= 0.5;
    if (!(a > 0.0)) return "cell " + std::to_string(c) + " is not counter-clockwise (area <= 0)";
    g.area[c] = a;
    g.cx[c] = sx / (6.0 * a);
    g.cy[c] = sy / (6.0 * a);
    g.width[c] = a / longest;
  }
  // stable by key: the first use of an edge belongs to the lowest cell index
  std::stable_sort(uses.begin(), uses.end(), [](const Use& u, const Use& v) { return u.key < v.key; });

  g.cf_ptr.assign(cell_ptr, cell_ptr + n_cell + 1);
  g.cf.assign(nent, 0);
  g.fL.clear(); g.fR.clear(); g.fn0.clear(); g.fn1.clear();
  g.nx.clear(); g.ny.clear(); g.len.clear(); g.midx.clear(); g.midy.clear();
  for (size_t i = 0; i < uses.size();) {
    size_t j = i + 1;
    while (j < uses.size() && uses[j].key == uses[i].key) ++j;
    if (j - i > 2) return "an edge is shared by more than two cells";
    const Use& u = uses[i];
    const int f = (int)g.fL.size();
    const double ex = X(u.n1) - X(u.n0), ey = Y(u.n1) - Y(u.n0), L = std::hypot(ex, ey);
    g.fL.push_back(u.cell);
    g.fn0.push_back(u.n0);
    g.fn1.push_back(u.n1);
    g.nx.push_back(ey / L);
    g.ny.push_back(-ex / L);
    g.len.push_back(L);
    g.midx.push_back(0.5 * (X(u.n0) + X(u.n1)));
    g.midy.push_back(0.5 * (Y(u.n0) + Y(u.n1)));
    g.cf[cell_ptr[u.cell] + u.pos] = f;
    if (j - i == 2) {
      const Use& v = uses[i + 1];
      if (v.n0 != u.n1 || v.n1 != u.n0)
        return "cells " + std::to_string(u.cell) + " and " + std::to_string(v.cell) +
               " traverse a shared edge in the same direction";
      if (v.cell == u.cell) return "cell " + std::to_string(u.cell) + " uses an edge twice";
      g.fR.push_back(v.cell);
      g.cf[cell_ptr[v.cell] + v.pos] = -f - 1;
    } else {
      g.fR.push_back(-1);
    }
    i = j;
  }

  g.mxx.assign(n_cell, 0.0);
  g.mxy.assign(n_cell, 0.0);
  g.myy.assign(n_cell, 0.0);
  for (int c = 0; c < n_cell; ++c) {
    double a = 0.0, b = 0.0, d = 0.0;
    for (int k = cell_ptr[c]; k < cell_ptr[c + 1]; ++k) {
      const int s = g.cf[k], f = s >= 0 ? s : -s - 1;
      const int o = s >= 0 ? g.fR[f] : g.fL[f];
      double dx, dy;
      if (o >= 0) {
        dx = g.cx[o] - g.cx[c];
        dy = g.cy[o] - g.cy[c];
      } else {
        dx = 2.0 * (g.midx[f] - g.cx[c]);
        dy = 2.0 * (g.midy[f] - g.cy[c]);
      }
      a += dx * dx;
      b += dx * dy;
      d += dy * dy;
    }
    const double det = a * d - b * b;
    if (!(det > 1e-14 * (a * d))) return "cell " + std::to_string(c) + " has a singular least-squares matrix";
    g.mxx[c] = d / det;
    g.mxy[c] = -b / det;
    g.myy[c] = a / det;
  }
  return "";
}

// Index of (x, y) in [0, 2^16)^2 along the Hilbert curve: at each scale s (from the top
// down) the quadrant (rx, ry) contributes s^2 (3 rx XOR ry), and the coordinates are then
// reflected / swapped into the orientation of that quadrant's sub-curve.
inline uint64_t hilbert_index(uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
    const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = s - 1 - (x & (s - 1)) + (x & ~(s - 1));
        y = s - 1 - (y & (s - 1)) + (y & ~(s - 1));
      }
      std::swap(x, y);
    }
  }
  return d;
}

// order[k] = the cell visited k-th; equal keys keep the cell order.
inline void hilbert_order(int n, const double* cx, const double* cy, int* order) {
  double x0 = cx[0], x1 = cx[0], y0 = cy[0], y1 = cy[0];
  for (int i = 1; i < n; ++i) {
    x0 = std::min(x0, cx[i]); x1 = std::max(x1, cx[i]);
    y0 = std::min(y0, cy[i]); y1 = std::max(y1, cy[i]);
  }
  const double span = std::max(x1 - x0, y1 - y0);
  const double sc = span > 0.0 ? 65535.0 / span : 0.0;
  std::vector<uint64_t> key(n);
  for (int i = 0; i < n; ++i) {
    const uint32_t qx = (uint32_t)std::lround((cx[i] - x0) * sc), qy = (uint32_t)std::lround((cy[i] - y0) * sc);
    key[i] = hilbert_index(std::min(qx, 65535u), std::min(qy, 65535u));
  }
  std::iota(order, order + n, 0);
  std::stable_sort(order, order + n, [&](int a, int b) { return key[a] < key[b]; });
}

}  // namespace mlvs
