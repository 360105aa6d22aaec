// Runs the library's mapping kernel k_map (a CTA of 256 threads mapping G columns through
// shared-memory reductions) on the CPU with emulated thread blocks.  Test infrastructure.
#include "cta_shim.hpp"

#include "../../paper_2609_35258_b300/csrc/mapping.cuh"
#include "../../paper_2609_35258_b300/csrc/vspace_host.hpp"

using namespace mlvs;

namespace {

VSpace space_of(int n, const double* vt) {
  VSpace s;
  s.D = 2;
  s.xix.assign(vt, vt + n);
  s.xiy.assign(vt + n, vt + 2 * n);
  s.wx.assign(vt + 2 * n, vt + 3 * n);
  s.wy.assign(vt + 3 * n, vt + 4 * n);
  s.w.resize(n);
  for (int i = 0; i < n; ++i) s.w[i] = s.wx[i] * s.wy[i];
  return s;
}

template <int G> void run(const MapArgs& a) {
  const unsigned grid = (unsigned)((a.nitems + G - 1) / G);
  emu_launch(grid, 256, [&a] { k_map<double, double, double, 2, SRC_TILDE, G>(a); });
}

}  // namespace

// Maps nitems columns src[2][ns][nitems] from space s to space t into dst[2][nt][nitems] with
// k_map's projection and four-moment correction, G columns per block; the target space's
// mapping inverse comes from the library's host function.  Returns 0, or 1 if it is singular.
extern "C" int emu_kmap(int ns, const double* svt, int nt, const double* tvt, const int* off, const int* idx,
                        const double* wgt, const double* src, double* dst, int nitems, double R, double K, int G) {
  double sinv[16], tinv[16];
  if (!mapping_inverse(space_of(ns, svt), 2, sinv) || !mapping_inverse(space_of(nt, tvt), 2, tinv)) return 1;
  std::vector<MapItem> items(nitems);
  for (int i = 0; i < nitems; ++i) items[i] = {i, i, i};
  MapArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s = {ns, svt, sinv};
  a.t = {nt, tvt, tinv};
  a.off = off;
  a.idx = idx;
  a.wgt = wgt;
  a.src = src;
  a.src_ld = nitems;
  a.dst = dst;
  a.dst_ld = nitems;
  a.items = items.data();
  a.nitems = nitems;
  a.R = R;
  a.c0 = K + 3.0 - 2.0;
  a.cv = 0.5 * (3.0 + K) * R;
  a.twoK = 2.0 * K;
  a.correct = 1;
  if (G == 8) run<8>(a);
  else if (G == 4) run<4>(a);
  else if (G == 2) run<2>(a);
  else run<1>(a);
  return 0;
}
