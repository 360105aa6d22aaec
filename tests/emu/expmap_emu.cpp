// Runs the library's per-item state mappings (the functions its CUDA kernels call) on the CPU
// for one item: the positivity fallback and the nine-moment mapping.  Test infrastructure.
#include "emu_shim.hpp"

#include "../../paper_2609_35258_b300/csrc/map9.cuh"

using namespace mlvs;

namespace {

MapArgs one_item(int ns, const double* svt, int nt, const double* tvt, const int* off, const int* idx,
                 const double* wgt, const double* src, double* dst, const MapItem* it) {
  MapArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s.nv = ns;
  a.s.vt = svt;
  a.t.nv = nt;
  a.t.vt = tvt;
  a.off = off;
  a.idx = idx;
  a.wgt = wgt;
  a.src = src;
  a.src_ld = 1;
  a.dst = dst;
  a.dst_ld = 1;
  a.items = it;
  a.nitems = 1;
  return a;
}

}  // namespace

extern "C" int emu_map9(int ns, const double* svt, int nt, const double* tvt, const int* off, const int* idx,
                        const double* wgt, const double* src, double* dst) {
  const MapItem it = {0, 0, 0};
  const MapArgs a = one_item(ns, svt, nt, tvt, off, idx, wgt, src, dst, &it);
  return map9_item<double, double, double, SRC_TILDE>(a, 0) ? 1 : 0;
}

extern "C" int emu_expmap(int ns, const double* svt, int nt, const double* tvt, const int* off, const int* idx,
                          const double* wgt, const double* src, double* dst) {
  MapArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s.nv = ns;
  a.s.vt = svt;
  a.t.nv = nt;
  a.t.vt = tvt;
  a.off = off;
  a.idx = idx;
  a.wgt = wgt;
  a.src = src;
  a.src_ld = 1;
  a.dst = dst;
  a.dst_ld = 1;
  const MapItem it = {0, 0, 0};
  a.items = &it;
  a.nitems = 1;
  return expmap_item<double, double, double, SRC_TILDE>(a, 0);
}
