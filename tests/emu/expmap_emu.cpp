// Runs the library's positivity fallback of the state mapping (the per-item function its CUDA
// kernel calls) on the CPU for one item.  Test infrastructure.
#include "emu_shim.hpp"

#include "../../paper_2609_35258_b300/csrc/expmap.cuh"

using namespace mlvs;

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
  return expmap_item<double, double>(a, 0);
}
