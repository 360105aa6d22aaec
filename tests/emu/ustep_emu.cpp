// Runs the library's unstructured-step passes (the per-element functions its CUDA kernels
// loop over, and the same step sequence) in plain loops on the CPU.  Test infrastructure: it
// lets the tests check the passes' arithmetic and indexing against the oracle without a GPU,
// and under AddressSanitizer every buffer access against the buffer's extent.
#include "emu_shim.hpp"

#include <string>
#include <vector>

#ifdef EMU_CONTRACT
// The device functions only: fuse a * b + c into one rounding wherever the source leaves the
// compiler free to, as nvcc does for device code (with -mfma).  The host geometry stays
// uncontracted, as the library's host compiler builds it.
#pragma GCC push_options
#pragma GCC optimize("fp-contract=fast")
#include "../../paper_2609_35258_b300/csrc/ustep.cuh"
#pragma GCC pop_options
#endif
#include "../../paper_2609_35258_b300/csrc/ustep_host.hpp"

using namespace mlvs;

namespace {

template <class T> struct HostRun {
  const UArgs<T>* a;
  template <int E> void pass(long n) {
    for (long i = 0; i < n; ++i) u_elem<E, T>(*a, i);
  }
};

struct EmuBase {
  virtual ~EmuBase() = default;
  virtual int step(int n) = 0;
  virtual void read(double* g, double* h) const = 0;
  UHost u;
  UHostConfig c;
};

template <class T> struct Emu : EmuBase {
  std::vector<std::vector<unsigned char>> buf;   // one exactly sized allocation per buffer
  UArgs<T> a;
  int* err = nullptr;

  bool init(const double* W0, std::string& msg) {
    void* p[UB_N];
    buf.resize(UB_N);
    for (int b = 0; b < UB_N; ++b) {
      int type;
      size_t count;
      u_buffer(u, b, type, count);
      const size_t es = type == 0 ? sizeof(T) : type == 1 ? sizeof(int) : sizeof(double);
      buf[b].assign(count * es, 0);
      p[b] = buf[b].data();
      std::vector<T> tv;
      std::vector<int> iv;
      u_constant<T>(u, b, tv, iv);
      if (!tv.empty()) std::memcpy(p[b], tv.data(), tv.size() * sizeof(T));
      if (!iv.empty()) std::memcpy(p[b], iv.data(), iv.size() * sizeof(int));
    }
    std::memcpy(p[UB_W0], W0, 4 * sizeof(double) * u.nc);
    err = static_cast<int*>(p[UB_ERR]);
    a = u_wire<T>(u, c, p);
    HostRun<T> run{&a};
    u_init_sequence<T>(run, a);
    if (*err) {
      msg = "initial state failed";
      return false;
    }
    return true;
  }
  int step(int n) override {
    HostRun<T> run{&a};
    for (int s = 0; s < n && *err == 0; ++s) u_step_sequence<T>(run, a);
    return *err;
  }
  void read(double* g, double* h) const override {
    const size_t nc = u.nc, nv = u.nv;
    for (size_t v = 0; v < nv; ++v)
      for (size_t i = 0; i < nc; ++i) {
        g[i * nv + v] = (double)a.f[v * nc + i];
        h[i * nv + v] = (double)a.f[(nv + v) * nc + i];
      }
  }
};

}  // namespace

extern "C" {

// Returns a runner or null (msg receives the reason).
void* emu_create(const mlvs_uconfig* cfg, int n_node, const double* xy, int n_cell, const int* cell_ptr,
                 const int* cell_nodes, const int* edge_wall, const double* W0, char* msg, int msgcap) {
  std::string why;
  UHostConfig c;
  UHost u;
  why = u_config(*cfg, c);
  if (why.empty()) why = u_build_host(n_node, xy, n_cell, cell_ptr, cell_nodes, edge_wall, c, u);
  EmuBase* e = nullptr;
  if (why.empty()) {
    if (cfg->storage == MLVS_F64) e = new Emu<double>();
    else e = new Emu<float>();
    e->u = u;
    e->c = c;
    const bool ok = cfg->storage == MLVS_F64 ? static_cast<Emu<double>*>(e)->init(W0, why)
                                             : static_cast<Emu<float>*>(e)->init(W0, why);
    if (!ok) {
      delete e;
      e = nullptr;
    }
  }
  if (!e && msg && msgcap > 0) std::snprintf(msg, msgcap, "%s", why.c_str());
  return e;
}

int emu_step(void* e, int n) { return static_cast<EmuBase*>(e)->step(n); }
void emu_read(void* e, double* g, double* h) { static_cast<EmuBase*>(e)->read(g, h); }
double emu_dt(void* e) { return static_cast<EmuBase*>(e)->u.dt; }
int emu_nv(void* e) { return static_cast<EmuBase*>(e)->u.nv; }
void emu_destroy(void* e) { delete static_cast<EmuBase*>(e); }

}
