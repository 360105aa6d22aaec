// Tile kernels of one DUGKS step on a structured Cartesian mesh (Sec. 2.2).
//
// A CTA owns a TX x TY tile of cells and a contiguous chunk of velocities, processed VB
// velocities per barrier round.  Per round it stages in shared memory
//   phase 1  phi-bar-plus of the tile and its two-cell halo (the derived conversion
//            phi-bar-plus = phi~ + b (phi^S - phi~) of Sec. 2.2);
//   phase 2  limited slopes (Eq. reconstruction) of the cells that can be upwind of a face;
//   phase 3  the face phi-bar of the upwind side by the characteristic
//            (Eq. bar_phi_transport).  MODE 0 accumulates the face moments over the chunk
//            (input of Eq. W_from_bar).  MODE 1 recovers the face phi (Eq. recover_phi);
//   phase 4  (MODE 1) Eq. explicit_update of the tile's cells, the store of phi~^{n+1} and
//            the cell moments of the stored values (input of Eq. discrete_W / discrete_q).
// Velocity is uniform across the CTA inside a round, so the upwind choice by sign(xi.n) is
// a uniform branch.  Halo sources are wrapped (periodic sides) or clamped (ghost copies of
// the boundary cell on the other sides).
#pragma once
#include "mlvs_common.cuh"

namespace mlvs {

struct TileArgs {
  StepConst k;           // mesh-wide constants (k.ncell, k.nface: the whole mesh)
  const void* f_in;      // [2][nv][nslot] phi~ of this level's cells (storage type)
  void* f_out;           // [2][nv][nslot] (MODE 1)
  int nslot;             // cells on this level
  const void* cparam;    // [NP][nslot]  type T
  const void* fparam;    // [NP][nface]  type T (MODE 1)
  const void* vt;        // [4][nv]      type T
  double* part;          // MODE 0: [nchunk][NMOM][nface], MODE 1: [nchunk][NMOM][nslot]
  const int* tiles;      // tile ids launched for this level
  int ntx, nty;          // tiles per axis of the mesh
  int level;
  const int* lvl_of;     // [ncell] level of every cell
  const int* slot_of;    // [ncell] column of every cell in its level's arrays
  const int* ghost_of;   // [ncell] column in this level's ghost array, or -1 (may be null)
  const void* ghost;     // (T) [2][nv][nghost] phi-bar-plus of other-level stencil cells on this space
  int nghost;
  const unsigned char* frole;  // [nface] role of every face on this level (FR_*)
  const int* fslot;      // [nface] column in X (FR_CROSS) or Y (FR_RECV)
  void* X;               // (T) [2][nv][nX] microfluxes of the cross faces evaluated here
  int nX;
  const void* Y;         // (T) [2][nv][nY] microfluxes mapped here from other face spaces
  int nY;
  const void* ucell;     // (T) [2][ncell] cell velocities (face moment shifts)
  const void* cgeo;      // curvilinear (T) [5][ncell]: J^{-T} (4, row-major), dt/|V|
  const void* fgeo;      // curvilinear (T) [7][nface]: normal (2), |S|, x_b - x_L (2), x_b - x_R (2)
  const unsigned* step;  // device step counter (BF16 stochastic rounding: the random bits
  unsigned salt;         // come from hash(step, salt, cell, velocity); salt: instance, level)
};

// Advance the device step counter of an instance (one thread; part of every BF16 step, so a
// captured graph draws new random bits on every replay).
__global__ void k_step_counter(unsigned* c) { *c += 1u; }


template <int TX, int TY, int D> struct TileGeom {
  static constexpr int NT = TX * TY;
  static constexpr int EW = TX + 4;
  static constexpr int EH = (D == 2) ? TY + 4 : 1;
  static constexpr int NEXT = EW * EH;
  static constexpr int NHALO = NEXT - NT;
  static constexpr int SW = TX + 2;
  static constexpr int SH = (D == 2) ? TY + 2 : 1;
  static constexpr int NSL = SW * SH;
  static constexpr int NFXL = (TX + 1) * TY;
  static constexpr int NFYL = (D == 2) ? TX * (TY + 1) : 0;
  static constexpr int NF = NFXL + NFYL;
  // ext index of tile-local cell (x, y), x in [-2, TX+1], y in [-2, TY+1]
  static __device__ __forceinline__ int eidx(int x, int y) {
    return (D == 2) ? (y + 2) * EW + (x + 2) : (x + 2);
  }
  // slope index of tile-local cell (x, y), x in [-1, TX], y in [-1, TY]
  static __device__ __forceinline__ int sidx(int x, int y) {
    return (D == 2) ? (y + 1) * SW + (x + 1) : (x + 1);
  }
  // k-th halo position of the extended tile
  static __device__ __forceinline__ void halo_pos(int k, int& x, int& y) {
    if (D == 1) {
      x = (k < 2) ? k - 2 : TX + (k - 2);
      y = 0;
      return;
    }
    if (k < 2 * EW) { y = k / EW - 2; x = k % EW - 2; return; }
    k -= 2 * EW;
    if (k < 2 * EW) { y = TY + k / EW; x = k % EW - 2; return; }
    k -= 2 * EW;
    y = k / 4;
    const int c = k % 4;
    x = (c < 2) ? c - 2 : TX + (c - 2);
  }
  // tile-local coordinates of face f: x-faces first, then y-faces
  static __device__ __forceinline__ void face_pos(int f, int& dir, int& li, int& lj) {
    if (f < NFXL) { dir = 0; li = f % (TX + 1); lj = f / (TX + 1); }
    else { f -= NFXL; dir = 1; li = f % TX; lj = f / TX; }
  }
};

// Shared-memory layout of a tile kernel (bytes), identical on host and device.
template <class T, int TX, int TY, int D, int VB, int MODE, bool CV = false> struct TileSmem {
  using G = TileGeom<TX, TY, D>;
  static constexpr size_t P = 0;                                           // T [VB][2][NEXT]
  static constexpr size_t SL = P + sizeof(T) * VB * 2 * G::NEXT;            // T [VB][4][NSL]
  static constexpr size_t F = SL + sizeof(T) * VB * 4 * G::NSL;             // T [VB][2][NF]   (MODE 1)
  static constexpr size_t FP = F + (MODE == 1 ? sizeof(T) * VB * 2 * G::NF : 0);  // T [16][NF] (MODE 1)
  static constexpr size_t ACC = FP + (MODE == 1 ? sizeof(T) * 16 * G::NF : 0);     // T [16][NF] (MODE 0)
  static constexpr size_t META = ACC + (MODE == 0 ? sizeof(T) * 16 * G::NF : 0);   // int [2][NF]
  static constexpr size_t JT = META + sizeof(int) * 2 * G::NF;                      // T [4][NSL] (CV)
  static constexpr size_t FG = JT + (CV ? sizeof(T) * 4 * G::NSL : 0);               // T [7][NF]  (CV)
  static constexpr size_t BYTES = FG + (CV ? sizeof(T) * 7 * G::NF : 0);
};

__device__ __forceinline__ int wrap_or_clamp(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// van Leer limited slope (reading of Eq. reconstruction): 2ab/(a+b)/h for a, b of equal
// strict sign (ab > 0; an underflowing product counts as 0), else 0.  limiter == 1: central difference (a+b)/(2h).
template <class T>
__device__ __forceinline__ T limited(T a, T b, T inv_h, int limiter) {
  using N = Num<T>;
  if (limiter) return N::mul(N::mul(T(0.5), N::add(a, b)), inv_h);
  const T ab = N::mul(a, b);
  return (ab > T(0)) ? N::mul(N::dv(N::mul(T(2), ab), N::add(a, b)), inv_h) : T(0);
}

// face metadata word: bit 0 valid, bit 1 owned (MODE 0 accumulates), bits 2-4 kind, role above
enum { FM_VALID = 1, FM_OWNED = 2 };

// Face accumulators: Kahan pairs (s, c) for M0, MX, MY, E in slots 0..7, plain sums of
// Gxx, Gxy, Gyy, Jx, Jy in slots 8..12.
template <class T>
__device__ __forceinline__ void fold_partials(T (&acc)[13], const T (&part)[9]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const T sum = acc[2 * p], cmp = acc[2 * p + 1];
    const T y = part[p] - cmp;
    const T t = sum + y;
    acc[2 * p + 1] = (t - sum) - y;
    acc[2 * p] = t;
  }
#pragma unroll
  for (int p = 4; p < 9; ++p) acc[4 + p] += part[p];
}
template <class T>
__device__ __forceinline__ void fold_partials_smem(T* acc, int st, const T (&part)[9]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const T sum = acc[2 * p * st], cmp = acc[(2 * p + 1) * st];
    const T y = part[p] - cmp;
    const T t = sum + y;
    acc[(2 * p + 1) * st] = (t - sum) - y;
    acc[2 * p * st] = t;
  }
#pragma unroll
  for (int p = 4; p < 9; ++p) acc[(4 + p) * st] += part[p];
}
template <class T, int D>
__device__ __forceinline__ void write_partials(const T (&acc)[13], double* P, long st) {
  P[MO_0 * st] = (double)acc[0] - (double)acc[1];
  P[MO_X * st] = (double)acc[2] - (double)acc[3];
  P[MO_Y * st] = (D == 2) ? (double)acc[4] - (double)acc[5] : 0.0;
  P[MO_E * st] = (double)acc[6] - (double)acc[7];
  P[MO_GXX * st] = (double)acc[8];
  P[MO_GXY * st] = (double)acc[9];
  P[MO_GYY * st] = (double)acc[10];
  P[MO_JX * st] = (double)acc[11];
  P[MO_JY * st] = (double)acc[12];
}
template <class T, int D>
__device__ __forceinline__ void write_partials_smem(const T* acc, int sa, double* P, long st) {
  P[MO_0 * st] = (double)acc[0] - (double)acc[sa];
  P[MO_X * st] = (double)acc[2 * sa] - (double)acc[3 * sa];
  P[MO_Y * st] = (D == 2) ? (double)acc[4 * sa] - (double)acc[5 * sa] : 0.0;
  P[MO_E * st] = (double)acc[6 * sa] - (double)acc[7 * sa];
  P[MO_GXX * st] = (double)acc[8 * sa];
  P[MO_GXY * st] = (double)acc[9 * sa];
  P[MO_GYY * st] = (double)acc[10 * sa];
  P[MO_JX * st] = (double)acc[11 * sa];
  P[MO_JY * st] = (double)acc[12 * sa];
}

// ML = false: the level holds every cell of the mesh (one velocity space), so every stencil
// position is an own cell in natural order and every face is a normal face; the level
// tables are not read.
// CV: structured curvilinear mesh (2-D): slopes along the index directions turned into
// physical slopes with the cell's J^{-T}, faces with their own normals, areas and centroid
// offsets (precomputed per face, so the two tiles of a face read the same values), and the
// update scaled by dt/|V|.
template <class S, class T, int D, int TX, int TY, int VB, int MODE, bool ML, bool CV>
__global__ void __launch_bounds__(TX * TY)
k_tile(const TileArgs a, int limiter) {
  using G = TileGeom<TX, TY, D>;
  using L = TileSmem<T, TX, TY, D, VB, MODE, CV>;
  static_assert(!CV || D == 2, "curvilinear meshes are two-dimensional");
  using N = Num<T>;
  static_assert(G::NHALO <= G::NT, "halo larger than the thread count");
  static_assert(G::NSL <= 2 * G::NT, "slope rectangle larger than two per thread");
  static_assert(G::NF <= 3 * G::NT, "faces larger than three per thread");
  extern __shared__ __align__(16) unsigned char smem[];
  T* sP = reinterpret_cast<T*>(smem + L::P);
  T* sS = reinterpret_cast<T*>(smem + L::SL);
  T* sF = reinterpret_cast<T*>(smem + L::F);
  T* sFP = reinterpret_cast<T*>(smem + L::FP);
  T* sAcc = reinterpret_cast<T*>(smem + L::ACC);
  int* sMeta = reinterpret_cast<int*>(smem + L::META);
  T* sJt = reinterpret_cast<T*>(smem + L::JT);
  T* sFG = reinterpret_cast<T*>(smem + L::FG);
  const T* __restrict__ cg = reinterpret_cast<const T*>(a.cgeo);
  const T* __restrict__ fg = reinterpret_cast<const T*>(a.fgeo);

  const StepConst& k = a.k;
  const S* __restrict__ fin = reinterpret_cast<const S*>(a.f_in);
  const T* __restrict__ cp = reinterpret_cast<const T*>(a.cparam);
  const T* __restrict__ fp = reinterpret_cast<const T*>(a.fparam);
  const T* __restrict__ vt = reinterpret_cast<const T*>(a.vt);
  const T* __restrict__ gst = reinterpret_cast<const T*>(a.ghost);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.ucell);
  const long ns = a.nslot;
  const long ng = a.nghost;
  const long nv = k.nv;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  unsigned seed = 0;
  if constexpr (MODE == 1 && sizeof(S) == 2) seed = hash32(*a.step * 0x632be5abu + a.salt);
  const int tile = a.tiles[blockIdx.x];
  const int bx = tile % a.ntx, by = tile / a.ntx;
  const int x0 = bx * TX, y0 = by * TY;
  const int chunk = blockIdx.y;
  const int v0 = chunk * k.vpc;
  const int v1 = min(k.nv, v0 + k.vpc);

  // ---- extended positions: own cell + at most one halo cell.  A position holds a cell of
  // this level (phi~ + parameters -> phi-bar-plus), a ghost (phi-bar-plus mapped to this
  // space), or nothing (never read by a face evaluated here).
  auto classify = [&](int ex, int ey, int& kind, long& base, long& ld) {
    const int c = wrap_or_clamp(y0 + ey, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + ex, k.nx, k.px);
    kind = 0; base = 0; ld = 0;
    if (!ML) { kind = 1; base = c; ld = ns; }
    else if (a.lvl_of[c] == a.level) { kind = 1; base = a.slot_of[c]; ld = ns; }
    else if (a.ghost_of && a.ghost_of[c] >= 0) { kind = 2; base = a.ghost_of[c]; ld = ng; }
    return c;
  };
  const int ey0 = (D == 2) ? ty : 0;
  int kind0, kind1 = 0;
  long col0, ld0, col1 = 0, ld1 = 0;
  const int c0g = classify(tx, ey0, kind0, col0, ld0);
  const bool own_active = (x0 + tx < k.nx) && (D == 1 || y0 + ty < k.ny) && kind0 == 1 &&
                          c0g == (y0 + ey0) * k.nx + (x0 + tx);
  int ex1 = 0, ey1 = 0;
  if (tid < G::NHALO) {
    G::halo_pos(tid, ex1, ey1);
    classify(ex1, ey1, kind1, col1, ld1);
  }
  MP<T> m0, m1;
  if (kind0 == 1) m0.load(cp, ns, col0);
  if (kind1 == 1) m1.load(cp, ns, col1);
  const int e0 = G::eidx(tx, ey0);
  const int e1 = (tid < G::NHALO) ? G::eidx(ex1, ey1) : 0;

  // ---- face metadata (and MODE 1 parameters, MODE 0 shifts/accumulators) in shared memory
  for (int f = tid; f < G::NF; f += G::NT) {
    int dir, li, lj;
    G::face_pos(f, dir, li, lj);
    const int gi = x0 + li, gj = y0 + lj;
    int meta = 0, fid = -1, role = FR_NONE;
    if (dir == 0) {
      if (gi <= k.nx && (D == 1 || gj < k.ny)) {
        const int pi = (k.px && gi == k.nx) ? 0 : gi;
        fid = ((D == 2) ? gj : 0) * k.nfx + pi;
        role = ML ? a.frole[fid] : FR_NORMAL;
        meta = FM_VALID;
        if ((gi < k.nx) ? (li < TX) : !k.px) meta |= FM_OWNED;
        if (!k.px && gi == 0 && k.bc[0] == BC_WALL) meta |= FK_WALL_LO << 2;
        if (!k.px && gi == k.nx && k.bc[1] == BC_WALL) meta |= FK_WALL_HI << 2;
        if (!k.px && gi == 0 && k.bc[0] == BC_FREE) meta |= FK_FREE_LO << 2;
        if (!k.px && gi == k.nx && k.bc[1] == BC_FREE) meta |= FK_FREE_HI << 2;
      }
    } else {
      if (gi < k.nx && gj <= k.ny) {
        const int pj = (k.py && gj == k.ny) ? 0 : gj;
        fid = k.nfx * k.ny + pj * k.nx + gi;
        role = ML ? a.frole[fid] : FR_NORMAL;
        meta = FM_VALID;
        if ((gj < k.ny) ? (lj < TY) : !k.py) meta |= FM_OWNED;
        if (!k.py && gj == 0 && k.bc[2] == BC_WALL) meta |= FK_WALL_LO << 2;
        if (!k.py && gj == k.ny && k.bc[3] == BC_WALL) meta |= FK_WALL_HI << 2;
        if (!k.py && gj == 0 && k.bc[2] == BC_FREE) meta |= FK_FREE_LO << 2;
        if (!k.py && gj == k.ny && k.bc[3] == BC_FREE) meta |= FK_FREE_HI << 2;
      }
    }
    if (role == FR_NONE) meta = 0;
    meta |= role << 5;
    sMeta[f] = meta;
    sMeta[G::NF + f] = (role == FR_CROSS || role == FR_RECV) ? a.fslot[fid] : fid;
    if constexpr (CV) {
#pragma unroll
      for (int p = 0; p < 7; ++p) sFG[p * G::NF + f] = fid >= 0 ? fg[(long)p * k.nface + fid] : T(0);
    }
    if (MODE == 1 && (role == FR_NORMAL || role == FR_CROSS)) {
#pragma unroll
      for (int p = 0; p < 13; ++p) sFP[p * G::NF + f] = fp[(long)p * k.nface + fid];
    }
    if (MODE == 0) {
      T shx = T(0), shy = T(0);
      if (fid >= 0) {
        const int xl = (dir == 0) ? li - 1 : li, yl = (dir == 0) ? lj : lj - 1;
        const int sL = wrap_or_clamp(y0 + yl, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + xl, k.nx, k.px);
        const int sR = wrap_or_clamp(y0 + lj, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + li, k.nx, k.px);
        shx = T(0.5) * (uc[sL] + uc[sR]);
        if (D == 2) shy = T(0.5) * (uc[k.ncell + sL] + uc[k.ncell + sR]);
      }
#pragma unroll
      for (int p = 0; p < 13; ++p) sAcc[p * G::NF + f] = T(0);
      sAcc[13 * G::NF + f] = shx;   // slots 13, 14 hold the shift (never accumulated)
      sAcc[14 * G::NF + f] = shy;
      // the face partials of this level are read only where the role says so
      if (fid >= 0 && (role == FR_NORMAL || role == FR_CROSS)) sMeta[G::NF + f] = fid;
    }
  }

  // curvilinear: J^{-T} of the slope rectangle (ghost positions take the boundary cell's)
  if constexpr (CV) {
    for (int q = tid; q < G::NSL; q += G::NT) {
      const int sx = q % G::SW - 1, sy = q / G::SW - 1;
      const int c = wrap_or_clamp(y0 + sy, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + sx, k.nx, k.px);
#pragma unroll
      for (int p = 0; p < 4; ++p) sJt[p * G::NSL + q] = cg[(long)p * k.ncell + c];
    }
  }
  // MODE 0 accumulators of the thread's first two faces in registers:
  // Kahan (s, c) for M0, MX, MY, E, plain for Gxx, Gxy, Gyy, Jx, Jy
  T ra[2][13];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int p = 0; p < 13; ++p) ra[q][p] = T(0);
  // MODE 1 accumulators of the own cell
  KSum<T> c0k, cxk, cyk, cek;
  c0k.zero(); cxk.zero(); cyk.zero(); cek.zero();
  T cgxx = T(0), cgxy = T(0), cgyy = T(0), cjx = T(0), cjy = T(0);

  const T c0 = T(k.c0), twoK = T(k.twoK);
  const T s = T(0.5 * k.dt);
  const T hdx = T(0.5 * k.dx), hdy = T(0.5 * k.dy);
  const T idx_ = T(1.0 / k.dx), idy_ = T(1.0 / k.dy);
  T lamx = T(k.dt / k.dx), lamy = T(k.dt / k.dy);
  if constexpr (CV) {
    if (own_active) lamx = lamy = cg[4L * k.ncell + c0g];   // dt / |V| of the own cell
  }
  S* __restrict__ fout = reinterpret_cast<S*>(a.f_out);
  T* __restrict__ Xo = reinterpret_cast<T*>(a.X);
  const T* __restrict__ Yi = reinterpret_cast<const T*>(a.Y);
  __syncthreads();
  // shifts of the thread's register-held faces (MODE 0)
  T fshx[2] = {T(0), T(0)}, fshy[2] = {T(0), T(0)};
  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int f = tid + q * G::NT;
      if (f < G::NF) { fshx[q] = sAcc[13 * G::NF + f]; fshy[q] = sAcc[14 * G::NF + f]; }
    }
  }

  // loads of one velocity for a position of each kind
  auto load_pos = [&](int kind, long col, int v, T& g, T& h) {
    if (!ML || kind == 1) {
      g = ldf<S, T>(fin + (long)v * ns + col);
      h = ldf<S, T>(fin + (nv + v) * ns + col);
    } else if (kind == 2) {
      g = gst[(long)v * ng + col];
      h = gst[(nv + v) * ng + col];
    } else {
      g = T(0);
      h = T(0);
    }
  };

  // register prefetch of the first round
  T ng0[VB], nh0[VB], ng1[VB], nh1[VB];
#pragma unroll
  for (int b = 0; b < VB; ++b) {
    const int v = v0 + b;
    ng0[b] = nh0[b] = ng1[b] = nh1[b] = T(0);
    if (v < v1) {
      load_pos(kind0, col0, v, ng0[b], nh0[b]);
      load_pos(kind1, col1, v, ng1[b], nh1[b]);
    }
  }

  for (int vb0 = v0; vb0 < v1; vb0 += VB) {
    T g0[VB], h0[VB], dg0[VB], dh0[VB];
    T xixb[VB], xiyb[VB], wxb[VB], wyb[VB];
    // ---- phase 1: phi-bar-plus on the extended tile, and the prefetch of the next round
#pragma unroll
    for (int b = 0; b < VB; ++b) {
      const int v = vb0 + b;
      const bool on = v < v1;
      const int vv = on ? v : v0;
      xixb[b] = vt[vv];
      xiyb[b] = (D == 2) ? vt[nv + vv] : T(0);
      wxb[b] = vt[2 * nv + vv];
      wyb[b] = vt[3 * nv + vv];
      g0[b] = ng0[b]; h0[b] = nh0[b];
      const T g1 = ng1[b], h1 = nh1[b];
      const int vn = v + VB;
      if (vn < v1) {
        load_pos(kind0, col0, vn, ng0[b], nh0[b]);
        load_pos(kind1, col1, vn, ng1[b], nh1[b]);
      }
      T* Pg = sP + (b * 2 + 0) * G::NEXT;
      T* Ph = sP + (b * 2 + 1) * G::NEXT;
      T gs, hs;
      if (!ML || kind0 == 1) {
        model_eval<T, D>(m0, xixb[b], xiyb[b], c0, twoK, gs, hs);
        dg0[b] = N::sub(gs, g0[b]);
        dh0[b] = N::sub(hs, h0[b]);
        Pg[e0] = N::fma(m0.c1, dg0[b], g0[b]);
        Ph[e0] = N::fma(m0.c1, dh0[b], h0[b]);
      } else {
        dg0[b] = T(0);
        dh0[b] = T(0);
        Pg[e0] = g0[b];
        Ph[e0] = h0[b];
      }
      if (tid < G::NHALO) {
        if (!ML || kind1 == 1) {
          model_eval<T, D>(m1, xixb[b], xiyb[b], c0, twoK, gs, hs);
          Pg[e1] = N::fma(m1.c1, N::sub(gs, g1), g1);
          Ph[e1] = N::fma(m1.c1, N::sub(hs, h1), h1);
        } else {
          Pg[e1] = g1;
          Ph[e1] = h1;
        }
      }
    }
    __syncthreads();
    // ---- phase 2: limited slopes
    for (int q = tid; q < G::NSL; q += G::NT) {
      const int sx = q % G::SW - 1, sy = (D == 2) ? q / G::SW - 1 : 0;
      const int e = G::eidx(sx, sy);
#pragma unroll
      for (int b = 0; b < VB; ++b) {
        const T* Pg = sP + (b * 2 + 0) * G::NEXT;
        const T* Ph = sP + (b * 2 + 1) * G::NEXT;
        T* Sb = sS + b * 4 * G::NSL;
        if constexpr (CV) {
          // index-direction slopes (unit spacing) -> physical slopes: sigma = J^{-T} (d_i, d_j)
          const T one = T(1);
          const T gi = limited(N::sub(Pg[e + 1], Pg[e]), N::sub(Pg[e], Pg[e - 1]), one, limiter);
          const T hi = limited(N::sub(Ph[e + 1], Ph[e]), N::sub(Ph[e], Ph[e - 1]), one, limiter);
          const T gj = limited(N::sub(Pg[e + G::EW], Pg[e]), N::sub(Pg[e], Pg[e - G::EW]), one, limiter);
          const T hj = limited(N::sub(Ph[e + G::EW], Ph[e]), N::sub(Ph[e], Ph[e - G::EW]), one, limiter);
          const T j00 = sJt[q], j01 = sJt[G::NSL + q], j10 = sJt[2 * G::NSL + q], j11 = sJt[3 * G::NSL + q];
          Sb[q] = N::fma(j01, gj, N::mul(j00, gi));
          Sb[G::NSL + q] = N::fma(j01, hj, N::mul(j00, hi));
          Sb[2 * G::NSL + q] = N::fma(j11, gj, N::mul(j10, gi));
          Sb[3 * G::NSL + q] = N::fma(j11, hj, N::mul(j10, hi));
          continue;
        }
        Sb[q] = limited(N::sub(Pg[e + 1], Pg[e]), N::sub(Pg[e], Pg[e - 1]), idx_, limiter);
        Sb[G::NSL + q] = limited(N::sub(Ph[e + 1], Ph[e]), N::sub(Ph[e], Ph[e - 1]), idx_, limiter);
        if (D == 2) {
          Sb[2 * G::NSL + q] = limited(N::sub(Pg[e + G::EW], Pg[e]), N::sub(Pg[e], Pg[e - G::EW]), idy_, limiter);
          Sb[3 * G::NSL + q] = limited(N::sub(Ph[e + G::EW], Ph[e]), N::sub(Ph[e], Ph[e - G::EW]), idy_, limiter);
        }
      }
    }
    __syncthreads();
    // ---- phase 3: faces
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int f = tid + q * G::NT;
      if (f >= G::NF) break;
      const int meta = sMeta[f];
      if (!(meta & FM_VALID)) continue;
      const int role = meta >> 5;
      if (MODE == 0 && (!(meta & FM_OWNED) || (ML && role == FR_RECV))) continue;
      const int kind = (meta >> 2) & 7;
      int dir, li, lj;
      G::face_pos(f, dir, li, lj);
      if (ML && MODE == 1 && role == FR_RECV) {
        // microflux mapped from the face's own space (Eq. native_flux_moment_matching)
        const int col = sMeta[G::NF + f];
#pragma unroll
        for (int b = 0; b < VB; ++b) {
          const int v = vb0 + b;
          if (v >= v1) break;
          sF[(b * 2 + 0) * G::NF + f] = Yi[(long)v * a.nY + col];
          sF[(b * 2 + 1) * G::NF + f] = Yi[(nv + v) * a.nY + col];
        }
        continue;
      }
      MP<T> fm;
      if (MODE == 1) {
        fm.load(sFP, G::NF, f);
      }
      T part[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) part[p] = T(0);
      T fsx = T(0), fsy = T(0);
      if (MODE == 0) {
        if (q < 2) { fsx = fshx[q < 2 ? q : 0]; fsy = fshy[q < 2 ? q : 0]; }
        else { fsx = sAcc[13 * G::NF + f]; fsy = sAcc[14 * G::NF + f]; }
      }
#pragma unroll
      for (int b = 0; b < VB; ++b) {
        const int v = vb0 + b;
        if (v >= v1) break;
        const T* Pg = sP + (b * 2 + 0) * G::NEXT;
        const T* Ph = sP + (b * 2 + 1) * G::NEXT;
        const T* Sb = sS + b * 4 * G::NSL;
        const T xix = xixb[b], xiy = xiyb[b];
        const T bx_ = N::mul(-xix, s), by_ = N::mul(-xiy, s);
        T gb, hb, xn;
        // upwind side only (the mean of both sides when xi.n = 0)
        if constexpr (CV) {
          // xi.n as two rounded products and a rounded sum: its sign picks the upwind side,
          // and a velocity tangential to the face gives the same rounded value wherever
          // this is evaluated
          xn = N::add(N::mul(xix, sFG[f]), N::mul(xiy, sFG[G::NF + f]));
          auto rec = [&](int cx, int cy, T ox, T oy, T& gg, T& hh) {
            const int e = G::eidx(cx, cy), si = G::sidx(cx, cy);
            gg = N::fma(N::add(oy, by_), Sb[2 * G::NSL + si], N::fma(N::add(ox, bx_), Sb[si], Pg[e]));
            hh = N::fma(N::add(oy, by_), Sb[3 * G::NSL + si], N::fma(N::add(ox, bx_), Sb[G::NSL + si], Ph[e]));
          };
          const int lx = dir == 0 ? li - 1 : li, ly = dir == 0 ? lj : lj - 1;
          const T dLx = sFG[3 * G::NF + f], dLy = sFG[4 * G::NF + f];
          const T dRx = sFG[5 * G::NF + f], dRy = sFG[6 * G::NF + f];
          if (xn > T(0)) rec(lx, ly, dLx, dLy, gb, hb);
          else if (xn < T(0)) rec(li, lj, dRx, dRy, gb, hb);
          else {
            T g2, h2;
            rec(lx, ly, dLx, dLy, gb, hb);
            rec(li, lj, dRx, dRy, g2, h2);
            gb = N::mul(T(0.5), N::add(gb, g2));
            hb = N::mul(T(0.5), N::add(hb, h2));
          }
        } else if (dir == 0) {
          xn = xix;
          auto rec = [&](int cx, T off, T& gg, T& hh) {
            const int e = G::eidx(cx, lj), si = G::sidx(cx, lj);
            gg = N::fma(N::add(off, bx_), Sb[si], Pg[e]);
            hh = N::fma(N::add(off, bx_), Sb[G::NSL + si], Ph[e]);
            if (D == 2) {
              gg = N::fma(by_, Sb[2 * G::NSL + si], gg);
              hh = N::fma(by_, Sb[3 * G::NSL + si], hh);
            }
          };
          if (xix > T(0)) rec(li - 1, hdx, gb, hb);
          else if (xix < T(0)) rec(li, -hdx, gb, hb);
          else {
            T g2, h2;
            rec(li - 1, hdx, gb, hb);
            rec(li, -hdx, g2, h2);
            gb = N::mul(T(0.5), N::add(gb, g2));
            hb = N::mul(T(0.5), N::add(hb, h2));
          }
        } else {
          xn = xiy;
          auto rec = [&](int cy, T off, T& gg, T& hh) {
            const int e = G::eidx(li, cy), si = G::sidx(li, cy);
            gg = N::fma(N::add(off, by_), Sb[2 * G::NSL + si], N::fma(bx_, Sb[si], Pg[e]));
            hh = N::fma(N::add(off, by_), Sb[3 * G::NSL + si], N::fma(bx_, Sb[G::NSL + si], Ph[e]));
          };
          if (xiy > T(0)) rec(lj - 1, hdy, gb, hb);
          else if (xiy < T(0)) rec(lj, -hdy, gb, hb);
          else {
            T g2, h2;
            rec(lj - 1, hdy, gb, hb);
            rec(lj, -hdy, g2, h2);
            gb = N::mul(T(0.5), N::add(gb, g2));
            hb = N::mul(T(0.5), N::add(hb, h2));
          }
        }
        if (MODE == 0) {
          const T wxv = wxb[b], wyv = wyb[b];
          if (kind == FK_INTERIOR) {
            const T xp = xix - fsx, yp = (D == 2) ? xiy - fsy : T(0);
            const T wg = wxv * (wyv * gb);
            const T e = wxv * (wyv * ((xp * xp + yp * yp) * gb + hb));
            part[0] += wg;
            part[1] += wg * xp;
            part[2] += wg * yp;
            part[3] += e;
            part[4] += wg * xp * xp;
            part[5] += wg * xp * yp;
            part[6] += wg * yp * yp;
            part[7] += e * xp;
            part[8] += e * yp;
          } else if (kind == FK_WALL_LO || kind == FK_WALL_HI) {
            // wall: outgoing normal mass flux sum_{xi.n_in <= 0} w (xi.n_in) g-bar
            const T xin = (kind == FK_WALL_LO) ? xn : -xn;
            if (xin <= T(0)) part[0] += wxv * (wyv * (xin * gb));
          }
        } else {
          T gf, hf;
          if (kind == FK_INTERIOR) {
            T gs, hs;
            model_eval<T, D>(fm, xix, xiy, c0, twoK, gs, hs);
            // Eq. recover_phi with weights summing to one; explicitly rounded so the two tiles
            // that evaluate a shared face produce the same bits (exact flux telescoping)
            gf = N::fma(fm.c2, N::sub(gs, gb), gb);
            hf = N::fma(fm.c2, N::sub(hs, hb), hb);
          } else {
            // boundary: the model enters (wall: rho_w = c1 + c2 times the unit-density wall
            // Maxwellian; freestream: c1 = 1, c2 = 0 and the corrected freestream Maxwellian),
            // the reconstruction leaves
            const T xin = fk_low(kind) ? xn : -xn;
            if (xin > T(0)) {
              T gs, hs;
              model_eval<T, D>(fm, xix, xiy, c0, twoK, gs, hs);
              gf = N::fma(fm.c1, gs, N::mul(fm.c2, gs));
              hf = N::fma(fm.c1, hs, N::mul(fm.c2, hs));
            } else {
              gf = gb;
              hf = hb;
            }
          }
          // microflux (xi.n) phi on this space (Eq. interface_reduced_fluxes), times |S| on
          // curvilinear meshes
          T xs = xn;
          if constexpr (CV) xs = N::mul(xn, sFG[2 * G::NF + f]);
          const T Fg = N::mul(xs, gf), Fh = N::mul(xs, hf);
          sF[(b * 2 + 0) * G::NF + f] = Fg;
          sF[(b * 2 + 1) * G::NF + f] = Fh;
          if (ML && role == FR_CROSS && (meta & FM_OWNED)) {
            const int col = sMeta[G::NF + f];
            Xo[(long)v * a.nX + col] = Fg;
            Xo[(nv + v) * a.nX + col] = Fh;
          }
        }
      }
      if (MODE == 0) {
        // fold the round's partial sums into the chunk accumulators (compensated for M0..E)
        if (q < 2) fold_partials<T>(ra[q < 2 ? q : 0], part);
        else fold_partials_smem<T>(sAcc + f, G::NF, part);
      }
    }
    __syncthreads();
    if (MODE == 1) {
      // ---- phase 4: update of the tile's cells of this level (Eq. explicit_update)
      if (own_active) {
        const int wI = (D == 2) ? ty * (TX + 1) + tx : tx;
        const int sI = G::NFXL + ty * TX + tx;
#pragma unroll
        for (int b = 0; b < VB; ++b) {
          const int v = vb0 + b;
          if (v >= v1) break;
          const T* Fg = sF + (b * 2 + 0) * G::NF;
          const T* Fh = sF + (b * 2 + 1) * G::NF;
          const T xix = xixb[b], xiy = xiyb[b];
          // phi~+ = phi~ + (4/3) b (phi^S - phi~), then the microflux divergence
          T gn = g0[b] + m0.c2 * dg0[b] - lamx * (Fg[wI + 1] - Fg[wI]);
          T hn = h0[b] + m0.c2 * dh0[b] - lamx * (Fh[wI + 1] - Fh[wI]);
          if (D == 2) {
            gn -= lamy * (Fg[sI + TX] - Fg[sI]);
            hn -= lamy * (Fh[sI + TX] - Fh[sI]);
          }
          unsigned rb = 0;
          if constexpr (sizeof(S) == 2) rb = hash32(seed ^ hash32((unsigned)col0 * 0x9e3779b1u + (unsigned)v));
          const S sg = Stored<S, T>::enc(gn, rb), sh = Stored<S, T>::enc(hn, rb >> 16);
          fout[(long)v * ns + col0] = sg;
          fout[(nv + v) * ns + col0] = sh;
          const T gq = Stored<S, T>::dec(sg), hq = Stored<S, T>::dec(sh);
          const T wxv = wxb[b], wyv = wyb[b];
          const T xp = xix - m0.ux, yp = (D == 2) ? xiy - m0.uy : T(0);
          const T wg = wxv * (wyv * gq);
          const T e = wxv * (wyv * ((xp * xp + yp * yp) * gq + hq));
          c0k.add(wg);
          cxk.add(wg * xp);
          cek.add(e);
          cgxx += wg * xp * xp;
          cjx += e * xp;
          if (D == 2) {
            cyk.add(wg * yp);
            cgxy += wg * xp * yp;
            cgyy += wg * yp * yp;
            cjy += e * yp;
          }
        }
      }
    }
  }

  // ---- write the chunk's partial moments
  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int f = tid + q * G::NT;
      if (f >= G::NF) break;
      const int meta = sMeta[f];
      const int role = meta >> 5;
      if (!(meta & FM_VALID) || !(meta & FM_OWNED) || role == FR_RECV) continue;
      const int fid = sMeta[G::NF + f];
      double* P = a.part + (long)chunk * NMOM * k.nface + fid;
      if (q < 2) write_partials<T, D>(ra[q < 2 ? q : 0], P, k.nface);
      else write_partials_smem<T, D>(sAcc + f, G::NF, P, k.nface);
    }
  } else if (own_active) {
    double* P = a.part + (long)chunk * NMOM * ns + col0;
    P[MO_0 * ns] = c0k.val();
    P[MO_X * ns] = cxk.val();
    P[MO_Y * ns] = (D == 2) ? cyk.val() : 0.0;
    P[MO_E * ns] = cek.val();
    P[MO_GXX * ns] = (double)cgxx;
    P[MO_GXY * ns] = (double)cgxy;
    P[MO_GYY * ns] = (double)cgyy;
    P[MO_JX * ns] = (double)cjx;
    P[MO_JY * ns] = (double)cjy;
  }
}

}  // namespace mlvs
