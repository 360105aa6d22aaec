// Tile kernels of one DUGKS step on a structured Cartesian mesh (Sec. 2.2).
//
// k_faces: a CTA owns a TX x TY tile of cells and a contiguous chunk of velocities, processed
// VB velocities per barrier round.  Per round it stages in shared memory
//   phase 1  phi-bar-plus of the tile and its two-cell halo (the derived conversion
//            phi-bar-plus = phi~ + b (phi^S - phi~) of Sec. 2.2);
//   phase 2  limited slopes (Eq. reconstruction) of the cells that can be upwind of a face;
//   phase 3  the face phi-bar of the upwind side by the characteristic
//            (Eq. bar_phi_transport) for the faces the tile owns: stored to the face buffer
//            and accumulated into the face moments over the chunk (input of Eq. W_from_bar).
// k_update: the same tiles and chunks, no halo.  Per round each thread evaluates the face
// phi (Eq. recover_phi) of its cell's low-side faces (and the tile's high-side boundary faces)
// from the stored face phi-bar and the face model, the microflux (xi.n) phi, and after a
// barrier Eq. explicit_update of its cell, the store of phi~^{n+1} and the cell moments of
// the stored values (input of Eq. discrete_W / discrete_q).
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
  const int* xfid;       // [nX] face id of every column of X
  const void* cparam8;   // eight-moment correction (C8): (T) [4][nslot] b4..b7 of the cells
  const void* fparam8;   //                                (T) [4][nface] b4..b7 of the faces
  const void* Y;         // (T) [2][nv][nY] microfluxes mapped here from other face spaces
  int nY;
  void* fbar;            // (T) [2][nv][nface] face phi-bar of the faces this level evaluates
                         // (k_faces writes the faces its tile owns, k_update reads them)
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

// The box of cells k_faces stages per round: the tile and a halo of two cells on the low
// sides and one on the high sides, x in [-2, TX], y in [-2, TY].  That covers every upwind
// cell of the faces the tile owns (low-side faces li in [0, TX), lj in [0, TY), and the last
// face of a non-periodic axis when it falls on the tile's edge) with the neighbours of its
// slopes.  A slope at the high edge of the box belongs to a ghost cell beyond a non-periodic
// mesh end, whose neighbour beyond is the same ghost copy.
template <int TX, int TY, int D> struct FaceBox {
  static constexpr int NT = TX * TY;
  static constexpr int BW = TX + 3;
  static constexpr int BH = (D == 2) ? TY + 3 : 1;
  static constexpr int NB = BW * BH;
  static constexpr int NH = NB - NT;     // halo cells
  static constexpr int SW = TX + 2;      // curvilinear J^{-T} rectangle, x in [-1, TX], y in [-1, TY]
  static constexpr int SH = (D == 2) ? TY + 2 : 1;
  static constexpr int NSL = SW * SH;
  static __device__ __forceinline__ int bidx(int x, int y) { return (D == 2) ? (y + 2) * BW + (x + 2) : (x + 2); }
  static __device__ __forceinline__ int sidx(int x, int y) { return (D == 2) ? (y + 1) * SW + (x + 1) : (x + 1); }
  // k-th halo cell: the two rows below the tile, the row above it, then per tile row the two
  // cells on the left and the one on the right
  static __device__ __forceinline__ void halo_pos(int k, int& x, int& y) {
    if (D == 1) {
      x = (k < 2) ? k - 2 : TX;
      y = 0;
      return;
    }
    if (k < 2 * BW) { y = k / BW - 2; x = k % BW - 2; return; }
    k -= 2 * BW;
    if (k < BW) { y = TY; x = k - 2; return; }
    k -= BW;
    y = k / 3;
    const int c = k % 3;
    x = (c < 2) ? c - 2 : TX;
  }
};

// Shared-memory layout of k_faces (bytes), identical on host and device: the chunk's velocity
// table by pairs; phi-bar-plus of the box by pairs, double-buffered (one barrier per round);
// the accumulators of the high-edge faces (warp 0, mesh-end tiles); on curvilinear meshes
// J^{-T} of the possible upwind cells and the geometry of the tile's faces.
constexpr int kVpcMax = 384;   // largest velocity chunk of a tile launch (even)

template <class T, int TX, int TY, int D, bool CV = false> struct TileSmem {
  using B = FaceBox<TX, TY, D>;
  using G = TileGeom<TX, TY, D>;
  using V = V2<T>;
  static constexpr int NX3 = (D == 2) ? TX + TY : 1;
  static constexpr size_t VT = 0;                                          // V [kVpcMax/2][4]
  static constexpr size_t P = VT + sizeof(V) * 4 * (kVpcMax / 2);           // V [2][2][NB]
  static constexpr size_t ACC = P + sizeof(V) * 2 * 2 * B::NB;              // T [13][NX3]
  static constexpr size_t JT = ACC + sizeof(T) * 13 * NX3;                  // T [4][NSL] (CV)
  static constexpr size_t FG = JT + (CV ? sizeof(T) * 4 * B::NSL : 0);      // T [7][NF]  (CV)
  static constexpr size_t BYTES = FG + (CV ? sizeof(T) * 7 * G::NF : 0);
};

// Shared-memory layout of k_update (bytes): the microfluxes of the faces A and B of a round
// by pairs, double-buffered so one barrier per round suffices; the microfluxes of the tile's
// high-side faces C over a sub-chunk of SC pairs, double-buffered; the chunk's velocity table
// by pairs (padded to whole sub-chunks); the parameters and ids of the faces C.
template <class T, int TX, int TY, int D, int VPC> struct UpdSmem {
  using G = TileGeom<TX, TY, D>;
  using V = V2<T>;
  static constexpr int NX3 = (D == 2) ? TX + TY : 1;                        // high-side faces
  static constexpr int SC = 16;                                            // pairs per sub-chunk
  static constexpr int NPT = ((VPC / 2) + SC - 1) / SC * SC;               // padded pairs
  static constexpr size_t F = 0;                                           // V [2][2][NF]
  static constexpr size_t C = F + sizeof(V) * 2 * 2 * G::NF;               // V [2][2][SC][NX3]
  static constexpr size_t VT = C + sizeof(V) * 2 * 2 * SC * NX3;           // V [NPT][4]
  static constexpr size_t XP = VT + sizeof(V) * 4 * NPT;                   // T [20][NX3]
  static constexpr size_t XI = XP + sizeof(T) * 20 * NX3;                  // long [4][NX3]
  static constexpr size_t BYTES = (XI + sizeof(long) * 4 * NX3 + 15) / 16 * 16;
};

__device__ __forceinline__ int wrap_or_clamp(int g, int n, int periodic) {
  if (periodic) { g %= n; return g < 0 ? g + n : g; }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// van Leer limited slope (reading of Eq. reconstruction): 2ab/(a+b)/h for a, b of equal
// strict sign (ab > 0; an underflowing product counts as 0), else 0.  limiter == 1: central
// difference (a+b)/(2h).  Both are formed and one is selected (no branch); a quotient of a
// pair that is not selected may be infinite or NaN.
template <class T>
__device__ __forceinline__ T limited(T a, T b, T inv_h, int limiter) {
  using N = Num<T>;
  const T ab = N::mul(a, b);
  const T sum = N::add(a, b);
  const T vl = N::mul(N::dv(N::mul(T(2), ab), sum), inv_h);
  const T ce = N::mul(N::mul(T(0.5), sum), inv_h);
  return limiter ? ce : ((ab > T(0)) ? vl : T(0));
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

// Metadata of tile-local face f of the tile at (x0, y0): returns the meta word (bit 0 valid,
// bit 1 owned by this tile, bits 2-4 boundary kind, role above) and the global face id (-1 if
// the face is outside the mesh).  A face is owned by the tile on its high side (its li < TX),
// the last face of a non-periodic axis by the last tile.
template <int TX, int TY, int D, bool ML>
__device__ __forceinline__ int face_meta(const TileArgs& a, int x0, int y0, int f, int& fid) {
  using G = TileGeom<TX, TY, D>;
  const StepConst& k = a.k;
  int dir, li, lj;
  G::face_pos(f, dir, li, lj);
  const int gi = x0 + li, gj = y0 + lj;
  int meta = 0, role = FR_NONE;
  fid = -1;
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
  return meta | (role << 5);
}

// ---------------------------------------------------------------------------------------
// Velocity pairs.  Both tile kernels process the velocities of their chunk two at a time,
// lanes (v, v+1) of one thread, with the packed two-lane arithmetic of Pk<T>; chunks start
// at even velocities, and a pair past the end of the velocity set has a padding lane (its
// loads repeat the last velocity, its weight is zero and nothing of it is stored).  The face
// buffer interleaves the pair: fbar[comp][v / 2][face][v % 2].
__device__ __forceinline__ long fbar_at(long comp, long v, long fid, long nvp, long nfc) {
  return ((comp * nvp + (v >> 1)) * nfc + fid) * 2 + (v & 1);
}

// van Leer limited slopes of a pair (limited() lane by lane, the quotient per lane).
template <class T>
__device__ __forceinline__ V2<T> limited2(V2<T> a, V2<T> b, T inv_h, int limiter) {
  using P = Pk<T>;
  using N = Num<T>;
  const V2<T> ab = P::mul(a, b);
  const V2<T> sum = P::add(a, b);
  const V2<T> n2 = P::mul(P::splat(T(2)), ab);
  const V2<T> vl = P::mul(P::mk(N::dv(n2.x, sum.x), N::dv(n2.y, sum.y)), P::splat(inv_h));
  const V2<T> ce = P::mul(P::mul(P::splat(T(0.5)), sum), P::splat(inv_h));
  V2<T> r;
  r.x = limiter ? ce.x : ((ab.x > T(0)) ? vl.x : T(0));
  r.y = limiter ? ce.y : ((ab.y > T(0)) ? vl.y : T(0));
  return r;
}

// ML = false: the level holds every cell of the mesh (one velocity space), so every stencil
// position is an own cell in natural order and every face is a normal face; the level
// tables are not read.
// CV: structured curvilinear mesh (2-D): slopes along the index directions turned into
// physical slopes with the cell's J^{-T}, faces with their own normals, areas and centroid
// offsets (precomputed per face, so the two tiles of a face read the same values).
//
// Copy a level's tile arguments into shared memory (all threads; a barrier must follow).
__device__ __forceinline__ void load_args(TileArgs& dst, const TileArgs* __restrict__ src) {
  static_assert(sizeof(TileArgs) % 8 == 0, "tile arguments are copied in 8-byte words");
  constexpr int NW = (int)(sizeof(TileArgs) / 8);
  for (int i = threadIdx.x; i < NW; i += blockDim.x)
    reinterpret_cast<unsigned long long*>(&dst)[i] = reinterpret_cast<const unsigned long long*>(src)[i];
}

// The tile passes run in two forms.  ML = false (a level that holds every cell): the level's
// arguments are the kernel parameter a_, CTA (tile list index, velocity chunk) = (blockIdx.x,
// blockIdx.y).  ML = true (every level of a multi-level instance in one launch): CTA b takes
// work item work[b] = (level, tile list index, velocity chunk, 0) and the level's arguments
// tab[level], copied to shared memory.

// Per round (one velocity pair): every thread stages phi-bar-plus of its own cell, and the
// first NH threads of one halo cell, into the box (one barrier; the box is double-buffered);
// then each thread reconstructs its cell's two low-side faces (A: x-face, B: y-face) from the
// upwind cell, whose two limited slopes it evaluates from the box, stores the face phi-bar to
// the face buffer and accumulates the face moments.  When the two lanes of a face have the
// same strict sign of xi.n (nearly every pair) the pair takes one upwind cell; otherwise each
// lane is reconstructed on its own.  Warp 0 of a tile whose high edge is a non-periodic mesh
// end does the same for the faces on that edge.
template <class S, class T, int D, int TX, int TY, bool ML, bool CV, bool C8 = false>
__global__ void __launch_bounds__(TX * TY, (TX * TY >= 256) ? 2 : 4)
k_faces(const TileArgs a_, const TileArgs* __restrict__ tab, const int4* __restrict__ work, int limiter) {
  __shared__ __align__(16) TileArgs sa;
  int tile, chunk;
  if constexpr (ML) {
    const int4 w = work[blockIdx.x];
    load_args(sa, tab + w.x);
    __syncthreads();
    tile = sa.tiles[w.y];
    chunk = w.z;
  } else {
    tile = a_.tiles[blockIdx.x];
    chunk = (int)blockIdx.y;
  }
  const TileArgs& a = ML ? sa : a_;
  using G = TileGeom<TX, TY, D>;
  using B = FaceBox<TX, TY, D>;
  using L = TileSmem<T, TX, TY, D, CV>;
  using V = V2<T>;
  using P = Pk<T>;
  using N = Num<T>;
  static_assert(!CV || D == 2, "curvilinear meshes are two-dimensional");
  static_assert(B::NH <= G::NT, "more halo cells than threads");
  static_assert(L::NX3 <= 32, "high-edge faces beyond warp 0");
  extern __shared__ __align__(16) unsigned char smem[];
  V* sVT = reinterpret_cast<V*>(smem + L::VT);
  V* sP = reinterpret_cast<V*>(smem + L::P);
  T* sAcc = reinterpret_cast<T*>(smem + L::ACC);
  T* sJt = reinterpret_cast<T*>(smem + L::JT);
  T* sFG = reinterpret_cast<T*>(smem + L::FG);
  const T* __restrict__ cg = reinterpret_cast<const T*>(a.cgeo);
  const T* __restrict__ fg = reinterpret_cast<const T*>(a.fgeo);

  const StepConst& k = a.k;
  const S* __restrict__ fin = reinterpret_cast<const S*>(a.f_in);
  const T* __restrict__ cp = reinterpret_cast<const T*>(a.cparam);
  const T* __restrict__ vt = reinterpret_cast<const T*>(a.vt);
  const T* __restrict__ gst = reinterpret_cast<const T*>(a.ghost);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.ucell);
  T* __restrict__ fbo = reinterpret_cast<T*>(a.fbar);
  const long ns = a.nslot;
  const long ng = a.nghost;
  const long nv = k.nv;
  const long nvp = (k.nv + 1) / 2;
  const long nfc = k.nface;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = (D == 2) ? tid / TX : 0;
  const int bx = tile % a.ntx, by = tile / a.ntx;
  const int x0 = bx * TX, y0 = by * TY;
  const int v0 = chunk * k.vpc;               // even: k.vpc is even
  const int v1 = min(k.nv, v0 + k.vpc);
  const int npr = (v1 - v0 + 1) / 2;          // pairs of the chunk

  // the chunk's velocity table by pairs: (xi_x, xi_y, w_x, w_y), a padding lane with zeros
  for (int j = tid; j < npr; j += G::NT) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int v = v0 + 2 * j;
      const T e0 = (r == 1 && D == 1) ? T(0) : vt[r * nv + v];
      const T e1 = (v + 1 < v1 && !(r == 1 && D == 1)) ? vt[r * nv + v + 1] : T(0);
      sVT[4 * j + r] = P::mk(e0, e1);
    }
  }

  // ---- box positions: the own cell, and one halo cell for the first NH threads.  A position
  // holds a cell of this level (phi~ + parameters -> phi-bar-plus), a ghost (phi-bar-plus
  // mapped to this space), or nothing (never read by a face evaluated here).  Loads: a base
  // pointer and a velocity stride (0: a dummy element).
  auto classify = [&](int ex, int ey, int& kind, long& col) {
    const int c = wrap_or_clamp(y0 + ey, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + ex, k.nx, k.px);
    kind = 0; col = 0;
    if (!ML) { kind = 1; col = c; }
    else if (a.lvl_of[c] == a.level) { kind = 1; col = a.slot_of[c]; }
    else if (a.ghost_of && a.ghost_of[c] >= 0) { kind = 2; col = a.ghost_of[c]; }
  };
  int kind0, kind1 = 0;
  long col0, col1 = 0;
  classify(tx, ty, kind0, col0);
  const bool halo = tid < B::NH;
  int e1 = 0;
  if (halo) {
    int ex1, ey1;
    B::halo_pos(tid, ex1, ey1);
    classify(ex1, ey1, kind1, col1);
    e1 = B::bidx(ex1, ey1);
  }
  MP<T> m0, m1;
  m0.zero();
  m1.zero();
  if (kind0 == 1) m0.load(cp, ns, col0);
  if (kind1 == 1) m1.load(cp, ns, col1);
  // b4..b7 of the eight-moment correction (C8)
  T b80[4] = {T(0), T(0), T(0), T(0)}, b81[4] = {T(0), T(0), T(0), T(0)};
  if constexpr (C8) {
    const T* __restrict__ cp8 = reinterpret_cast<const T*>(a.cparam8);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (kind0 == 1) b80[m] = cp8[m * ns + col0];
      if (kind1 == 1) b81[m] = cp8[m * ns + col1];
    }
  }
  const int e0 = B::bidx(tx, ty);
  const void* p0 = fin;
  long st0 = 0;
  if (kind0 == 1) { p0 = fin + col0; st0 = ns; }
  else if (ML && kind0 == 2) { p0 = gst + col0; st0 = ng; }
  const void* p1 = fin;
  long st1 = 0;
  if (kind1 == 1) { p1 = fin + col1; st1 = ns; }
  else if (ML && kind1 == 2) { p1 = gst + col1; st1 = ng; }
  // the pair of lanes at velocities (v, v+1) of a position: g at p[v st], h at p[(nv + v) st]
  auto ld2 = [&](int kind, const void* p, long st, int v, V& g, V& h) {
    const long va = v, vb = min(v + 1, v1 - 1);
    if (!ML || kind != 2) {
      const S* q = reinterpret_cast<const S*>(p);
      g = P::mk(ldf<S, T>(q + va * st), ldf<S, T>(q + vb * st));
      h = P::mk(ldf<S, T>(q + (nv + va) * st), ldf<S, T>(q + (nv + vb) * st));
    } else {
      const T* q = reinterpret_cast<const T*>(p);
      g = P::mk(q[va * st], q[vb * st]);
      h = P::mk(q[(nv + va) * st], q[(nv + vb) * st]);
    }
  };

  // ---- faces: A (x-face li = tx, lj = ty), B (2-D: y-face li = tx, lj = ty), C (warp 0 of a
  // tile whose high edge is a non-periodic mesh end: the faces on that edge)
  struct FaceQ {
    int meta, kind, dir, li, lj, f;
    long fid;
    T shx, shy;
  };
  auto setup = [&](int f, FaceQ& F) {
    int fid;
    F.f = f;
    G::face_pos(f, F.dir, F.li, F.lj);
    F.meta = face_meta<TX, TY, D, ML>(a, x0, y0, f, fid);
    F.fid = fid;
    F.kind = (F.meta >> 2) & 7;
    const int role = F.meta >> 5;
    // evaluated here: owned, and a normal or cross face of this level
    if (!(F.meta & FM_VALID) || !(F.meta & FM_OWNED) || (ML && role == FR_RECV)) F.meta = 0;
    F.shx = F.shy = T(0);
    if (F.meta) {
      const int xl = (F.dir == 0) ? F.li - 1 : F.li, yl = (F.dir == 0) ? F.lj : F.lj - 1;
      const int sL = wrap_or_clamp(y0 + yl, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + xl, k.nx, k.px);
      const int sR = wrap_or_clamp(y0 + F.lj, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + F.li, k.nx, k.px);
      F.shx = T(0.5) * (uc[sL] + uc[sR]);
      if (D == 2) F.shy = T(0.5) * (uc[k.ncell + sL] + uc[k.ncell + sR]);
    }
  };
  FaceQ FA, FB;
  setup(ty * (TX + 1) + tx, FA);
  if (D == 2) setup(G::NFXL + ty * TX + tx, FB);
  else FB.meta = 0;
  const bool edgeC = (!k.px && x0 + TX == k.nx) || (D == 2 && !k.py && y0 + TY == k.ny);
  FaceQ FC;
  FC.meta = 0;
  if (edgeC && tid < L::NX3) {
    const int fC = (D == 1) ? TX : (tid < TY ? tid * (TX + 1) + TX : G::NFXL + TY * TX + (tid - TY));
    setup(fC, FC);
#pragma unroll
    for (int p = 0; p < 13; ++p) sAcc[p * L::NX3 + tid] = T(0);
  }
  if constexpr (CV) {
    for (int f = tid; f < G::NF; f += G::NT) {
      int fid;
      face_meta<TX, TY, D, ML>(a, x0, y0, f, fid);
#pragma unroll
      for (int p = 0; p < 7; ++p) sFG[p * G::NF + f] = fid >= 0 ? fg[(long)p * k.nface + fid] : T(0);
    }
    // J^{-T} of the possible upwind cells (ghost positions take the boundary cell's)
    for (int q = tid; q < B::NSL; q += G::NT) {
      const int sx = q % B::SW - 1, sy = q / B::SW - 1;
      const int c = wrap_or_clamp(y0 + sy, k.ny, k.py) * k.nx + wrap_or_clamp(x0 + sx, k.nx, k.px);
#pragma unroll
      for (int p = 0; p < 4; ++p) sJt[p * B::NSL + q] = cg[(long)p * k.ncell + c];
    }
  }
  // accumulators of faces A and B: Kahan (s, c) for M0, MX, MY, E, plain for Gxx, Gxy, Gyy, Jx, Jy
  T ra[2][13];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int p = 0; p < 13; ++p) ra[q][p] = T(0);

  const T c0 = T(k.c0), twoK = T(k.twoK);
  const T s = T(0.5 * k.dt);
  const T hdx = T(0.5 * k.dx), hdy = T(0.5 * k.dy);
  const T idx_ = T(1.0 / k.dx), idy_ = T(1.0 / k.dy);

  // limited slopes of box cell (cx, cy) along x and y (index directions on curvilinear
  // meshes): lane by lane from one plane of the box
  auto slopes = [&](const V* Pl, int cx, int cy, T hx, T hy, V& sx, V& sy) {
    const int e = B::bidx(cx, cy);
    const V pc = Pl[e];
    const V pxp = Pl[(cx < TX) ? e + 1 : e];
    sx = limited2<T>(P::sub(pxp, pc), P::sub(pc, Pl[e - 1]), hx, limiter);
    sy = P::splat(T(0));
    if (D == 2) {
      const V pyp = Pl[(cy < TY) ? e + B::BW : e];
      sy = limited2<T>(P::sub(pyp, pc), P::sub(pc, Pl[e - B::BW]), hy, limiter);
    }
  };
  // phi-bar of face F (Eq. bar_phi_transport with Eq. reconstruction), both lanes from one
  // upwind cell; (ox, oy) is x_b - x_up
  auto rec2 = [&](const FaceQ& F, const V* Pg, const V* Ph, int cx, int cy, V ox, V oy, V bx_, V by_, V& gb,
                  V& hb) {
    const int e = B::bidx(cx, cy);
    V gx, gy, hx, hy;
    if constexpr (CV) {
      V gi, gj, hi, hj;
      slopes(Pg, cx, cy, T(1), T(1), gi, gj);
      slopes(Ph, cx, cy, T(1), T(1), hi, hj);
      const int si = B::sidx(cx, cy);
      const V j00 = P::splat(sJt[si]), j01 = P::splat(sJt[B::NSL + si]);
      const V j10 = P::splat(sJt[2 * B::NSL + si]), j11 = P::splat(sJt[3 * B::NSL + si]);
      gx = P::fma(j01, gj, P::mul(j00, gi));
      hx = P::fma(j01, hj, P::mul(j00, hi));
      gy = P::fma(j11, gj, P::mul(j10, gi));
      hy = P::fma(j11, hj, P::mul(j10, hi));
      gb = P::fma(P::add(oy, by_), gy, P::fma(P::add(ox, bx_), gx, Pg[e]));
      hb = P::fma(P::add(oy, by_), hy, P::fma(P::add(ox, bx_), hx, Ph[e]));
      return;
    }
    slopes(Pg, cx, cy, idx_, idy_, gx, gy);
    slopes(Ph, cx, cy, idx_, idy_, hx, hy);
    (void)F;
    if (F.dir == 0) {
      gb = P::fma(P::add(ox, bx_), gx, Pg[e]);
      hb = P::fma(P::add(ox, bx_), hx, Ph[e]);
      if (D == 2) {
        gb = P::fma(by_, gy, gb);
        hb = P::fma(by_, hy, hb);
      }
    } else {
      gb = P::fma(P::add(oy, by_), gy, P::fma(bx_, gx, Pg[e]));
      hb = P::fma(P::add(oy, by_), hy, P::fma(bx_, hx, Ph[e]));
    }
  };
  // xi.n of face F for a pair, and the face phi-bar
  auto face_bar = [&](const FaceQ& F, const V* Pg, const V* Ph, V xix, V xiy, V& gb, V& hb, V& xn) {
    const V bx_ = P::mul(P::mk(-xix.x, -xix.y), P::splat(s)), by_ = P::mul(P::mk(-xiy.x, -xiy.y), P::splat(s));
    const int lx = F.dir == 0 ? F.li - 1 : F.li, ly = F.dir == 0 ? F.lj : F.lj - 1;
    V oLx, oLy, oRx, oRy;
    if constexpr (CV) {
      // xi.n as two rounded products and a rounded sum: its sign picks the upwind side, and a
      // velocity tangential to the face gives the same rounded value wherever this is evaluated
      xn = P::add(P::mul(xix, P::splat(sFG[F.f])), P::mul(xiy, P::splat(sFG[G::NF + F.f])));
      oLx = P::splat(sFG[3 * G::NF + F.f]); oLy = P::splat(sFG[4 * G::NF + F.f]);
      oRx = P::splat(sFG[5 * G::NF + F.f]); oRy = P::splat(sFG[6 * G::NF + F.f]);
    } else if (F.dir == 0) {
      xn = xix;
      oLx = P::splat(hdx); oRx = P::splat(-hdx); oLy = oRy = P::splat(T(0));
    } else {
      xn = xiy;
      oLy = P::splat(hdy); oRy = P::splat(-hdy); oLx = oRx = P::splat(T(0));
    }
    if ((xn.x > T(0) && xn.y > T(0)) || (xn.x < T(0) && xn.y < T(0))) {
      // one upwind cell for both lanes
      if (xn.x > T(0)) rec2(F, Pg, Ph, lx, ly, oLx, oLy, bx_, by_, gb, hb);
      else rec2(F, Pg, Ph, F.li, F.lj, oRx, oRy, bx_, by_, gb, hb);
    } else {
      // lane by lane: the upwind side of each lane, the mean of both sides where xi.n = 0
      V gL, hL, gR, hR;
      rec2(F, Pg, Ph, lx, ly, oLx, oLy, bx_, by_, gL, hL);
      rec2(F, Pg, Ph, F.li, F.lj, oRx, oRy, bx_, by_, gR, hR);
      const V gm = P::mul(P::splat(T(0.5)), P::add(gL, gR)), hm = P::mul(P::splat(T(0.5)), P::add(hL, hR));
      gb.x = xn.x > T(0) ? gL.x : (xn.x < T(0) ? gR.x : gm.x);
      gb.y = xn.y > T(0) ? gL.y : (xn.y < T(0) ? gR.y : gm.y);
      hb.x = xn.x > T(0) ? hL.x : (xn.x < T(0) ? hR.x : hm.x);
      hb.y = xn.y > T(0) ? hL.y : (xn.y < T(0) ? hR.y : hm.y);
    }
  };
  // the face's contribution of a pair to its moment partials (interior faces), or to the
  // outgoing normal mass flux sum_{xi.n_in <= 0} w (xi.n_in) g-bar (wall faces): lanes
  // summed in order, as scalar accumulation of the two velocities would
  // (no branch: a face that is not evaluated here contributes zeros)
  auto face_part = [&](const FaceQ& F, V gb, V hb, V xn, V xix, V xiy, V wxv, V wyv, T (&part)[9]) {
    const V xp = P::sub(xix, P::splat(F.shx));
    const V yp = (D == 2) ? P::sub(xiy, P::splat(F.shy)) : P::splat(T(0));
    const V wg = P::mul(wxv, P::mul(wyv, gb));
    const V e = P::mul(wxv, P::mul(wyv, P::fma(P::fma(yp, yp, P::mul(xp, xp)), gb, hb)));
    const V q1 = P::mul(wg, xp), q2 = P::mul(wg, yp);
    const V q4 = P::mul(q1, xp), q5 = P::mul(q1, yp), q6 = P::mul(q2, yp);
    const V q7 = P::mul(e, xp), q8 = P::mul(e, yp);
    const bool in = F.meta && F.kind == FK_INTERIOR;
    part[0] = in ? wg.x + wg.y : T(0); part[1] = in ? q1.x + q1.y : T(0); part[2] = in ? q2.x + q2.y : T(0);
    part[3] = in ? e.x + e.y : T(0); part[4] = in ? q4.x + q4.y : T(0); part[5] = in ? q5.x + q5.y : T(0);
    part[6] = in ? q6.x + q6.y : T(0); part[7] = in ? q7.x + q7.y : T(0); part[8] = in ? q8.x + q8.y : T(0);
    if (F.meta && (F.kind == FK_WALL_LO || F.kind == FK_WALL_HI)) {
      const V xin = (F.kind == FK_WALL_LO) ? xn : P::mk(-xn.x, -xn.y);
      const V o = P::mul(wxv, P::mul(wyv, P::mul(xin, gb)));
      part[0] = (xin.x <= T(0) ? o.x : T(0)) + (xin.y <= T(0) ? o.y : T(0));
    }
  };

  // a warp none of whose lanes evaluates a face here (a partly filled tile of a level) skips the
  // face work of every round; it still stages its box positions
  const bool wface = !ML || __any_sync(0xffffffffu, FA.meta != 0 || FB.meta != 0 || FC.meta != 0);

  // register prefetch of the first pair
  V ng0, nh0, ng1 = P::splat(T(0)), nh1 = P::splat(T(0));
  ld2(kind0, p0, st0, v0, ng0, nh0);
  if (halo) ld2(kind1, p1, st1, v0, ng1, nh1);

  __syncthreads();   // velocity table in place
  int buf = 0;
  for (int j = 0; j < npr; ++j, buf ^= 1) {
    const int v = v0 + 2 * j;
    V* Pg = sP + (buf * 2 + 0) * B::NB;
    V* Ph = sP + (buf * 2 + 1) * B::NB;
    const V g0 = ng0, h0 = nh0, g1 = ng1, h1 = nh1;
    if (j + 1 < npr) {
      ld2(kind0, p0, st0, v + 2, ng0, nh0);
      if (halo) ld2(kind1, p1, st1, v + 2, ng1, nh1);
    }
    const V xix = sVT[4 * j], xiy = sVT[4 * j + 1];
    // ---- phi-bar-plus = phi~ + b (phi^S - phi~) of the own cell and the halo cell
    if (!ML || kind0 == 1) {
      V gs, hs;
      if constexpr (C8) model_eval2c8<T>(m0, b80, xix, xiy, c0, twoK, gs, hs);
      else model_eval2<T, D>(m0, xix, xiy, c0, twoK, gs, hs);
      Pg[e0] = P::fma(P::splat(m0.c1), P::sub(gs, g0), g0);
      Ph[e0] = P::fma(P::splat(m0.c1), P::sub(hs, h0), h0);
    } else {
      Pg[e0] = g0;
      Ph[e0] = h0;
    }
    if (halo) {
      if (!ML || kind1 == 1) {
        V gs, hs;
        if constexpr (C8) model_eval2c8<T>(m1, b81, xix, xiy, c0, twoK, gs, hs);
        else model_eval2<T, D>(m1, xix, xiy, c0, twoK, gs, hs);
        Pg[e1] = P::fma(P::splat(m1.c1), P::sub(gs, g1), g1);
        Ph[e1] = P::fma(P::splat(m1.c1), P::sub(hs, h1), h1);
      } else {
        Pg[e1] = g1;
        Ph[e1] = h1;
      }
    }
    __syncthreads();
    // ---- the faces this thread evaluates
    const V wxv = sVT[4 * j + 2], wyv = sVT[4 * j + 3];
    // the pair of a face: phi-bar to the face buffer (read by k_update of the same level; a
    // padding lane is stored too, so that every lane k_update reads is finite), its moments
    // faces A and B are evaluated without a branch (so that their work interleaves); only a
    // face evaluated here is stored and accumulates nonzero moments
    auto one = [&](const FaceQ& F, T (&part)[9]) {
      V gb, hb, xn;
      face_bar(F, Pg, Ph, xix, xiy, gb, hb, xn);
      if (F.meta) {
        T* o = fbo + fbar_at(0, v, F.fid, nvp, nfc);
        *reinterpret_cast<V*>(o) = gb;
        *reinterpret_cast<V*>(o + 2 * nvp * nfc) = hb;
      }
      face_part(F, gb, hb, xn, xix, xiy, wxv, wyv, part);
    };
    if (wface) {
      T part[9];
      one(FA, part);
      fold_partials<T>(ra[0], part);
      if (D == 2) {
        one(FB, part);
        fold_partials<T>(ra[1], part);
      }
      if (FC.meta) { one(FC, part); fold_partials_smem<T>(sAcc + tid, L::NX3, part); }
    }
  }

  // ---- write the chunk's partial moments
  if (FA.meta) write_partials<T, D>(ra[0], a.part + (long)chunk * NMOM * k.nface + FA.fid, k.nface);
  if (D == 2 && FB.meta) write_partials<T, D>(ra[1], a.part + (long)chunk * NMOM * k.nface + FB.fid, k.nface);
  if (FC.meta) write_partials_smem<T, D>(sAcc + tid, L::NX3, a.part + (long)chunk * NMOM * k.nface + FC.fid, k.nface);
}

// One face of k_update as a thread holds it: metadata, the model parameters of an evaluated
// face, and on curvilinear meshes its unit normal and area.
template <class T> struct UFace {
  int meta = 0;   // face_meta word, 0 if the thread has no such face
  int kind = 0, role = FR_NONE;
  long fid = 0;   // global face id (face buffer column)
  long col = 0;   // column in X (FR_CROSS) or Y (FR_RECV)
  MP<T> m;
  T nx = T(0), ny = T(0), area = T(1);
  T b8[4] = {T(0), T(0), T(0), T(0)};   // eight-moment correction (C8)
};

// Microflux (xi.n) phi (Eq. interface_reduced_fluxes, times |S| on curvilinear meshes) of an
// evaluated face for a velocity pair from its stored phi-bar (gb, hb): Eq. recover_phi on
// interior faces; on boundary faces the model enters (wall: rho_w = c1 + c2 times the
// unit-density wall Maxwellian; freestream: c1 = 1, c2 = 0 and the corrected freestream
// Maxwellian) and the reconstruction leaves, lane by lane.
template <class T, int D, bool CV, bool C8 = false>
__device__ __forceinline__ void face_flux2(const UFace<T>& F, int dir, V2<T> xix, V2<T> xiy, V2<T> gb, V2<T> hb,
                                           T c0, T twoK, V2<T>& Fg, V2<T>& Fh) {
  using P = Pk<T>;
  V2<T> xn;
  // xi.n as two rounded products and a rounded sum (curvilinear): the same value in every
  // kernel that evaluates this face
  if constexpr (CV) xn = P::add(P::mul(xix, P::splat(F.nx)), P::mul(xiy, P::splat(F.ny)));
  else xn = (dir == 0) ? xix : xiy;
  V2<T> gs, hs, gf, hf;
  if constexpr (C8) model_eval2c8<T>(F.m, F.b8, xix, xiy, c0, twoK, gs, hs);
  else model_eval2<T, D>(F.m, xix, xiy, c0, twoK, gs, hs);
  if (F.kind == FK_INTERIOR) {
    // weights summing to one, explicitly rounded: the two tiles that evaluate a shared face
    // produce the same bits (exact flux telescoping)
    gf = P::fma(P::splat(F.m.c2), P::sub(gs, gb), gb);
    hf = P::fma(P::splat(F.m.c2), P::sub(hs, hb), hb);
  } else {
    const V2<T> xin = fk_low(F.kind) ? xn : P::mk(-xn.x, -xn.y);
    const V2<T> gw = P::fma(P::splat(F.m.c1), gs, P::mul(P::splat(F.m.c2), gs));
    const V2<T> hw = P::fma(P::splat(F.m.c1), hs, P::mul(P::splat(F.m.c2), hs));
    gf.x = xin.x > T(0) ? gw.x : gb.x;
    gf.y = xin.y > T(0) ? gw.y : gb.y;
    hf.x = xin.x > T(0) ? hw.x : hb.x;
    hf.y = xin.y > T(0) ? hw.y : hb.y;
  }
  V2<T> xs = xn;
  if constexpr (CV) xs = P::mul(xn, P::splat(F.area));
  Fg = P::mul(xs, gf);
  Fh = P::mul(xs, hf);
}

// Eq. explicit_update on a tile: phi~^{n+1} = phi~+ - dt/|V| sum_faces (xi.n) phi |S|, with the
// face phi from the face buffer written by k_faces, then the cell moments of the stored values
// over the chunk.  One velocity pair per round.  Thread (tx, ty) holds its cell and the cell's
// low-side faces (A: x-face tx, B: y-face ty in 2-D), whose microfluxes go through shared
// memory (double-buffered: one barrier per round).  The tile's high-side faces C (the column
// li = TX and the row lj = TY) are evaluated for a sub-chunk of SC pairs at a time by every
// thread (face tid % NX3, pairs tid / NX3 + k NT / NX3), so the work per round is the same in
// every warp.  A face received from another level takes the microflux mapped to this level
// (Y), which k_cross_flux and the mapping produce before the launch.  Requires k.vpc <= VPC.
template <class S, class T, int D, int TX, int TY, int VPC, bool ML, bool CV, bool C8 = false>
__global__ void __launch_bounds__(TX * TY, (TX * TY >= 256) ? 2 : 4)
k_update(const TileArgs a_, const TileArgs* __restrict__ tab, const int4* __restrict__ work) {
  __shared__ __align__(16) TileArgs sa;
  int tile, chunk;
  if constexpr (ML) {
    const int4 w = work[blockIdx.x];
    load_args(sa, tab + w.x);
    __syncthreads();
    tile = sa.tiles[w.y];
    chunk = w.z;
  } else {
    tile = a_.tiles[blockIdx.x];
    chunk = (int)blockIdx.y;
  }
  const TileArgs& a = ML ? sa : a_;
  using G = TileGeom<TX, TY, D>;
  using L = UpdSmem<T, TX, TY, D, VPC>;
  using V = V2<T>;
  using P = Pk<T>;
  static_assert(!CV || D == 2, "curvilinear meshes are two-dimensional");
  static_assert(L::NX3 <= G::NT && G::NT % L::NX3 == 0, "high-side faces must divide the threads");
  constexpr int NT = G::NT, NX3 = L::NX3, SC = L::SC;
  extern __shared__ __align__(16) unsigned char smem[];
  V* sF = reinterpret_cast<V*>(smem + L::F);       // [2][2][NF] by pair
  V* sC = reinterpret_cast<V*>(smem + L::C);       // [2][2][SC][NX3] by pair
  V* sVT = reinterpret_cast<V*>(smem + L::VT);
  T* sXP = reinterpret_cast<T*>(smem + L::XP);
  long* sXI = reinterpret_cast<long*>(smem + L::XI);

  const StepConst& k = a.k;
  const S* __restrict__ fin = reinterpret_cast<const S*>(a.f_in);
  S* __restrict__ fout = reinterpret_cast<S*>(a.f_out);
  const T* __restrict__ cp = reinterpret_cast<const T*>(a.cparam);
  const T* __restrict__ fp = reinterpret_cast<const T*>(a.fparam);
  const T* __restrict__ vt = reinterpret_cast<const T*>(a.vt);
  const T* __restrict__ fbi = reinterpret_cast<const T*>(a.fbar);
  const T* __restrict__ fg = reinterpret_cast<const T*>(a.fgeo);
  const T* __restrict__ cg = reinterpret_cast<const T*>(a.cgeo);
  const T* __restrict__ Yi = reinterpret_cast<const T*>(a.Y);
  const long ns = a.nslot;
  const long nv = k.nv;
  const long nvp = (k.nv + 1) / 2;
  const long nfc = k.nface;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = (D == 2) ? tid / TX : 0;
  // random bits of the stochastic rounding of stored values (BF16 and FP32 storage)
  unsigned seed = 0;
  if constexpr (sizeof(S) <= 4) seed = hash32(*a.step * 0x632be5abu + a.salt);
  const int bx = tile % a.ntx, by = tile / a.ntx;
  const int x0 = bx * TX, y0 = by * TY;
  const int v0 = chunk * k.vpc;               // even: k.vpc is even
  const int v1 = min(k.nv, v0 + k.vpc);
  const int npr = (v1 - v0 + 1) / 2;

  // the chunk's velocity table by pairs, padded with zeros to whole sub-chunks
  for (int j = tid; j < L::NPT; j += NT) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int v = v0 + 2 * j;
      const T e0 = (v < v1 && !(r == 1 && D == 1)) ? vt[r * nv + v] : T(0);
      const T e1 = (v + 1 < v1 && !(r == 1 && D == 1)) ? vt[r * nv + v + 1] : T(0);
      sVT[4 * j + r] = P::mk(e0, e1);
    }
  }

  // ---- own cell
  const int gx = x0 + tx, gy = y0 + ty;
  bool own_active = gx < k.nx && (D == 1 || gy < k.ny);
  long col0 = 0;
  if (own_active) {
    const int c = ((D == 2) ? gy : 0) * k.nx + gx;
    if (!ML) col0 = c;
    else if (a.lvl_of[c] == a.level) col0 = a.slot_of[c];
    else own_active = false;
  }
  MP<T> m0;
  if (own_active) m0.load(cp, ns, col0);
  else m0.zero();
  T b80[4] = {T(0), T(0), T(0), T(0)};   // b4..b7 of the eight-moment correction (C8)
  if constexpr (C8) {
    if (own_active)
#pragma unroll
      for (int m = 0; m < 4; ++m) b80[m] = reinterpret_cast<const T*>(a.cparam8)[m * ns + col0];
  }
  T lamx = T(k.dt / k.dx), lamy = T(k.dt / k.dy);
  if constexpr (CV) {
    if (own_active) lamx = lamy = cg[4L * k.ncell + ((D == 2) ? gy : 0) * k.nx + gx];   // dt / |V|
  }
  // loads of the own cell: base pointer and velocity stride (0: a dummy element, never stored)
  const S* pO = fin + (own_active ? col0 : 0);
  const long so = own_active ? ns : 0;

  auto setup = [&](int f, UFace<T>& F) {
    int fid;
    F.meta = face_meta<TX, TY, D, ML>(a, x0, y0, f, fid);
    F.fid = fid;
    F.kind = (F.meta >> 2) & 7;
    F.role = F.meta >> 5;
    F.col = 0;
    F.m.zero();
    if (!(F.meta & FM_VALID)) { F.meta = 0; F.role = FR_NONE; return; }
    if (F.role == FR_CROSS || F.role == FR_RECV) F.col = a.fslot[fid];
    if (F.role == FR_NORMAL || F.role == FR_CROSS) {
      F.m.load(fp, nfc, fid);
      if constexpr (C8)
#pragma unroll
        for (int m = 0; m < 4; ++m) F.b8[m] = reinterpret_cast<const T*>(a.fparam8)[m * nfc + fid];
    }
    if constexpr (CV) {
      F.nx = fg[fid];
      F.ny = fg[nfc + fid];
      F.area = fg[2 * nfc + fid];
    }
  };
  // a face's loaded pair at velocities (v, v+1): face phi-bar (evaluated faces), mapped
  // microflux (received faces) or zeros
  auto ldface = [&](int role, long fid, long col, int v, V& g, V& h) {
    if (role == FR_NORMAL || role == FR_CROSS) {
      const T* q = fbi + fbar_at(0, v, fid, nvp, nfc);
      g = *reinterpret_cast<const V*>(q);
      h = *reinterpret_cast<const V*>(q + 2 * nvp * nfc);
    } else if (ML && role == FR_RECV) {
      const long vb = min(v + 1, v1 - 1);
      g = P::mk(Yi[(long)v * a.nY + col], Yi[vb * a.nY + col]);
      h = P::mk(Yi[(nv + v) * a.nY + col], Yi[(nv + vb) * a.nY + col]);
    } else {
      g = h = P::splat(T(0));
    }
  };

  // ---- faces C: parameters and ids in shared memory
  if (tid < NX3) {
    const int fC = (D == 1) ? TX : (tid < TY ? tid * (TX + 1) + TX : G::NFXL + TY * TX + (tid - TY));
    UFace<T> FC;
    setup(fC, FC);
    const T pv[16] = {FC.m.ux, FC.m.uy, FC.m.lnh, FC.m.inv2RT, FC.m.kqx, FC.m.kqy, FC.m.RT, FC.m.b0,
                      FC.m.b1, FC.m.b2, FC.m.b3, FC.m.c1, FC.m.c2, FC.nx, FC.ny, FC.area};
#pragma unroll
    for (int p = 0; p < 16; ++p) sXP[p * NX3 + tid] = pv[p];
    if constexpr (C8)
#pragma unroll
      for (int m = 0; m < 4; ++m) sXP[(16 + m) * NX3 + tid] = FC.b8[m];
    sXI[tid] = FC.meta;
    sXI[NX3 + tid] = FC.kind;
    sXI[2 * NX3 + tid] = FC.fid;
    sXI[3 * NX3 + tid] = FC.col;
  }
  // ---- faces A and B in registers
  const int fA = ty * (TX + 1) + tx;
  const int fB = G::NFXL + ty * TX + tx;
  UFace<T> FA, FB;
  setup(fA, FA);
  if (D == 2) setup(fB, FB);
  else FB.meta = 0, FB.role = FR_NONE;
  const bool evA = FA.role == FR_NORMAL || FA.role == FR_CROSS;
  const bool evB = D == 2 && (FB.role == FR_NORMAL || FB.role == FR_CROSS);
  // where the fluxes of the own cell's high-side faces are: a face A / B of a neighbour in
  // the tile, or a face C (index ty in the column, TY + tx in the row)
  const bool eInTile = tx < TX - 1, nInTile = ty < TY - 1;
  const int cE = (D == 1) ? 0 : ty, cN = TY + tx;

  // moments of the updated cell (the next step's partials), in the cell's frame
  KSum<T> c0k, cxk, cyk, cek;
  c0k.zero(); cxk.zero(); cyk.zero(); cek.zero();
  T cgxx = T(0), cgxy = T(0), cgyy = T(0), cjx = T(0), cjy = T(0);
  const T c0 = T(k.c0), twoK = T(k.twoK);
  __syncthreads();   // velocity table and faces C in place

  // the faces C of this thread in the pre-pass: face tid % NX3, pairs tid / NX3 + k NT / NX3
  const int qc = tid % NX3, jc0 = tid / NX3;
  const int dirC = (D == 1 || qc < TY) ? 0 : 1;
  // the own cell's pair and the faces A and B of a round, loaded one round ahead in registers
  // where registers allow (FP32 arithmetic on a level that holds every cell; the level-batched
  // and FP64 forms would spill)
  constexpr bool PF = !ML && sizeof(T) == 4;
  auto ld_round = [&](int j, V& g0, V& h0, V& ga, V& ha, V& gbb, V& hbb) {
    const int v = v0 + 2 * j;
    const long vb = min(v + 1, v1 - 1);
    g0 = P::mk(ldf<S, T>(pO + (long)v * so), ldf<S, T>(pO + vb * so));
    h0 = P::mk(ldf<S, T>(pO + (nv + v) * so), ldf<S, T>(pO + (nv + vb) * so));
    ldface(FA.role, FA.fid, FA.col, v, ga, ha);
    if (D == 2) ldface(FB.role, FB.fid, FB.col, v, gbb, hbb);
    else gbb = hbb = P::splat(T(0));
  };
  V ng0, nh0, nga, nha, ngb, nhb;
  if constexpr (PF) ld_round(0, ng0, nh0, nga, nha, ngb, nhb);
  int cbuf = 0, buf = 0;
  for (int jb = 0; jb < npr; jb += SC, cbuf ^= 1) {
    // ---- pre-pass: the microfluxes of the faces C over the sub-chunk
    {
      const long metaC = sXI[qc];
      const int roleC = (int)(metaC >> 5);
      const bool evC = roleC == FR_NORMAL || roleC == FR_CROSS;
      const long fidC = sXI[2 * NX3 + qc], colC = sXI[3 * NX3 + qc];
      UFace<T> FC;
      const T* X3p = sXP + qc;
      FC.kind = (int)sXI[NX3 + qc];
      FC.m.ux = X3p[0]; FC.m.uy = X3p[NX3]; FC.m.lnh = X3p[2 * NX3]; FC.m.inv2RT = X3p[3 * NX3];
      FC.m.kqx = X3p[4 * NX3]; FC.m.kqy = X3p[5 * NX3]; FC.m.RT = X3p[6 * NX3]; FC.m.b0 = X3p[7 * NX3];
      FC.m.b1 = X3p[8 * NX3]; FC.m.b2 = X3p[9 * NX3]; FC.m.b3 = X3p[10 * NX3]; FC.m.c1 = X3p[11 * NX3];
      FC.m.c2 = X3p[12 * NX3]; FC.nx = X3p[13 * NX3]; FC.ny = X3p[14 * NX3]; FC.area = X3p[15 * NX3];
      if constexpr (C8)
#pragma unroll
        for (int m = 0; m < 4; ++m) FC.b8[m] = X3p[(16 + m) * NX3];
      V* Cg = sC + (cbuf * 2 + 0) * SC * NX3;
      V* Ch = sC + (cbuf * 2 + 1) * SC * NX3;
      for (int jj = jc0; jj < SC; jj += NT / NX3) {
        const int jp = min(jb + jj, npr - 1);
        const int v = v0 + 2 * jp;
        V gl, hl;
        ldface(roleC, fidC, colC, v, gl, hl);
        V Fg = gl, Fh = hl;
        if (evC) face_flux2<T, D, CV, C8>(FC, dirC, sVT[4 * (jb + jj)], sVT[4 * (jb + jj) + 1], gl, hl, c0, twoK, Fg, Fh);
        Cg[jj * NX3 + qc] = Fg;
        Ch[jj * NX3 + qc] = Fh;
      }
    }
    const int je = min(jb + SC, npr);
    for (int j = jb; j < je; ++j, buf ^= 1) {
      const int v = v0 + 2 * j;
      V g0, h0, ga, ha, gbb, hbb;
      const V xix = sVT[4 * j], xiy = sVT[4 * j + 1];
      V* Fg = sF + (buf * 2 + 0) * G::NF;
      V* Fh = sF + (buf * 2 + 1) * G::NF;
      if constexpr (PF) {
        g0 = ng0; h0 = nh0; ga = nga; ha = nha; gbb = ngb; hbb = nhb;
        if (j + 1 < npr) ld_round(j + 1, ng0, nh0, nga, nha, ngb, nhb);
      } else {
        ld_round(j, g0, h0, ga, ha, gbb, hbb);
      }
      // faces A and B evaluated without a branch (a received face takes its mapped flux)
      V FAg, FAh;
      face_flux2<T, D, CV, C8>(FA, 0, xix, xiy, ga, ha, c0, twoK, FAg, FAh);
      if (!evA) { FAg = ga; FAh = ha; }
      Fg[fA] = FAg;
      Fh[fA] = FAh;
      if (D == 2) {
        V FBg, FBh;
        face_flux2<T, D, CV, C8>(FB, 1, xix, xiy, gbb, hbb, c0, twoK, FBg, FBh);
        if (!evB) { FBg = gbb; FBh = hbb; }
        Fg[fB] = FBg;
        Fh[fB] = FBh;
      }
      // the collision part of phi~+ - phi~ = (4/3) b (phi^S - phi~)
      V gs, hs;
      if constexpr (C8) model_eval2c8<T>(m0, b80, xix, xiy, c0, twoK, gs, hs);
      else model_eval2<T, D>(m0, xix, xiy, c0, twoK, gs, hs);
      V dg = P::mul(P::splat(m0.c2), P::sub(gs, g0));
      V dh = P::mul(P::splat(m0.c2), P::sub(hs, h0));
      __syncthreads();
      // minus the microflux divergence: the increment of the step
      const V* Cg = sC + (cbuf * 2 + 0) * SC * NX3 + (j - jb) * NX3;
      const V* Ch = sC + (cbuf * 2 + 1) * SC * NX3 + (j - jb) * NX3;
      const V FEg = eInTile ? Fg[fA + 1] : Cg[cE], FEh = eInTile ? Fh[fA + 1] : Ch[cE];
      dg = P::fma(P::splat(-lamx), P::sub(FEg, Fg[fA]), dg);
      dh = P::fma(P::splat(-lamx), P::sub(FEh, Fh[fA]), dh);
      if (D == 2) {
        const V FNg = nInTile ? Fg[fB + TX] : Cg[cN], FNh = nInTile ? Fh[fB + TX] : Ch[cN];
        dg = P::fma(P::splat(-lamy), P::sub(FNg, Fg[fB]), dg);
        dh = P::fma(P::splat(-lamy), P::sub(FNh, Fh[fB]), dh);
      }
      // random bits: one hash of (step, level, cell, velocity pair) per 32 bits
      unsigned rb0 = 0, rb1 = 0;
      if constexpr (sizeof(S) <= 4) {
        const unsigned key = seed ^ ((unsigned)col0 * 0x9e3779b1u + (unsigned)v);
        rb0 = hash32(key);
        rb1 = hash32(key ^ 0x5bd1e995u);
      }
      // phi~^{n+1} = phi~ + increment, rounded to the storage: stochastically for FP32 (the sum
      // itself) and BF16 (the FP32 sum), to nearest for FP64
      S sg0, sh0, sg1, sh1;
      if constexpr (sizeof(S) == 4) {
        const float2 gq2 = sr_add2(g0, dg, rb0, rb1), hq2 = sr_add2(h0, dh, rb0 >> 16, rb1 >> 16);
        sg0 = gq2.x; sg1 = gq2.y; sh0 = hq2.x; sh1 = hq2.y;
      } else {
        const V gn = P::add(g0, dg), hn = P::add(h0, dh);
        sg0 = Stored<S, T>::enc(gn.x, rb0); sh0 = Stored<S, T>::enc(hn.x, rb0 >> 16);
        sg1 = Stored<S, T>::enc(gn.y, rb1); sh1 = Stored<S, T>::enc(hn.y, rb1 >> 16);
      }
      if (own_active) {
        fout[(long)v * ns + col0] = sg0;
        fout[(nv + v) * ns + col0] = sh0;
        if (v + 1 < v1) {
          fout[(long)(v + 1) * ns + col0] = sg1;
          fout[(nv + v + 1) * ns + col0] = sh1;
        }
      }
      const V gq = P::mk(Stored<S, T>::dec(sg0), Stored<S, T>::dec(sg1));
      const V hq = P::mk(Stored<S, T>::dec(sh0), Stored<S, T>::dec(sh1));
      const V wxv = sVT[4 * j + 2], wyv = sVT[4 * j + 3];
      const V xp = P::sub(xix, P::splat(m0.ux));
      const V yp = (D == 2) ? P::sub(xiy, P::splat(m0.uy)) : P::splat(T(0));
      const V wg = P::mul(wxv, P::mul(wyv, gq));
      const V e = P::mul(wxv, P::mul(wyv, P::fma(P::fma(yp, yp, P::mul(xp, xp)), gq, hq)));
      const V q1 = P::mul(wg, xp), q7 = P::mul(e, xp);
      c0k.add(wg.x); c0k.add(wg.y);
      cxk.add(q1.x); cxk.add(q1.y);
      cek.add(e.x); cek.add(e.y);
      const V q4 = P::mul(q1, xp);
      cgxx += q4.x + q4.y;
      cjx += q7.x + q7.y;
      if (D == 2) {
        const V q2 = P::mul(wg, yp), q5 = P::mul(q1, yp), q6 = P::mul(q2, yp), q8 = P::mul(e, yp);
        cyk.add(q2.x); cyk.add(q2.y);
        cgxy += q5.x + q5.y;
        cgyy += q6.x + q6.y;
        cjy += q8.x + q8.y;
      }
    }
  }

  // ---- write the chunk's partial moments of the own cell
  if (own_active) {
    double* Pp = a.part + (long)chunk * NMOM * ns + col0;
    Pp[MO_0 * ns] = c0k.val();
    Pp[MO_X * ns] = cxk.val();
    Pp[MO_Y * ns] = (D == 2) ? cyk.val() : 0.0;
    Pp[MO_E * ns] = cek.val();
    Pp[MO_GXX * ns] = (double)cgxx;
    Pp[MO_GXY * ns] = (double)cgxy;
    Pp[MO_GYY * ns] = (double)cgyy;
    Pp[MO_JX * ns] = (double)cjx;
    Pp[MO_JY * ns] = (double)cjy;
  }
}

// Microfluxes (xi.n) phi of the cross-level faces a level evaluates (Eq. interface_reduced_fluxes
// on the faces' common refinement space, Sec. 3.4) into the level's X array, from which the
// mapping takes them to the neighbouring levels.  The faces are interior faces: Eq. recover_phi
// from the face buffer and the face model, with the operations of k_update's evaluation of
// the same face, so both sides of the face see one flux.  One thread per X column, kXPairs
// velocity pairs per CTA; work item (level, first column, first pair, 0).
constexpr int kXPairs = 32;
template <class T, int D, bool CV>
__global__ void __launch_bounds__(128) k_cross_flux(const TileArgs* __restrict__ tab, const int4* __restrict__ work) {
  using V = V2<T>;
  using P = Pk<T>;
  __shared__ __align__(16) TileArgs sa;
  const int4 w = work[blockIdx.x];
  load_args(sa, tab + w.x);
  __syncthreads();
  const TileArgs& a = sa;
  const StepConst& k = a.k;
  const int col = w.y + (int)threadIdx.x;
  if (col >= a.nX) return;
  const long nv = k.nv, nvp = (k.nv + 1) / 2, nfc = k.nface;
  const long fid = a.xfid[col];
  const T* __restrict__ fp = reinterpret_cast<const T*>(a.fparam);
  const T* __restrict__ vt = reinterpret_cast<const T*>(a.vt);
  const T* __restrict__ fbi = reinterpret_cast<const T*>(a.fbar);
  T* __restrict__ Xo = reinterpret_cast<T*>(a.X);
  UFace<T> F;
  F.kind = FK_INTERIOR;
  F.m.load(fp, nfc, fid);
  if constexpr (CV) {
    const T* __restrict__ fg = reinterpret_cast<const T*>(a.fgeo);
    F.nx = fg[fid];
    F.ny = fg[nfc + fid];
    F.area = fg[2 * nfc + fid];
  }
  const int dir = fid < (long)k.nfx * k.ny ? 0 : 1;
  const T c0 = T(k.c0), twoK = T(k.twoK);
  const int j1 = min((int)nvp, w.z + kXPairs);
  for (int j = w.z; j < j1; ++j) {
    const int v = 2 * j;
    const bool hi = v + 1 < nv;
    const V xix = P::mk(vt[v], hi ? vt[v + 1] : T(0));
    const V xiy = (D == 2) ? P::mk(vt[nv + v], hi ? vt[nv + v + 1] : T(0)) : P::splat(T(0));
    const T* q = fbi + fbar_at(0, v, fid, nvp, nfc);
    const V gb = *reinterpret_cast<const V*>(q);
    const V hb = *reinterpret_cast<const V*>(q + 2 * nvp * nfc);
    V Fg, Fh;
    face_flux2<T, D, CV>(F, dir, xix, xiy, gb, hb, c0, twoK, Fg, Fh);
    Xo[(long)v * a.nX + col] = Fg.x;
    Xo[(nv + v) * a.nX + col] = Fh.x;
    if (hi) {
      Xo[(long)(v + 1) * a.nX + col] = Fg.y;
      Xo[(nv + v + 1) * a.nX + col] = Fh.y;
    }
  }
}

}  // namespace mlvs
