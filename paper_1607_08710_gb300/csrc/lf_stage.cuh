// Fused Heun stage of the Lagrange-flux scheme (arXiv:1607.08710, Sec. 4):
// per cell, primitive conversion (eq. 1), limited MUSCL slopes in x and y
// (eq. "sweby"), face states, the acoustic interface solve (eqs. 13-14), the
// upwind Lagrange flux (eq. 12) and the conservative update -- one kernel per
// stage, no face quantity ever written to memory.  A cell carries NF = 4 +
// nspecies fields: the transported mass fractions of Sec. 5 are reconstructed
// and upwinded with the gas state, so they add planes, not passes.
//
// Work decomposition.  A warp owns a strip of 32*CPL consecutive columns,
// CPL cells per lane, computed as one lane value (FP32: both cells of a lane
// as a packed pair on the paired FP32 instructions; FP64: one cell).  The two columns at each end are the halo the 5-point
// MUSCL stencil needs, so a strip produces 32*CPL - 4 output columns and all
// x-neighbour exchange is done with warp shuffles (no shared memory, no
// __syncthreads).  The warp marches up a tile of rows carrying the y-stencil
// in registers: primitives of three rows, y-slopes and the flux through the
// face below, each in three slots indexed by row mod 3.  The march is
// unrolled by three so the slots are compile-time register names and nothing
// is copied from row to row (the batched kernel can instead run one row body
// and rotate the window after each row: a third of the code, for a few
// register moves per row).  Rows are staged by cp.async into a per-warp
// shared-memory ring four rows ahead; the conservative values of the row
// being updated are read back from the ring rather than carried.  Every
// primitive, slope and face flux is computed once per cell, up to the 4 halo
// columns of a strip and the 2 halo rows below and above a tile.  The tile
// height is a launch parameter (MeshDesc::ty); strips that lie inside their
// rows run a march without per-lane copy and store choices.
//
// Memory safety.  Every load index is mapped into [0, nx) x [0, ny) by the
// boundary condition (clamp or wrap); vector loads/stores are used only when
// both cells of the pair are inside the row; stores are issued only for
// output cells (column < nx, row < ny).  In-plane element offsets are 32-bit:
// lf_init refuses meshes whose padded plane reaches 2^31 elements.
#pragma once

#include "lf_device.cuh"

namespace lf {

// Launch shape; the defaults were chosen by timing on GB300 and can be
// overridden at build time for tuning sweeps.
#ifndef LF_STAGE_WARPS
#define LF_STAGE_WARPS 1
#endif
#ifndef LF_TY_F32
#define LF_TY_F32 64
#endif
#ifndef LF_TY_F64
#define LF_TY_F64 64
#endif
#ifndef LF_MIN_BLOCKS0
#define LF_MIN_BLOCKS0 18
#endif
#ifndef LF_MIN_BLOCKS1
#define LF_MIN_BLOCKS1 17
#endif
constexpr int STAGE_WARPS = LF_STAGE_WARPS;  // warps per CTA, side by side in x

template <int CPL> struct StripGeom {
  static constexpr int COLS = 32 * CPL;     // columns covered by a warp
  static constexpr int OUT = 32 * CPL - 4;  // output columns per warp
};

// A strip whose 32*CPL columns [i0-2, i0-2+32*CPL) all lie inside the row,
// with vector accesses allowed (FP32 pairs need the even row pitch and the
// aligned planes that m.vec certifies).  Uniform over a warp.
template <int CPL>
__device__ __forceinline__ bool inner_strip(const MeshDesc& m, int i0) {
  return (CPL == 1 || m.vec) && i0 - 2 >= 0 && i0 - 2 + 32 * CPL <= m.nx;
}

// Rows are uniform across a warp; wrap or clamp without an integer division.
// map_row_ahead: for rows known to be >= 0 (the rows a march prefetches
// ahead of itself); stating that saves the march a wrap loop per row, which
// measured 5% of the 2D stage's time once the tile height became a runtime
// value and the compiler could no longer infer it.
__device__ __forceinline__ int map_row_ahead(int r, int n, int bc) {
  if (bc == BC_PERIODIC) {
    while (r >= n) r -= n;
    return r;
  }
  return r >= n ? n - 1 : r;
}
__device__ __forceinline__ int map_row(int r, int n, int bc) {
  if (bc == BC_PERIODIC) {
    while (r < 0) r += n;
    while (r >= n) r -= n;
    return r;
  }
  return r < 0 ? 0 : (r >= n ? n - 1 : r);
}

template <typename T, int CPL> struct VecLoad;
template <typename T> struct VecLoad<T, 1> {
  static __device__ __forceinline__ void load(const T* __restrict__ p, T v[1]) { v[0] = __ldg(p); }
  static __device__ __forceinline__ void load_plain(const T* p, T v[1]) { v[0] = *p; }
  static __device__ __forceinline__ void store(T* p, const T v[1]) { *p = v[0]; }
};
template <> struct VecLoad<float, 2> {
  static __device__ __forceinline__ void load(const float* __restrict__ p, float v[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
  static __device__ __forceinline__ void load_plain(const float* p, float v[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  }
  static __device__ __forceinline__ void store(float* p, const float v[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <> struct VecLoad<double, 2> {
  static __device__ __forceinline__ void load(const double* __restrict__ p, double v[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
  static __device__ __forceinline__ void load_plain(const double* p, double v[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  }
  static __device__ __forceinline__ void store(double* p, const double v[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// Per-lane column bookkeeping of a strip.
template <int CPL> struct LaneCols {
  int c0;           // first column of this lane (may be < 0 or >= nx)
  int ic[CPL];      // boundary-mapped columns
  bool vec_ok;      // all CPL columns inside [0, nx): one vector access
  bool out[CPL];    // cell is an output cell of this strip (and column < nx)
  bool any_out;
};

template <int CPL>
__device__ __forceinline__ LaneCols<CPL> lane_cols(int i0, int lane, int nx, int bc, int vec) {
  LaneCols<CPL> L;
  L.c0 = i0 - 2 + CPL * lane;
  L.any_out = false;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = L.c0 + j;
    L.ic[j] = map_index(c, nx, bc);
    const int k = CPL * lane + j;  // position in the strip
    L.out[j] = k >= 2 && k < 32 * CPL - 2 && c < nx;
    L.any_out |= L.out[j];
  }
  L.vec_ok = (CPL == 1 || vec) && L.c0 >= 0 && L.c0 + CPL - 1 < nx;
  return L;
}

// A lane value from / to the CPL cells of a lane.
__device__ __forceinline__ void make_lane(const float v[1], float& out) { out = v[0]; }
__device__ __forceinline__ void make_lane(const double v[1], double& out) { out = v[0]; }
__device__ __forceinline__ void make_lane(const float v[2], F2& out) { out = F2(v[0], v[1]); }
__device__ __forceinline__ void split_lane(float x, float v[1]) { v[0] = x; }
__device__ __forceinline__ void split_lane(double x, double v[1]) { v[0] = x; }
__device__ __forceinline__ void split_lane(F2 x, float v[2]) {
  v[0] = x.v.x;
  v[1] = x.v.y;
}

// The values one cell to the left / right of each of the lane's cells (the
// neighbouring lane's cells by warp shuffle).
constexpr unsigned FULL_MASK = 0xffffffffu;
__device__ __forceinline__ float prev_cell(float q) { return __shfl_up_sync(FULL_MASK, q, 1); }
__device__ __forceinline__ double prev_cell(double q) { return __shfl_up_sync(FULL_MASK, q, 1); }
__device__ __forceinline__ F2 prev_cell(F2 q) { return F2(__shfl_up_sync(FULL_MASK, q.v.y, 1), q.v.x); }
__device__ __forceinline__ float next_cell(float q) { return __shfl_down_sync(FULL_MASK, q, 1); }
__device__ __forceinline__ double next_cell(double q) { return __shfl_down_sync(FULL_MASK, q, 1); }
__device__ __forceinline__ F2 next_cell(F2 q) { return F2(q.v.y, __shfl_down_sync(FULL_MASK, q.v.x, 1)); }

// Conservative values of this lane's CPL cells in row `off` (= mapped row * pitch).
template <typename T, int CPL, int NF, typename V>
__device__ __forceinline__ void load_row(const T* const __restrict__ P[NF], const LaneCols<CPL>& L, int off,
                                         V U[NF]) {
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    T v[CPL];
    if (L.vec_ok) {
      VecLoad<T, CPL>::load(P[k] + off + L.c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) v[j] = __ldg(P[k] + off + L.ic[j]);
    }
    make_lane(v, U[k]);
  }
}

// Fluxes through the x-faces of this lane's cells, from the primitive lane
// values q of the current row.  Fr: right face of each cell, Fl: left face
// (valid for output cells).  Every x-face of the strip is computed once: the
// faces to the right of the lane's cells, whose right states are the next
// cells' (the last one from the next lane).
template <typename V, int LIM, int NF>
__device__ __forceinline__ void x_fluxes(const Phys<V>& P, const V q[NF], V Fl[NF], V Fr[NF]) {
  V qL[NF], qR[NF];  // left and right states of each cell's right face
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const V h = limiter_half<V, LIM>(q[k] - prev_cell(q[k]), next_cell(q[k]) - q[k], P.beta);
    qL[k] = q[k] + h;
    qR[k] = next_cell(q[k] - h);
  }
  lagrange_flux<V, 0, NF>(P, qL, qR, Fr);
#pragma unroll
  for (int k = 0; k < NF; ++k) Fl[k] = prev_cell(Fr[k]);
}

// Warp-level max and any(), then one atomic per warp.
template <typename T>
__device__ __forceinline__ void publish_speed(Scalars* sc, int wpar, T smax, bool bad) {
  constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(FULL, smax, o));
  const bool any_bad = __any_sync(FULL, bad);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_speed(&sc->smax[wpar], double(smax));
    if (any_bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
  }
}

// Cells per lane, lane value and tile height per precision (FP32: two cells
// per lane as one packed pair; FP64 keeps one cell per lane to stay clear of
// register spills).
template <typename T> struct StageShape { static constexpr int CPL = 2, TY = LF_TY_F32; using V = F2; };
template <> struct StageShape<double> { static constexpr int CPL = 1, TY = LF_TY_F64; using V = double; };

// ---------------------------------------------------------------------------
// Asynchronous row staging.  Every row a warp reads from global memory is
// copied with cp.async into a per-warp ring in shared memory a few rows ahead
// of its use, so no registers hold data in flight and memory latency is
// hidden behind the arithmetic of the rows in between.  Each lane copies and
// later reads back only its own CPL cells, so a lane's cp.async.wait_group is
// the only synchronisation needed (no __syncwarp / __syncthreads).
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Ring geometry.  Input rows: at row r the march reads row r+2 (new
// primitives) and row r (the cell values for the update) and issues row
// r+4, so rows r .. r+4 are live: 5 buffers.  U^n rows (corrector): row r is
// read and row r+2 issued: 3 buffers.  A buffer holds one row of the strip,
// laid out [field][lane][cell].
constexpr int RING_IN = 5, RING_UN = 3, AHEAD_IN = 4, AHEAD_UN = 2;

template <typename T, int CPL, int NF> struct Ring {
  static constexpr int ROW = NF * 32 * CPL;  // elements per buffer
  static __host__ __device__ constexpr int buffers(int stage) { return RING_IN + (stage ? RING_UN : 0); }
  static __host__ __device__ constexpr size_t warp_bytes(int stage) { return (size_t)buffers(stage) * ROW * sizeof(T); }
};

// How a strip's march makes its copies and stores.  An inner strip lies
// inside the row with vector accesses allowed for every lane (a warp-uniform
// property), so each lane issues one copy per field and row; other strips
// choose per lane between the vector and the per-cell boundary-mapped path.
//   MARCH_MAPPED: per-lane choice (any strip)
//   MARCH_INNER:  the strip is inner (compiled without the per-lane choice)
enum { MARCH_MAPPED = 0, MARCH_INNER = 1 };

// Copies this lane's cells of (mapped) row offset `off` into buffer `buf`.
template <typename T, int CPL, int NF, int MODE = MARCH_MAPPED>
__device__ __forceinline__ void issue_row(T* buf, const T* const P[NF], const LaneCols<CPL>& L, int off, int lane) {
  if (MODE == MARCH_INNER) {
#pragma unroll
    for (int k = 0; k < NF; ++k) cp_async<CPL * sizeof(T)>(buf + (k * 32 + lane) * CPL, P[k] + off + L.c0);
    return;
  }
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    T* dst = buf + (k * 32 + lane) * CPL;
    const T* src = P[k] + off;
    if (L.vec_ok) {
      cp_async<CPL * sizeof(T)>(dst, src + L.c0);
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) cp_async<sizeof(T)>(dst + j, src + L.ic[j]);
    }
  }
}

// Same for the output cells only (row offset `off` inside the mesh).  In an
// inner strip the halo lanes copy their in-row cells too (never read).
template <typename T, int CPL, int NF, int MODE = MARCH_MAPPED>
__device__ __forceinline__ void issue_out_cells(T* buf, const T* const P[NF], const LaneCols<CPL>& L, int off,
                                                int lane) {
  if (MODE == MARCH_INNER) {
#pragma unroll
    for (int k = 0; k < NF; ++k) cp_async<CPL * sizeof(T)>(buf + (k * 32 + lane) * CPL, P[k] + off + L.c0);
    return;
  }
  if (!L.any_out) return;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    T* dst = buf + (k * 32 + lane) * CPL;
    const T* src = P[k] + off + L.c0;
    if (L.vec_ok) {
      cp_async<CPL * sizeof(T)>(dst, src);  // with vec_ok, all or none of the lane's cells are outputs
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j)
        if (L.out[j]) cp_async<sizeof(T)>(dst + j, src + j);
    }
  }
}

template <typename T, int CPL, int NF, typename V>
__device__ __forceinline__ void read_row(const T* buf, int lane, V out[NF]) {
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    T v[CPL];
    VecLoad<T, CPL>::load_plain(buf + (k * 32 + lane) * CPL, v);
    make_lane(v, out[k]);
  }
}

// Stages of the time integrators, out = alpha U^n + beta (Uin - dt D(Uin)):
//   0: alpha 0,   beta 1    first stage of Heun (Sec. 4, step 6) and of SSP-RK3
//   1: alpha 1/2, beta 1/2  Heun corrector (Sec. 4, step 11), + wave-speed max
//   2: alpha 3/4, beta 1/4  second SSP-RK3 stage
//   3: alpha 1/3, beta 2/3  third SSP-RK3 stage, + wave-speed max
// Stages >= 1 read U^n at the cell; the last stage of a step feeds the CFL
// maximum of the new state.
template <int STAGE> struct StageCoef;
template <> struct StageCoef<0> { static constexpr double alpha = 0.0, beta = 1.0; static constexpr bool speed = false; };
template <> struct StageCoef<1> { static constexpr double alpha = 0.5, beta = 0.5; static constexpr bool speed = true; };
template <> struct StageCoef<2> { static constexpr double alpha = 0.75, beta = 0.25; static constexpr bool speed = false; };
template <> struct StageCoef<3> { static constexpr double alpha = 1.0 / 3.0, beta = 2.0 / 3.0; static constexpr bool speed = true; };

// State of the y-march: three register slots indexed by row mod 3.
template <typename V, int NF> struct March {
  V q[3][NF];  // primitives of rows r, r+1, r+2
  V s[3][NF];  // half y-slopes (limiter_half)
  V G[3][NF];  // G[slot(r)] = flux through face r-1/2
};

template <typename T, int STAGE, int CPL, int NF> struct StageArgs {
  const T* P[NF];  // Uin planes (read with halo)
  const T* N[NF];  // U^n planes (corrector, read at the cell)
  T* O[NF];        // output planes
  T* ring_in;     // this warp's input ring
  T* ring_un;     // this warp's U^n ring (corrector)
  int j0;         // first row of the tile
};

__device__ __forceinline__ int ring_slot(int row, int j0, int n) { return (row - j0 + 2 * n) % n; }

// One row of the march.  S = slot of row r in the register window.
// ring slot of row r + k, given si = slot of row r (0 <= k < RING_IN)
__device__ __forceinline__ int ring_in_plus(int si, int k) {
  const int t = si + k;
  return t >= RING_IN ? t - RING_IN : t;
}

template <typename T, typename V, int LIM, int STAGE, int CPL, int NF, int S, int MODE>
__device__ __forceinline__ void march_row(const Phys<V>& P, const MeshDesc& m,
                                          const StageArgs<T, STAGE, CPL, NF>& A, const LaneCols<CPL>& L,
                                          March<V, NF>& M, int lane, int r, int si, V ncx, V ncy,
                                          T& smax, bool& bad, int un_cur = S, int un_ahead = (S + 2) % 3) {
  constexpr int S1 = (S + 1) % 3, S2 = (S + 2) % 3;
  constexpr int ROW = Ring<T, CPL, NF>::ROW;
  static_assert(RING_UN == 3, "the U^n ring is indexed by the register slot");
  // the group issued two rows ago (input row r+2, U^n row r) has landed
  cp_wait<1>();
  {
    V Ut[NF];
    read_row<T, CPL, NF>(A.ring_in + ring_in_plus(si, 2) * ROW, lane, Ut);
    to_prim<V, NF>(P, Ut, M.q[S2]);
  }
  // Rows r+4 (input) and r+2 (U^n) are issued on every row, also near the
  // end of the tile where they are not needed: the row index stays valid
  // (boundary-mapped, or clamped to the last row) and the target buffers
  // (rows r-1) are no longer read, so the branch-free row body costs two idle
  // copies per tile.  strip_tile_impl drains them before returning.
  issue_row<T, CPL, NF, MODE>(A.ring_in + ring_in_plus(si, AHEAD_IN) * ROW, A.P, L,
                              map_row_ahead(r + AHEAD_IN, m.ny, m.bc) * m.pitch, lane);
  if (STAGE >= 1)  // U^n row r+2 lives in register slot S2's ring buffer
    issue_out_cells<T, CPL, NF, MODE>(A.ring_un + un_ahead * ROW, A.N, L, min(r + AHEAD_UN, m.ny - 1) * m.pitch,
                                      lane);
  cp_commit();
  // y-slopes of row r+1 and the flux through face r+1/2
  {
    V Lq[NF], Rq[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      M.s[S1][k] = limiter_half<V, LIM>(M.q[S1][k] - M.q[S][k], M.q[S2][k] - M.q[S1][k], P.beta);
      Lq[k] = M.q[S][k] + M.s[S][k];
      Rq[k] = M.q[S1][k] - M.s[S1][k];
    }
    lagrange_flux<V, 1, NF>(P, Lq, Rq, M.G[S1]);
  }
  // x-faces of row r
  V Fl[NF], Fr[NF];
  x_fluxes<V, LIM, NF>(P, M.q[S], Fl, Fr);
  // update the output cells of row r (computed on every lane; only output
  // cells are stored and enter the wave-speed maximum)
  V U[NF], Un[NF];
  read_row<T, CPL, NF>(A.ring_in + si * ROW, lane, U);
  if (STAGE >= 1) read_row<T, CPL, NF>(A.ring_un + un_cur * ROW, lane, Un);
  V W[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const V base = STAGE == 0 ? U[k]
                 : STAGE == 1 ? splat<V>(0.5) * (Un[k] + U[k])
                              : fma_(splat<V>(StageCoef<STAGE>::alpha), Un[k], splat<V>(StageCoef<STAGE>::beta) * U[k]);
    W[k] = fma_(ncy, M.G[S1][k] - M.G[S][k], fma_(ncx, Fr[k] - Fl[k], base));
  }
  const int off = r * m.pitch;
  if ((MODE == MARCH_INNER || L.vec_ok) && L.any_out) {
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T v[CPL];
      split_lane(W[k], v);
      VecLoad<T, CPL>::store(A.O[k] + off + L.c0, v);
    }
  } else if (MODE != MARCH_INNER && !L.vec_ok) {
#pragma unroll
    for (int j = 0; j < CPL; ++j)
      if (L.out[j])
#pragma unroll
        for (int k = 0; k < NF; ++k) A.O[k][off + L.c0 + j] = get(W[k], j);
  }
  if (StageCoef<STAGE>::speed) {
    typename LaneT<V>::M ok;
    const V sp = cell_speed<V, 2>(P, W, ok);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      smax = L.out[j] ? fmax(smax, get(sp, j)) : smax;
      bad |= L.out[j] && !get(ok, j);
    }
  }
}

// One warp's strip of columns [i0-2, i0-2+32*CPL) over the tile rows
// [j0, jend): the whole y-march, from the prologue to the last row.  The
// warp's rings start empty and are left with no copy in flight.
// STAGE 0: out = Uin - dt L(Uin).  STAGE 1: out = (Un + Uin)/2 - dt/2 L(Uin).
template <typename T, typename V, int LIM, int STAGE, int CPL, int NF, int MODE, bool ROT = false>
__device__ __forceinline__ void strip_tile_impl(const Phys<V>& P, const MeshDesc& m, const T* Uin, const T* Un,
                                                T* out, int i0, int j0, int jend, T cx, T cy, T* ring_in, int lane,
                                                T& smax, bool& bad) {
  const LaneCols<CPL> L = lane_cols<CPL>(i0, lane, m.nx, m.bc, m.vec);
  constexpr int ROW = Ring<T, CPL, NF>::ROW;
  StageArgs<T, STAGE, CPL, NF> A;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    A.P[k] = Uin + k * m.plane;
    A.N[k] = Un + k * m.plane;
    A.O[k] = out + k * m.plane;
  }
  A.ring_in = ring_in;
  A.ring_un = ring_in + RING_IN * ROW;
  A.j0 = j0;

  // Prologue.  Group 0: input rows j0-2 .. j0+1.  Group 1: input row j0+2 and
  // U^n row j0.  Rows j0-2 .. j0+1 give the register window: primitives in
  // slots (row - j0 + 3) % 3, y-slopes of rows j0-1 (slot 2) and j0 (slot 0),
  // and the flux through face j0-1/2 (slot 0).  Group 2 (input row j0+3, U^n
  // row j0+1) reuses row j0-2's buffer, so it is issued after that row is read.
  for (int row = j0 - 2; row <= j0 + 1; ++row)
    issue_row<T, CPL, NF, MODE>(A.ring_in + ring_slot(row, j0, RING_IN) * ROW, A.P, L,
                                map_row(row, m.ny, m.bc) * m.pitch, lane);
  cp_commit();
  issue_row<T, CPL, NF, MODE>(A.ring_in + ring_slot(j0 + 2, j0, RING_IN) * ROW, A.P, L,
                              map_row(j0 + 2, m.ny, m.bc) * m.pitch, lane);
  if (STAGE >= 1) issue_out_cells<T, CPL, NF, MODE>(A.ring_un + 0 * ROW, A.N, L, j0 * m.pitch, lane);
  cp_commit();
  cp_wait<1>();
  March<V, NF> M;
  {
    V Ut[NF];
    const int slot_of[4] = {1, 2, 0, 1};  // rows j0-2, j0-1, j0, j0+1 -> register slots
    V qm2[NF];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      read_row<T, CPL, NF>(A.ring_in + ring_slot(j0 - 2 + t, j0, RING_IN) * ROW, lane, Ut);
      to_prim<V, NF>(P, Ut, t == 0 ? qm2 : M.q[slot_of[t]]);
    }
    V Lq[NF], Rq[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      M.s[2][k] = limiter_half<V, LIM>(M.q[2][k] - qm2[k], M.q[0][k] - M.q[2][k], P.beta);
      M.s[0][k] = limiter_half<V, LIM>(M.q[0][k] - M.q[2][k], M.q[1][k] - M.q[0][k], P.beta);
      Lq[k] = M.q[2][k] + M.s[2][k];
      Rq[k] = M.q[0][k] - M.s[0][k];
    }
    lagrange_flux<V, 1, NF>(P, Lq, Rq, M.G[0]);
  }
  if (j0 + 1 < jend) {
    issue_row<T, CPL, NF, MODE>(A.ring_in + ring_slot(j0 + 3, j0, RING_IN) * ROW, A.P, L,
                                map_row(j0 + 3, m.ny, m.bc) * m.pitch, lane);
    if (STAGE >= 1)
      issue_out_cells<T, CPL, NF, MODE>(A.ring_un + 1 * ROW, A.N, L, (j0 + 1) * m.pitch, lane);
  }
  cp_commit();

  // si: input-ring slot of row r (row j0 is in slot 0); the update's dt/dx
  // and dt/dy enter negated (fma(-c, d, b) == fma(c', d, b) with c' = -c)
  const V ncx = V(-cx), ncy = V(-cy);
  if constexpr (ROT) {
    // One row body, the register window rotated after each row (a third of
    // the code of the unrolled march, for a few register moves per row); the
    // U^n ring follows the row index mod 3.
    for (int r = j0, si = 0, ui = 0;;) {
      march_row<T, V, LIM, STAGE, CPL, NF, 0, MODE>(P, m, A, L, M, lane, r, si, ncx, ncy, smax, bad, ui,
                                                    ui == 0 ? 2 : ui - 1);
#pragma unroll
      for (int k = 0; k < NF; ++k) {  // row r+1 -> slot 0, r+2 -> slot 1
        M.q[0][k] = M.q[1][k];
        M.q[1][k] = M.q[2][k];
        M.s[0][k] = M.s[1][k];
        M.G[0][k] = M.G[1][k];
      }
      if (++r >= jend) break;
      si = ring_in_plus(si, 1);
      ui = ui == 2 ? 0 : ui + 1;
    }
    cp_wait_all();
    return;
  }
  for (int r = j0, si = 0;;) {
    march_row<T, V, LIM, STAGE, CPL, NF, 0, MODE>(P, m, A, L, M, lane, r, si, ncx, ncy, smax, bad);
    if (++r >= jend) break;
    si = ring_in_plus(si, 1);
    march_row<T, V, LIM, STAGE, CPL, NF, 1, MODE>(P, m, A, L, M, lane, r, si, ncx, ncy, smax, bad);
    if (++r >= jend) break;
    si = ring_in_plus(si, 1);
    march_row<T, V, LIM, STAGE, CPL, NF, 2, MODE>(P, m, A, L, M, lane, r, si, ncx, ncy, smax, bad);
    if (++r >= jend) break;
    si = ring_in_plus(si, 1);
  }
  cp_wait_all();
}

// A strip whose 32*CPL columns all lie inside the row, with vector accesses
// allowed, runs the march without per-lane copy or store choices (decided
// once per warp: i0 is warp-uniform); edge strips take the mapped path.  Both
// do the same arithmetic, so results do not depend on which one ran.
// ROT: 0 = both marches unrolled by three, 1 = both with one row body and a
// rotating register window, 2 = only the mapped (edge-strip) march rotating.
template <typename T, typename V, int LIM, int STAGE, int CPL, int NF, int ROT = 0>
__device__ __forceinline__ void strip_tile(const Phys<V>& P, const MeshDesc& m, const T* Uin, const T* Un, T* out,
                                           int i0, int j0, int jend, T cx, T cy, T* ring_in, int lane, T& smax,
                                           bool& bad) {
  if (inner_strip<CPL>(m, i0))
    strip_tile_impl<T, V, LIM, STAGE, CPL, NF, MARCH_INNER, ROT == 1>(P, m, Uin, Un, out, i0, j0, jend, cx, cy,
                                                                      ring_in, lane, smax, bad);
  else
    strip_tile_impl<T, V, LIM, STAGE, CPL, NF, MARCH_MAPPED, ROT != 0>(P, m, Uin, Un, out, i0, j0, jend, cx, cy,
                                                                       ring_in, lane, smax, bad);
}

// One mesh: a 2D grid of (strips / STAGE_WARPS) x (row tiles) CTAs.
// Dynamic shared memory: STAGE_WARPS * Ring<T,CPL,NF>::warp_bytes(STAGE).
// Resident CTAs per SM requested from the register allocator: FP32 stages are
// issue-bound and gain from more warps (predictor 18 CTAs -> 92 registers,
// corrector 16 -> 114, no spills); with species the march carries more
// fields and gets more registers per thread; FP64 is bound by its arithmetic
// pipe and keeps the registers it wants.
#ifndef LF_MIN_BLOCKS_SPECIES0
#define LF_MIN_BLOCKS_SPECIES0 12
#endif
#ifndef LF_MIN_BLOCKS_SPECIES1
#define LF_MIN_BLOCKS_SPECIES1 10
#endif
template <typename T, int STAGE, int NF> struct MinBlocks {
  static constexpr int value = NF == 4 ? (STAGE == 0 ? LF_MIN_BLOCKS0 : LF_MIN_BLOCKS1)
                                       : (STAGE == 0 ? LF_MIN_BLOCKS_SPECIES0 : LF_MIN_BLOCKS_SPECIES1);
};
template <int STAGE, int NF> struct MinBlocks<double, STAGE, NF> { static constexpr int value = 1; };

template <typename T, int LIM, int STAGE, int CPL, int TY, int NF>
__global__ void __launch_bounds__(STAGE_WARPS * 32, (MinBlocks<T, STAGE, NF>::value))
stage2d_kernel(const MeshDesc m, const T* __restrict__ Uin, const T* Un, T* out, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char lf_stage_smem[];
  const double dtd = sc->dt;
  if (!(dtd > 0.0)) return;
  const int wpar = sc->parity ^ 1;
  using V = typename StageShape<T>::V;
  const Phys<V> P(m);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (blockIdx.x * STAGE_WARPS + warp) * StripGeom<CPL>::OUT;
  if (i0 >= m.nx) return;  // whole warp
  const int ty = m.ty > 0 ? m.ty : TY;
  const int j0 = blockIdx.y * ty;
  const int jend = min(j0 + ty, m.ny);
  const double hs = StageCoef<STAGE>::beta;
  const T cx = T(hs * dtd * m.rdx), cy = T(hs * dtd * m.rdy);
  T* ring = reinterpret_cast<T*>(lf_stage_smem + warp * Ring<T, CPL, NF>::warp_bytes(STAGE));
  T smax = T(0);
  bool bad = false;
  strip_tile<T, V, LIM, STAGE, CPL, NF>(P, m, Uin, Un, out, i0, j0, jend, cx, cy, ring, lane, smax, bad);
  if (StageCoef<STAGE>::speed) publish_speed(sc, wpar, smax, bad);
}

// 1D: one row, no y-terms.
template <typename T, int LIM, int STAGE, int CPL, int NF>
__global__ void __launch_bounds__(STAGE_WARPS * 32)
stage1d_kernel(const MeshDesc m, const T* __restrict__ Uin, const T* Un, T* out, Scalars* sc) {
  using V = typename StageShape<T>::V;
  const double dtd = sc->dt;
  if (!(dtd > 0.0)) return;
  const int wpar = sc->parity ^ 1;
  const Phys<V> P(m);
  const int lane = threadIdx.x & 31;
  const int i0 = (blockIdx.x * STAGE_WARPS + (threadIdx.x >> 5)) * StripGeom<CPL>::OUT;
  if (i0 >= m.nx) return;
  const LaneCols<CPL> L = lane_cols<CPL>(i0, lane, m.nx, m.bc, m.vec);
  const V ncx = V(-T(StageCoef<STAGE>::beta * dtd * m.rdx));
  const T* Pp[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) Pp[k] = Uin + k * m.plane;
  V U[NF], q[NF], Fl[NF], Fr[NF];
  load_row<T, CPL, NF>(Pp, L, 0, U);
  to_prim<V, NF>(P, U, q);
  x_fluxes<V, LIM, NF>(P, q, Fl, Fr);
  V W[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    V base = U[k];
    if (STAGE >= 1) {
      T v[CPL];  // U^n at the lane's output cells (other cells: any finite value, never stored)
#pragma unroll
      for (int j = 0; j < CPL; ++j) v[j] = L.out[j] ? Un[k * m.plane + L.c0 + j] : T(0);
      V un;
      make_lane(v, un);
      base = STAGE == 1 ? splat<V>(0.5) * (un + U[k])
                        : fma_(splat<V>(StageCoef<STAGE>::alpha), un, splat<V>(StageCoef<STAGE>::beta) * U[k]);
    }
    W[k] = fma_(ncx, Fr[k] - Fl[k], base);
  }
  T smax = T(0);
  bool bad = false;
  typename LaneT<V>::M ok;
  V sp;
  if (StageCoef<STAGE>::speed) sp = cell_speed<V, 1>(P, W, ok);
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    if (!L.out[j]) continue;
#pragma unroll
    for (int k = 0; k < NF; ++k) out[k * m.plane + L.c0 + j] = get(W[k], j);
    if (StageCoef<STAGE>::speed) {
      smax = fmax(smax, get(sp, j));
      bad |= !get(ok, j);
    }
  }
  if (StageCoef<STAGE>::speed) publish_speed(sc, wpar, smax, bad);
}

template <typename T, int LIM, int NF>
cudaError_t launch_stage_lim(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                             cudaStream_t s) {
  constexpr int CPL = StageShape<T>::CPL, TY = StageShape<T>::TY;
  const int strips = (m.nx + StripGeom<CPL>::OUT - 1) / StripGeom<CPL>::OUT;
  dim3 block(STAGE_WARPS * 32);
  if (m.dim == 1) {
    dim3 grid((strips + STAGE_WARPS - 1) / STAGE_WARPS);
    switch (stage) {
      case 0: stage1d_kernel<T, LIM, 0, CPL, NF><<<grid, block, 0, s>>>(m, Uin, Un, out, sc); break;
      case 1: stage1d_kernel<T, LIM, 1, CPL, NF><<<grid, block, 0, s>>>(m, Uin, Un, out, sc); break;
      case 2: stage1d_kernel<T, LIM, 2, CPL, NF><<<grid, block, 0, s>>>(m, Uin, Un, out, sc); break;
      default: stage1d_kernel<T, LIM, 3, CPL, NF><<<grid, block, 0, s>>>(m, Uin, Un, out, sc);
    }
  } else {
    const int ty = m.ty > 0 ? m.ty : TY;
    dim3 grid((strips + STAGE_WARPS - 1) / STAGE_WARPS, (m.ny + ty - 1) / ty);
    const size_t smem = STAGE_WARPS * Ring<T, CPL, NF>::warp_bytes(stage);
    switch (stage) {
      case 0: stage2d_kernel<T, LIM, 0, CPL, TY, NF><<<grid, block, smem, s>>>(m, Uin, Un, out, sc); break;
      case 1: stage2d_kernel<T, LIM, 1, CPL, TY, NF><<<grid, block, smem, s>>>(m, Uin, Un, out, sc); break;
      case 2: stage2d_kernel<T, LIM, 2, CPL, TY, NF><<<grid, block, smem, s>>>(m, Uin, Un, out, sc); break;
      default: stage2d_kernel<T, LIM, 3, CPL, TY, NF><<<grid, block, smem, s>>>(m, Uin, Un, out, sc);
    }
  }
  return cudaGetLastError();
}

// Stage launch for meshes with NF fields per cell.
template <typename T, int NF>
cudaError_t launch_stage_nf(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                            cudaStream_t s) {
  switch (m.limiter) {
    case LIM_MINMOD: return launch_stage_lim<T, LIM_MINMOD, NF>(stage, m, Uin, Un, out, sc, s);
    case LIM_SWEBY: return launch_stage_lim<T, LIM_SWEBY, NF>(stage, m, Uin, Un, out, sc, s);
    default: return launch_stage_lim<T, LIM_VANLEER, NF>(stage, m, Uin, Un, out, sc, s);
  }
}

}  // namespace lf
