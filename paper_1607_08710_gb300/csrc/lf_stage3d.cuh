// Fused stage of the three-dimensional Lagrange-flux step (arXiv:1607.08710,
// Sec. 4 with faces normal to x, y and z): primitive conversion, limited
// MUSCL slopes, face states, eqs. 13-14 and the upwind flux of eq. 12 on the
// six faces of every cell, and the Runge-Kutta update, in one pass.
//
// Work decomposition.  A CTA owns a strip of 32*CPL columns (x) of ROWS3
// consecutive rows (y), one warp per row, and marches along z over a tile of
// planes.  Each warp carries its own row's z-stencil in registers (primitives
// of three planes, z-slopes and the flux through the face below, in three
// slots), like the y-march of the 2D kernel, but with one plane body and a
// rotation of the slots after each plane (the kernel is large enough that
// the three-fold unrolled body stalled on instruction fetch);
// x-neighbours come by warp shuffles.  The y-stencil needs the neighbouring
// rows: every plane, the warps publish their row's primitives in a shared
// plane buffer (with the two halo rows on each side converted by four of the
// warps), and after a CTA barrier each warp reads the five rows around its own
// to form the slopes and the two y-faces of its cells.  A y-face shared by two
// warps is computed by both from the same operands in the same order, so the
// two copies are bitwise equal and the update stays conservative.
//
// Memory.  The CTA's own input rows (all fields) are staged into a shared
// ring four planes deep by cp.async, each warp copying its own row; the four
// halo rows, copied by warps 0-3, into a ring two planes deep (they are read
// only at their own plane); the U^n rows of the later stages into a
// two-plane ring.  CTAs whose strip lies inside the rows make these copies in
// one CTA-uniform branch, one vector copy per field and row.  One commit
// group per plane: at the top of a step the group issued one step earlier is
// complete.  Every lane reads back only the ring cells it copied, so its own
// cp.async wait is the only synchronisation the rings need; the warps
// exchange data only through the primitive plane buffer, which alternates
// between two buffers from plane to plane, so one barrier per plane (after
// the buffer is written) suffices.  The planes per z-tile are a launch
// parameter (Mesh3Desc::tz).
// Every global index is mapped into the mesh by the boundary condition, and
// only output cells (column < nx, row < ny, plane < nz) are stored.
#pragma once

#include <atomic>

#include "lf_device3d.cuh"
#include "lf_internal3d.h"
#include "lf_stage.cuh"

namespace lf {

#ifndef LF_3D_ROWS
#define LF_3D_ROWS 4
#endif
#ifndef LF_3D_TZ
#define LF_3D_TZ 64
#endif
#ifndef LF_3D_MIN_BLOCKS
#define LF_3D_MIN_BLOCKS 3
#endif
// z-march code shape: 0 = one plane body and a rotation of the register
// window after each plane (a third of the code; measured 6% faster, the
// unrolled kernel stalls on instruction fetch), 1 = unrolled by three with
// statically named slots.
#ifndef LF_3D_UNROLL3
#define LF_3D_UNROLL3 0
#endif
constexpr int ROWS3 = LF_3D_ROWS;  // output rows (warps) per CTA
constexpr int TZ3 = LF_3D_TZ;      // planes per z-tile
constexpr int HALO3 = 4;           // y-halo rows, two on each side
constexpr int RING3 = 4;           // own input rows: planes staged (k .. k+3 at step k)
constexpr int HRING3 = 2;          // halo input rows: planes staged (k, k+1 at step k)
constexpr int RUN3 = 2;            // U^n planes staged (k, k+1 at step k)
static_assert(ROWS3 >= HALO3, "the halo rows are converted by the first four warps");

template <typename T, int CPL, int NF> struct Smem3 {
  static constexpr int COLS = 32 * CPL;
  static constexpr int ROWSEG = NF * COLS;                   // one row: [field][column]
  static constexpr int PLANE_OWN = ROWS3 * ROWSEG;           // the CTA's rows j0 .. j0+ROWS3-1
  static constexpr int PLANE_HALO = HALO3 * ROWSEG;          // rows j0-2, j0-1, j0+ROWS3, j0+ROWS3+1
  static constexpr int PLANE_IN = (ROWS3 + HALO3) * ROWSEG;  // primitives of rows j0-2 .. j0+ROWS3+1
  static constexpr int PLANE_UN = ROWS3 * ROWSEG;            // rows j0 .. j0+ROWS3-1
  // the own-row ring, the halo-row ring, two primitive plane buffers
  // (planes alternate between them) and the U^n ring
  static __host__ __device__ constexpr size_t bytes(int stage) {
    return sizeof(T) * ((size_t)RING3 * PLANE_OWN + (size_t)HRING3 * PLANE_HALO + 2 * (size_t)PLANE_IN +
                        (stage ? (size_t)RUN3 * PLANE_UN : 0));
  }
};

// x-face fluxes of a row (as x_fluxes, with the 3D field order).
template <typename V, int LIM, int NF>
__device__ __forceinline__ void x_fluxes3(const Phys<V>& P, const V q[NF], V Fl[NF], V Fr[NF]) {
  V qL[NF], qR[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const V h = limiter_half<V, LIM>(q[k] - prev_cell(q[k]), next_cell(q[k]) - q[k], P.beta);
    qL[k] = q[k] + h;
    qR[k] = next_cell(q[k] - h);
  }
  lagrange_flux3<V, 0, NF>(P, qL, qR, Fr);
#pragma unroll
  for (int k = 0; k < NF; ++k) Fl[k] = prev_cell(Fr[k]);
}

template <typename T, int CPL, int NF, typename V>
__device__ __forceinline__ void read_seg(const T* seg, int lane, V out[NF]) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T v[CPL];
    VecLoad<T, CPL>::load_plain(seg + f * 32 * CPL + CPL * lane, v);
    make_lane(v, out[f]);
  }
}

template <typename T, int CPL, int NF, typename V>
__device__ __forceinline__ void write_seg(T* seg, int lane, const V in[NF]) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T v[CPL];
    split_lane(in[f], v);
    VecLoad<T, CPL>::store(seg + f * 32 * CPL + CPL * lane, v);
  }
}

template <typename T, int CPL>
__device__ __forceinline__ void copy_cells(T* dst, const T* src_row, const LaneCols<CPL>& L) {
  if (L.vec_ok) {
    cp_async<CPL * sizeof(T)>(dst, src_row + L.c0);
  } else {
#pragma unroll
    for (int j = 0; j < CPL; ++j) cp_async<sizeof(T)>(dst + j, src_row + L.ic[j]);
  }
}

template <typename T, int STAGE, int NF>
struct Args3 {
  const T* Uin;
  const T* Un;
  T* out;
  T* ring;   // RING3 planes of the CTA's own input rows (plane k in slot (k - k0) & 3)
  T* hring;  // HRING3 planes of the halo input rows (plane k in slot k & 1)
  T* P;      // primitives of a plane, all CTA rows: two buffers, plane k in buffer k & 1
  T* unr;   // RUN3 U^n planes
  int j0, k0, kend;
  long long own_off;   // element offset of this warp's (mapped) row in a plane of rows
  long long halo_off;  // the same for the halo row this warp copies (warps 0-3)
  int halo_rr;         // that halo row's index in the CTA's rows (-1: none)
  bool inner;          // the strip lies inside the rows: one vector copy per lane and row (CTA-uniform)
};

// This warp's copies of its own row of input plane `k` into the own-row
// ring, all fields, each lane copying its own CPL cells.
// AHEAD: k >= 0 (the march's prefetch; the prologue also asks for k0-2, k0-1).
template <typename T, int STAGE, int CPL, int NF, bool AHEAD = false>
__device__ __forceinline__ void issue_plane3(const Mesh3Desc& m, const Args3<T, STAGE, NF>& A, const LaneCols<CPL>& L,
                                             int k, int warp, int lane) {
  using SM = Smem3<T, CPL, NF>;
  const int kz = AHEAD ? map_row_ahead(k, m.nz, m.bc) : map_row(k, m.nz, m.bc);
  const long long zoff = (long long)kz * m.ny * m.pitch;
  T* slot = A.ring + ((k - A.k0 + 4) & 3) * SM::PLANE_OWN + warp * SM::ROWSEG + CPL * lane;
  const T* src = A.Uin + zoff + A.own_off;
  if (A.inner) {  // a uniform branch around all copies of the row
#pragma unroll
    for (int f = 0; f < NF; ++f) cp_async<CPL * sizeof(T)>(slot + f * 32 * CPL, src + f * m.plane + L.c0);
    return;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) copy_cells<T, CPL>(slot + f * 32 * CPL, src + f * m.plane, L);
}

// Warps 0-3: the copies of one halo row of input plane `k` into the
// halo-row ring (slot k & 1, row index = warp).  The halo rows are used only
// at their own plane, so they are staged one plane ahead, not three.
template <typename T, int STAGE, int CPL, int NF, bool AHEAD = false>
__device__ __forceinline__ void issue_halo3(const Mesh3Desc& m, const Args3<T, STAGE, NF>& A, const LaneCols<CPL>& L,
                                            int k, int warp, int lane) {
  using SM = Smem3<T, CPL, NF>;
  if (A.halo_rr < 0) return;  // uniform over the warp
  const int kz = AHEAD ? map_row_ahead(k, m.nz, m.bc) : map_row(k, m.nz, m.bc);
  const long long zoff = (long long)kz * m.ny * m.pitch;
  T* slot = A.hring + (k & 1) * SM::PLANE_HALO + warp * SM::ROWSEG + CPL * lane;
  const T* hsrc = A.Uin + zoff + A.halo_off;
  if (A.inner) {
#pragma unroll
    for (int f = 0; f < NF; ++f) cp_async<CPL * sizeof(T)>(slot + f * 32 * CPL, hsrc + f * m.plane + L.c0);
    return;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) copy_cells<T, CPL>(slot + f * 32 * CPL, hsrc + f * m.plane, L);
}

// U^n of this warp's own row at plane k (output cells only; plane clamped).
template <typename T, int STAGE, int CPL, int NF>
__device__ __forceinline__ void issue_un3(const Mesh3Desc& m, const Args3<T, STAGE, NF>& A, const LaneCols<CPL>& L,
                                          int k, int warp, int lane, int jrow) {
  using SM = Smem3<T, CPL, NF>;
  if (STAGE == 0 || jrow >= m.ny) return;  // uniform over the warp
  const int zc = min(k, m.nz - 1);
  T* seg = A.unr + ((k - A.k0) & 1) * SM::PLANE_UN + warp * SM::ROWSEG;
  const T* row = A.Un + ((long long)zc * m.ny + jrow) * m.pitch + L.c0;
  if (A.inner) {  // halo lanes copy their in-row cells too (never read)
#pragma unroll
    for (int f = 0; f < NF; ++f) cp_async<CPL * sizeof(T)>(seg + f * 32 * CPL + CPL * lane, row + f * m.plane);
    return;
  }
  if (!L.any_out) return;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T* src = row + f * m.plane;
    T* dst = seg + f * 32 * CPL + CPL * lane;
    if (L.vec_ok) {
      cp_async<CPL * sizeof(T)>(dst, src);
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j)
        if (L.out[j]) cp_async<sizeof(T)>(dst + j, src + j);
    }
  }
}

template <typename V, int NF> struct March3 {
  V q[3][NF];  // primitives of planes k, k+1, k+2 (own row)
  V s[3][NF];  // half z-slopes
  V G[3][NF];  // G[slot(k)] = flux through face k-1/2
};

// One plane of the march.  S = register slot of plane k.
template <typename T, typename V, int LIM, int STAGE, int CPL, int NF, int S>
__device__ __forceinline__ void march_plane3(const Phys<V>& P, const Mesh3Desc& m, const Args3<T, STAGE, NF>& A,
                                             const LaneCols<CPL>& L, March3<V, NF>& M, int warp, int lane, int k,
                                             int jrow, V ncx, V ncy, V ncz, V rdz, T& smax, bool& bad) {
  using SM = Smem3<T, CPL, NF>;
  constexpr int S1 = (S + 1) % 3, S2 = (S + 2) % 3;
  // The group issued one step ago (input plane k+2, U^n plane k) has landed.
  // Every lane reads back only the ring cells it copied itself, so its own
  // wait suffices there; the one cross-warp exchange, the primitive plane
  // buffer, alternates between two buffers, so this plane's writes cannot
  // meet the previous plane's reads (all of them precede the barrier below
  // in the previous step).
  cp_wait_all();
  T* const Pk = A.P + (k & 1) * SM::PLANE_IN;
  const T* own_k = A.ring + ((k - A.k0 + 4) & 3) * SM::PLANE_OWN + warp * SM::ROWSEG;  // this row, plane k
  {
    V Ut[NF];
    read_seg<T, CPL, NF>(A.ring + ((k + 2 - A.k0 + 4) & 3) * SM::PLANE_OWN + warp * SM::ROWSEG, lane, Ut);
    to_prim3<V, NF>(P, Ut, M.q[S2]);
  }
  // publish this row's primitives of plane k; warps 0-3 convert the halo rows
  write_seg<T, CPL, NF>(Pk + (warp + 2) * SM::ROWSEG, lane, M.q[S]);
  if (A.halo_rr >= 0) {
    const int rr = A.halo_rr;
    V Uh[NF], qh[NF];
    read_seg<T, CPL, NF>(A.hring + (k & 1) * SM::PLANE_HALO + warp * SM::ROWSEG, lane, Uh);
    to_prim3<V, NF>(P, Uh, qh);
    write_seg<T, CPL, NF>(Pk + rr * SM::ROWSEG, lane, qh);
  }
  // next copies: own input row of plane k+3 (into plane k-1's slot), halo
  // row of plane k+1 (into plane k-1's halo slot), U^n plane k+1
  issue_plane3<T, STAGE, CPL, NF, true>(m, A, L, k + 3, warp, lane);
  issue_halo3<T, STAGE, CPL, NF, true>(m, A, L, k + 1, warp, lane);
  issue_un3<T, STAGE, CPL, NF>(m, A, L, k + 1, warp, lane, jrow);
  cp_commit();
  __syncthreads();

  // z: slopes of plane k+1 and the flux through face k+1/2
  {
    V Lq[NF], Rq[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      M.s[S1][f] = limiter_half<V, LIM>(M.q[S1][f] - M.q[S][f], M.q[S2][f] - M.q[S1][f], P.beta);
      Lq[f] = M.q[S][f] + M.s[S][f];
      Rq[f] = M.q[S1][f] - M.s[S1][f];
    }
    lagrange_flux3<V, 2, NF>(P, Lq, Rq, M.G[S1]);
  }
  // base of the update, then the x-, y- and z-flux differences
  V W[NF];
  {
    V U[NF];
    read_seg<T, CPL, NF>(own_k, lane, U);
    if (STAGE >= 1) {
      V Un[NF];
      read_seg<T, CPL, NF>(A.unr + ((k - A.k0) & 1) * SM::PLANE_UN + warp * SM::ROWSEG, lane, Un);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        W[f] = STAGE == 1 ? splat<V>(0.5) * (Un[f] + U[f])
                          : fma_(splat<V>(StageCoef<STAGE>::alpha), Un[f], splat<V>(StageCoef<STAGE>::beta) * U[f]);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) W[f] = U[f];
    }
  }
  {
    V Fl[NF], Fr[NF];
    x_fluxes3<V, LIM, NF>(P, M.q[S], Fl, Fr);
#pragma unroll
    for (int f = 0; f < NF; ++f) W[f] = fma_(ncx, Fr[f] - Fl[f], W[f]);
  }
  {
    // y: rows j-2 .. j+2 of plane k; slopes at j-1, j, j+1; faces j-1/2, j+1/2
    const T* P0 = Pk + warp * SM::ROWSEG;  // row j-2
    V Lq[NF], Rq[NF], sj[NF], Glo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T v[CPL];
      V a, b, d;
      VecLoad<T, CPL>::load_plain(P0 + f * 32 * CPL + CPL * lane, v);
      make_lane(v, a);
      VecLoad<T, CPL>::load_plain(P0 + SM::ROWSEG + f * 32 * CPL + CPL * lane, v);
      make_lane(v, b);
      VecLoad<T, CPL>::load_plain(P0 + 3 * SM::ROWSEG + f * 32 * CPL + CPL * lane, v);
      make_lane(v, d);
      const V c = M.q[S][f];
      const V sm = limiter_half<V, LIM>(b - a, c - b, P.beta);
      sj[f] = limiter_half<V, LIM>(c - b, d - c, P.beta);
      Lq[f] = b + sm;
      Rq[f] = c - sj[f];
    }
    lagrange_flux3<V, 1, NF>(P, Lq, Rq, Glo);
    V Ghi[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T v[CPL];
      V d, e;
      VecLoad<T, CPL>::load_plain(P0 + 3 * SM::ROWSEG + f * 32 * CPL + CPL * lane, v);
      make_lane(v, d);
      VecLoad<T, CPL>::load_plain(P0 + 4 * SM::ROWSEG + f * 32 * CPL + CPL * lane, v);
      make_lane(v, e);
      const V c = M.q[S][f];
      const V sp = limiter_half<V, LIM>(d - c, e - d, P.beta);
      Lq[f] = c + sj[f];
      Rq[f] = d - sp;
    }
    lagrange_flux3<V, 1, NF>(P, Lq, Rq, Ghi);
#pragma unroll
    for (int f = 0; f < NF; ++f) W[f] = fma_(ncy, Ghi[f] - Glo[f], W[f]);
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) W[f] = fma_(ncz, M.G[S1][f] - M.G[S][f], W[f]);

  if (jrow < m.ny && k < A.kend) {
    T* dst = A.out + ((long long)k * m.ny + jrow) * m.pitch;
    if (L.vec_ok && L.any_out) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T v[CPL];
        split_lane(W[f], v);
        VecLoad<T, CPL>::store(dst + f * m.plane + L.c0, v);
      }
    } else if (!L.vec_ok) {
#pragma unroll
      for (int j = 0; j < CPL; ++j)
        if (L.out[j])
#pragma unroll
          for (int f = 0; f < NF; ++f) dst[f * m.plane + L.c0 + j] = get(W[f], j);
    }
    if (StageCoef<STAGE>::speed) {
      typename LaneT<V>::M ok;
      const V sp = cell_speed3<V>(P, rdz, W, ok);
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        smax = L.out[j] ? fmax(smax, get(sp, j)) : smax;
        bad |= L.out[j] && !get(ok, j);
      }
    }
  }
}

// FP32 gas dynamics: LF_3D_MIN_BLOCKS resident CTAs (LF_3D_MIN_BLOCKS0 for
// the first stage, whose smaller shared-memory footprint leaves room for
// more); with species the window carries more fields and the allocator is
// asked for two; FP64 is uncapped.
#ifndef LF_3D_MIN_BLOCKS0
#define LF_3D_MIN_BLOCKS0 LF_3D_MIN_BLOCKS
#endif
template <typename T, int STAGE, int NF> struct MinBlocks3 {
  static constexpr int value = NF == 5 ? (STAGE == 0 ? LF_3D_MIN_BLOCKS0 : LF_3D_MIN_BLOCKS) : 2;
};
template <int STAGE, int NF> struct MinBlocks3<double, STAGE, NF> { static constexpr int value = 1; };

// Grid: (strips, ceil(ny / ROWS3), ceil(nz / tz)), tz = m.tz or TZ3; ROWS3 warps per CTA.
template <typename T, int LIM, int STAGE, int NF>
__global__ void __launch_bounds__(ROWS3 * 32, (MinBlocks3<T, STAGE, NF>::value))
stage3d_kernel(const Mesh3Desc m, const T* __restrict__ Uin, const T* Un, T* out, Scalars* sc) {
  using V = typename StageShape<T>::V;
  constexpr int CPL = StageShape<T>::CPL;
  using SM = Smem3<T, CPL, NF>;
  extern __shared__ __align__(16) unsigned char lf_stage3_smem[];
  const double dtd = sc->dt;
  if (!(dtd > 0.0)) return;  // uniform over the grid
  const int wpar = sc->parity ^ 1;
  const Phys<V> P(mesh_view(m, 0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * StripGeom<CPL>::OUT;
  const int j0 = blockIdx.y * ROWS3;
  const int jrow = j0 + warp;  // rows past the mesh (no output) still take part in the copies and barriers
  Args3<T, STAGE, NF> A;
  A.Uin = Uin;
  A.Un = Un;
  A.out = out;
  A.ring = reinterpret_cast<T*>(lf_stage3_smem);
  A.hring = A.ring + RING3 * SM::PLANE_OWN;
  A.P = A.hring + HRING3 * SM::PLANE_HALO;
  A.unr = A.P + 2 * SM::PLANE_IN;
  A.j0 = j0;
  const int tz = m.tz > 0 ? m.tz : TZ3;
  A.k0 = blockIdx.z * tz;
  A.kend = min(A.k0 + tz, m.nz);
  A.own_off = (long long)map_row(jrow, m.ny, m.bc) * m.pitch;
  A.halo_rr = warp < HALO3 ? (warp < 2 ? warp : ROWS3 + warp) : -1;
  A.halo_off = A.halo_rr >= 0 ? (long long)map_row(j0 - 2 + A.halo_rr, m.ny, m.bc) * m.pitch : 0;
  A.inner = i0 - 2 >= 0 && i0 - 2 + 32 * CPL <= m.nx;
  const LaneCols<CPL> L = lane_cols<CPL>(i0, lane, m.nx, m.bc, 1);
  const double hs = StageCoef<STAGE>::beta;
  const V ncx = V(-T(hs * dtd * m.rdx)), ncy = V(-T(hs * dtd * m.rdy)), ncz = V(-T(hs * dtd * m.rdz));
  const V rdz = V(T(m.rdz));
  const int k0 = A.k0;

  // Prologue: input planes k0-2 .. k0+1 and U^n plane k0; the register
  // window gets the primitives of planes k0-1 (slot 2), k0 (0), k0+1 (1),
  // the z-slopes of k0-1 and k0 and the flux through face k0-1/2.
  for (int k = k0 - 2; k <= k0 + 1; ++k) issue_plane3<T, STAGE, CPL, NF>(m, A, L, k, warp, lane);
  issue_halo3<T, STAGE, CPL, NF>(m, A, L, k0, warp, lane);
  issue_un3<T, STAGE, CPL, NF>(m, A, L, k0, warp, lane, jrow);
  cp_commit();
  cp_wait_all();
  __syncthreads();
  March3<V, NF> M;
  {
    V Ut[NF], qm2[NF];
    const int slot_of[4] = {-1, 2, 0, 1};  // register slots of planes k0-1 .. k0+1 (k0-2 goes to qm2)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      read_seg<T, CPL, NF>(A.ring + ((t - 2 + 4) & 3) * SM::PLANE_OWN + warp * SM::ROWSEG, lane, Ut);
      to_prim3<V, NF>(P, Ut, t == 0 ? qm2 : M.q[slot_of[t]]);
    }
    V Lq[NF], Rq[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      M.s[2][f] = limiter_half<V, LIM>(M.q[2][f] - qm2[f], M.q[0][f] - M.q[2][f], P.beta);
      M.s[0][f] = limiter_half<V, LIM>(M.q[0][f] - M.q[2][f], M.q[1][f] - M.q[0][f], P.beta);
      Lq[f] = M.q[2][f] + M.s[2][f];
      Rq[f] = M.q[0][f] - M.s[0][f];
    }
    lagrange_flux3<V, 2, NF>(P, Lq, Rq, M.G[0]);
  }
  __syncthreads();  // plane k0-2's slot is reused next
  issue_plane3<T, STAGE, CPL, NF>(m, A, L, k0 + 2, warp, lane);
  cp_commit();

  T smax = T(0);
  bool bad = false;
#if LF_3D_UNROLL3
  for (int k = k0;;) {
    march_plane3<T, V, LIM, STAGE, CPL, NF, 0>(P, m, A, L, M, warp, lane, k, jrow, ncx, ncy, ncz, rdz, smax, bad);
    if (++k >= A.kend) break;
    march_plane3<T, V, LIM, STAGE, CPL, NF, 1>(P, m, A, L, M, warp, lane, k, jrow, ncx, ncy, ncz, rdz, smax, bad);
    if (++k >= A.kend) break;
    march_plane3<T, V, LIM, STAGE, CPL, NF, 2>(P, m, A, L, M, warp, lane, k, jrow, ncx, ncy, ncz, rdz, smax, bad);
    if (++k >= A.kend) break;
  }
#else
  for (int k = k0; k < A.kend; ++k) {
    march_plane3<T, V, LIM, STAGE, CPL, NF, 0>(P, m, A, L, M, warp, lane, k, jrow, ncx, ncy, ncz, rdz, smax, bad);
#pragma unroll
    for (int f = 0; f < NF; ++f) {  // rotate the window: plane k+1 -> slot 0, k+2 -> slot 1
      M.q[0][f] = M.q[1][f];
      M.q[1][f] = M.q[2][f];
      M.s[0][f] = M.s[1][f];
      M.G[0][f] = M.G[1][f];
    }
  }
#endif
  cp_wait_all();
  if (StageCoef<STAGE>::speed) publish_speed(sc, wpar, smax, bad);
}

template <typename T, int LIM, int NF>
cudaError_t launch_stage3d_lim(int stage, const Mesh3Desc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                               cudaStream_t s) {
  constexpr int CPL = StageShape<T>::CPL;
  using SM = Smem3<T, CPL, NF>;
  const int strips = (m.nx + StripGeom<CPL>::OUT - 1) / StripGeom<CPL>::OUT;
  const int tz = m.tz > 0 ? m.tz : TZ3;
  const dim3 grid(strips, (m.ny + ROWS3 - 1) / ROWS3, (m.nz + tz - 1) / tz);
  const dim3 block(ROWS3 * 32);
  const size_t smem = SM::bytes(stage);
  cudaError_t e = cudaSuccess;
  switch (stage) {
// The shared-memory opt-in is a per-device function attribute, set before the
// first launch on each device (setting it twice is harmless, so the flags
// only need to be atomic, not ordered).
#define LF_STAGE3_CASE(ST)                                                                                    \
  case ST: {                                                                                                  \
    static std::atomic<bool> opted[64];                                                                       \
    int dev = 0;                                                                                              \
    e = cudaGetDevice(&dev);                                                                                  \
    if (e == cudaSuccess && (dev >= 64 || !opted[dev].load(std::memory_order_relaxed))) {                     \
      e = cudaFuncSetAttribute(stage3d_kernel<T, LIM, ST, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                               (int)SM::bytes(ST));                                                           \
      if (e == cudaSuccess && dev < 64) opted[dev].store(true, std::memory_order_relaxed);                    \
    }                                                                                                         \
    if (e == cudaSuccess) stage3d_kernel<T, LIM, ST, NF><<<grid, block, smem, s>>>(m, Uin, Un, out, sc);      \
    break;                                                                                                    \
  }
    LF_STAGE3_CASE(0)
    LF_STAGE3_CASE(1)
    LF_STAGE3_CASE(2)
    default:
      LF_STAGE3_CASE(3)
#undef LF_STAGE3_CASE
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

template <typename T, int NF>
cudaError_t launch_stage3d_nf(int stage, const Mesh3Desc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                              cudaStream_t s) {
  switch (m.limiter) {
    case LIM_MINMOD: return launch_stage3d_lim<T, LIM_MINMOD, NF>(stage, m, Uin, Un, out, sc, s);
    case LIM_SWEBY: return launch_stage3d_lim<T, LIM_SWEBY, NF>(stage, m, Uin, Un, out, sc, s);
    default: return launch_stage3d_lim<T, LIM_VANLEER, NF>(stage, m, Uin, Un, out, sc, s);
  }
}

// nspecies transported mass fractions: 5 + nspecies fields per cell.
template <typename T>
cudaError_t launch_stage3d_impl(int stage, const Mesh3Desc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                                cudaStream_t s) {
  switch (m.nspecies) {
    case 0: return launch_stage3d_nf<T, 5>(stage, m, Uin, Un, out, sc, s);
    case 1: return launch_stage3d_nf<T, 6>(stage, m, Uin, Un, out, sc, s);
    case 2: return launch_stage3d_nf<T, 7>(stage, m, Uin, Un, out, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lf
