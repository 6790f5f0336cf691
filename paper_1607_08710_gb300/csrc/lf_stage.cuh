// Fused Heun stage of the Lagrange-flux scheme (arXiv:1607.08710, Sec. 4):
// per cell, primitive conversion (eq. 1), limited MUSCL slopes in x and y
// (eq. "sweby"), face states, the acoustic interface solve (eqs. 13-14), the
// upwind Lagrange flux (eq. 12) and the conservative update -- in one kernel
// per stage, with no face quantity ever written to memory.
//
// Work decomposition.  A warp owns a strip of 32 consecutive columns: lanes
// 2..29 produce output cells, lanes 0,1 and 30,31 are the two-cell halo the
// 5-point MUSCL stencil needs, so x-neighbours are exchanged with warp
// shuffles and nothing is staged in shared memory.  The warp marches up a
// tile of rows, carrying the y-stencil (three rows of primitives, two rows of
// y-slopes and the flux through the face below) in registers, so every
// primitive, slope and face flux is computed once per cell (up to the halo
// lanes and the two rows of y-halo at the bottom of a tile).  The next row is
// prefetched one iteration ahead to cover memory latency.
#pragma once

#include "lf_device.cuh"

namespace lf {

constexpr int STRIP_OUT = 28;   // output columns per warp
constexpr int STAGE_WARPS = 4;  // warps per CTA, side by side in x
constexpr int STAGE_TY = 64;    // rows per CTA tile in 2D

// Fluxes through the right (i+1/2) and left (i-1/2) x-faces of this lane's
// cell, from the primitive state q of the lane's column (valid on lanes 2..29).
template <typename T, int LIM>
__device__ __forceinline__ void x_fluxes(const Phys<T>& P, const T q[4], T Fp[4], T Fm[4]) {
  constexpr unsigned FULL = 0xffffffffu;
  T qplus[4], qright[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T qm = __shfl_up_sync(FULL, q[k], 1);
    const T qp = __shfl_down_sync(FULL, q[k], 1);
    const T s = limiter<T, LIM>(q[k] - qm, qp - q[k], P.beta);
    qplus[k] = q[k] + T(0.5) * s;            // left state of face i+1/2
    const T qminus = q[k] - T(0.5) * s;      // right state of face i-1/2
    qright[k] = __shfl_down_sync(FULL, qminus, 1);  // right state of face i+1/2
  }
  lagrange_flux<T, 0>(P, qplus, qright, Fp);
#pragma unroll
  for (int k = 0; k < 4; ++k) Fm[k] = __shfl_up_sync(FULL, Fp[k], 1);
}

template <typename T>
__device__ __forceinline__ void load_cell(const T* __restrict__ U, long long plane, long long idx, T out[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = __ldg(U + k * plane + idx);
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

// STAGE 0: out = Uin - dt L(Uin).  STAGE 1: out = (Un + Uin)/2 - dt/2 L(Uin).
template <typename T, int LIM, int STAGE>
__global__ void __launch_bounds__(STAGE_WARPS * 32)
stage2d_kernel(const MeshDesc m, const T* __restrict__ Uin, const T* Un, T* out, Scalars* sc) {
  const double dtd = sc->dt;
  if (!(dtd > 0.0)) return;
  const int wpar = sc->parity ^ 1;
  const Phys<T> P(m);
  const int lane = threadIdx.x & 31;
  const int i0 = (blockIdx.x * STAGE_WARPS + (threadIdx.x >> 5)) * STRIP_OUT;
  if (i0 >= m.nx) return;  // whole warp
  const int c = i0 - 2 + lane;
  const int ic = map_index(c, m.nx, m.bc);
  const bool writer = lane >= 2 && lane < 2 + STRIP_OUT && c < m.nx;
  const int j0 = blockIdx.y * STAGE_TY;
  const int jend = min(j0 + STAGE_TY, m.ny);
  const double hs = STAGE == 0 ? 1.0 : 0.5;
  const T cx = T(hs * dtd * m.rdx), cy = T(hs * dtd * m.rdy);
  const long long pl = m.plane;

  auto row_index = [&](int r) -> long long { return (long long)map_index(r, m.ny, m.bc) * m.pitch + ic; };

  // Prologue: rows j0-2 .. j0+1, the y-slopes of rows j0-1 and j0, and the
  // flux through face j0-1/2.
  T Ua[4], Ub[4], Uc[4], qa[4], qb[4], qc[4], sa[4], sb[4], Gm[4], Gp[4];
  {
    T Um2[4], Um1[4], qm2[4], qm1[4], sm1[4];
    load_cell(Uin, pl, row_index(j0 - 2), Um2);
    load_cell(Uin, pl, row_index(j0 - 1), Um1);
    load_cell(Uin, pl, row_index(j0), Ua);
    load_cell(Uin, pl, row_index(j0 + 1), Ub);
    to_prim(P, Um2, qm2);
    to_prim(P, Um1, qm1);
    to_prim(P, Ua, qa);
    to_prim(P, Ub, qb);
    T L[4], R[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sm1[k] = limiter<T, LIM>(qm1[k] - qm2[k], qa[k] - qm1[k], P.beta);
      sa[k] = limiter<T, LIM>(qa[k] - qm1[k], qb[k] - qa[k], P.beta);
      L[k] = qm1[k] + T(0.5) * sm1[k];
      R[k] = qa[k] - T(0.5) * sa[k];
    }
    lagrange_flux<T, 1>(P, L, R, Gm);
  }
  T Unext[4];
  load_cell(Uin, pl, row_index(j0 + 2), Unext);
  T Unold[4], Unold_next[4];
  if (STAGE == 1 && writer) {
    const long long idx = (long long)j0 * m.pitch + c;
#pragma unroll
    for (int k = 0; k < 4; ++k) Unold_next[k] = Un[k * pl + idx];
  }

  T smax = T(0);
  bool bad = false;
  for (int r = j0; r < jend; ++r) {
#pragma unroll
    for (int k = 0; k < 4; ++k) Uc[k] = Unext[k];
    if (r + 1 < jend) load_cell(Uin, pl, row_index(r + 3), Unext);
    if (STAGE == 1 && writer) {
#pragma unroll
      for (int k = 0; k < 4; ++k) Unold[k] = Unold_next[k];
      if (r + 1 < jend) {
        const long long idx = (long long)(r + 1) * m.pitch + c;
#pragma unroll
        for (int k = 0; k < 4; ++k) Unold_next[k] = Un[k * pl + idx];
      }
    }
    to_prim(P, Uc, qc);
    T L[4], R[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sb[k] = limiter<T, LIM>(qb[k] - qa[k], qc[k] - qb[k], P.beta);  // y-slope of row r+1
      L[k] = qa[k] + T(0.5) * sa[k];
      R[k] = qb[k] - T(0.5) * sb[k];
    }
    lagrange_flux<T, 1>(P, L, R, Gp);  // face r+1/2
    T Fp[4], Fm[4];
    x_fluxes<T, LIM>(P, qa, Fp, Fm);

    if (writer) {
      T Unew[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T base = STAGE == 0 ? Ua[k] : T(0.5) * (Unold[k] + Ua[k]);
        Unew[k] = base - cx * (Fp[k] - Fm[k]) - cy * (Gp[k] - Gm[k]);
      }
      const long long idx = (long long)r * m.pitch + c;
#pragma unroll
      for (int k = 0; k < 4; ++k) out[k * pl + idx] = Unew[k];
      if (STAGE == 1) {
        bool ok;
        smax = fmax(smax, cell_speed<T, 2>(P, Unew, ok));
        bad |= !ok;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Ua[k] = Ub[k];
      Ub[k] = Uc[k];
      qa[k] = qb[k];
      qb[k] = qc[k];
      sa[k] = sb[k];
      Gm[k] = Gp[k];
    }
  }
  if (STAGE == 1) publish_speed(sc, wpar, smax, bad);
}

template <typename T, int LIM, int STAGE>
__global__ void __launch_bounds__(STAGE_WARPS * 32)
stage1d_kernel(const MeshDesc m, const T* __restrict__ Uin, const T* Un, T* out, Scalars* sc) {
  const double dtd = sc->dt;
  if (!(dtd > 0.0)) return;
  const int wpar = sc->parity ^ 1;
  const Phys<T> P(m);
  const int lane = threadIdx.x & 31;
  const int i0 = (blockIdx.x * STAGE_WARPS + (threadIdx.x >> 5)) * STRIP_OUT;
  if (i0 >= m.nx) return;
  const int c = i0 - 2 + lane;
  const int ic = map_index(c, m.nx, m.bc);
  const bool writer = lane >= 2 && lane < 2 + STRIP_OUT && c < m.nx;
  const T cx = T((STAGE == 0 ? 1.0 : 0.5) * dtd * m.rdx);
  const long long pl = m.plane;
  T U[4], q[4], Fp[4], Fm[4];
  load_cell(Uin, pl, ic, U);
  to_prim(P, U, q);
  x_fluxes<T, LIM>(P, q, Fp, Fm);
  T smax = T(0);
  bool bad = false;
  if (writer) {
    T Unew[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T base = STAGE == 0 ? U[k] : T(0.5) * (Un[k * pl + c] + U[k]);
      Unew[k] = base - cx * (Fp[k] - Fm[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k * pl + c] = Unew[k];
    if (STAGE == 1) {
      bool ok;
      smax = cell_speed<T, 1>(P, Unew, ok);
      bad = !ok;
    }
  }
  if (STAGE == 1) publish_speed(sc, wpar, smax, bad);
}

template <typename T, int LIM>
cudaError_t launch_stage_lim(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                             cudaStream_t s) {
  const int strips = (m.nx + STRIP_OUT - 1) / STRIP_OUT;
  dim3 block(STAGE_WARPS * 32);
  if (m.dim == 1) {
    dim3 grid((strips + STAGE_WARPS - 1) / STAGE_WARPS);
    if (stage == 0) stage1d_kernel<T, LIM, 0><<<grid, block, 0, s>>>(m, Uin, Un, out, sc);
    else stage1d_kernel<T, LIM, 1><<<grid, block, 0, s>>>(m, Uin, Un, out, sc);
  } else {
    dim3 grid((strips + STAGE_WARPS - 1) / STAGE_WARPS, (m.ny + STAGE_TY - 1) / STAGE_TY);
    if (stage == 0) stage2d_kernel<T, LIM, 0><<<grid, block, 0, s>>>(m, Uin, Un, out, sc);
    else stage2d_kernel<T, LIM, 1><<<grid, block, 0, s>>>(m, Uin, Un, out, sc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_impl(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                              cudaStream_t s) {
  switch (m.limiter) {
    case LIM_MINMOD: return launch_stage_lim<T, LIM_MINMOD>(stage, m, Uin, Un, out, sc, s);
    case LIM_SWEBY: return launch_stage_lim<T, LIM_SWEBY>(stage, m, Uin, Un, out, sc, s);
    default: return launch_stage_lim<T, LIM_VANLEER>(stage, m, Uin, Un, out, sc, s);
  }
}

}  // namespace lf
