// Batched Heun stages of the Lagrange-flux scheme (arXiv:1607.08710, Sec. 4)
// over many independent meshes of different sizes in one persistent launch
// per stage.  The per-strip march and its arithmetic are those of the
// single-mesh kernel (lf_stage.cuh).
#pragma once

#include "lf_stage.cuh"

namespace lf {

// March code shape of the batched kernel: 1 = one row body with a rotation
// of the register window, 0 = unrolled by three (as the single-mesh kernel),
// 2 = the inner march unrolled, the edge-strip march rotating.
// Persistent warps run unit prologues, inner and edge marches at the same
// time, so the smaller code matters more here than in the single-mesh grid.
#ifndef LF_BATCH_ROTATE
#define LF_BATCH_ROTATE 1
#endif
#ifndef LF_BATCH_MIN_BLOCKS
#define LF_BATCH_MIN_BLOCKS (16 / LF_STAGE_WARPS)
#endif
template <typename T> struct BatchMinBlocks { static constexpr int value = LF_BATCH_MIN_BLOCKS; };
template <> struct BatchMinBlocks<double> { static constexpr int value = 1; };

// Many meshes: a persistent grid whose warps pull work units (problem, strip,
// row tile) from an atomic counter until the list is exhausted.  Each problem
// uses its own dt, and its corrector units feed its own wave-speed maximum.
// (Gas dynamics only: NF = 4.)

template <typename T, int LIM, int STAGE, int CPL>
__global__ void __launch_bounds__(STAGE_WARPS * 32, (BatchMinBlocks<T>::value))
batch_stage_kernel(const BatchDesc b, const T* Uin, const T* Un, T* out, Scalars* sc, int* counter) {
  extern __shared__ __align__(16) unsigned char lf_stage_smem[];
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* ring = reinterpret_cast<T*>(lf_stage_smem + warp * Ring<T, CPL, 4>::warp_bytes(STAGE));
  // The counter's answer for the next unit is requested as soon as a unit
  // starts and read only when the next one starts, so the atomic's round
  // trip overlaps the current unit's march instead of stalling the warp.
  int next = lane == 0 ? atomicAdd(counter, 1) : 0;
  for (;;) {
    const int u = __shfl_sync(FULL, next, 0);
    if (u >= b.nunits) break;
    if (lane == 0) next = atomicAdd(counter, 1);
    const Unit un = b.units[u];
    const ProbDesc& pd = un.d;
    Scalars* scp = sc + un.p;
    const double dtd = scp->dt;
    if (!(dtd > 0.0)) continue;  // problem finished (t_end reached) or flagged
    MeshDesc m = b.common;
    m.nx = pd.nx;
    m.ny = pd.ny;
    m.pitch = pd.pitch;
    m.plane = pd.plane;
    m.rdx = pd.rdx;
    m.rdy = pd.rdy;
    using V = typename StageShape<T>::V;
    const Phys<V> P(m);
    const double hs = StageCoef<STAGE>::beta;
    const T cx = T(hs * dtd * m.rdx), cy = T(hs * dtd * m.rdy);
    T smax = T(0);
    bool bad = false;
    // The inner or the mapped march, as for one mesh.  (With both marches
    // unrolled by three and the units in mesh order, the alternating bodies
    // measured 18% slower than the mapped body alone, through instruction-cache
    // pressure; with the rotating marches, mesh order is the faster order.)
    strip_tile<T, V, LIM, STAGE, CPL, 4, LF_BATCH_ROTATE>(P, m, Uin + pd.off, Un + pd.off, out + pd.off, un.i0,
                                                               un.j0, un.jend, cx, cy, ring, lane, smax, bad);
    if (StageCoef<STAGE>::speed) publish_speed(scp, scp->parity ^ 1, smax, bad);
  }
}

template <typename T, int LIM>
cudaError_t launch_batch_stage_lim(int stage, const BatchDesc& b, const T* Uin, const T* Un, T* out, Scalars* sc,
                                   int* counter, cudaStream_t s) {
  constexpr int CPL = StageShape<T>::CPL;
  const size_t smem = STAGE_WARPS * Ring<T, CPL, 4>::warp_bytes(stage);
  if (stage == 0) batch_stage_kernel<T, LIM, 0, CPL><<<b.grid, STAGE_WARPS * 32, smem, s>>>(b, Uin, Un, out, sc, counter);
  else batch_stage_kernel<T, LIM, 1, CPL><<<b.grid, STAGE_WARPS * 32, smem, s>>>(b, Uin, Un, out, sc, counter);
  return cudaGetLastError();
}

template <typename T, int LIM>
int batch_blocks_lim(int stage) {
  constexpr int CPL = StageShape<T>::CPL;
  const size_t smem = STAGE_WARPS * Ring<T, CPL, 4>::warp_bytes(stage);
  int nb = 0;
  cudaError_t e = stage == 0
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<T, LIM, 0, CPL>, STAGE_WARPS * 32, smem)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<T, LIM, 1, CPL>, STAGE_WARPS * 32, smem);
  return e == cudaSuccess ? nb : 0;
}

template <typename T>
cudaError_t launch_batch_stage_impl(int stage, const BatchDesc& b, const T* Uin, const T* Un, T* out, Scalars* sc,
                                    int* counter, cudaStream_t s) {
  switch (b.common.limiter) {
    case LIM_MINMOD: return launch_batch_stage_lim<T, LIM_MINMOD>(stage, b, Uin, Un, out, sc, counter, s);
    case LIM_SWEBY: return launch_batch_stage_lim<T, LIM_SWEBY>(stage, b, Uin, Un, out, sc, counter, s);
    default: return launch_batch_stage_lim<T, LIM_VANLEER>(stage, b, Uin, Un, out, sc, counter, s);
  }
}

template <typename T>
int batch_blocks_impl(int stage, int limiter) {
  switch (limiter) {
    case LIM_MINMOD: return batch_blocks_lim<T, LIM_MINMOD>(stage);
    case LIM_SWEBY: return batch_blocks_lim<T, LIM_SWEBY>(stage);
    default: return batch_blocks_lim<T, LIM_VANLEER>(stage);
  }
}

}  // namespace lf
