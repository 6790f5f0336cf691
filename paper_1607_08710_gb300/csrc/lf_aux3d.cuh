// Element-wise kernels of the 3D path: the CFL wave-speed maximum of a state
// (Sec. 4, Heun step 1) and the primitive <-> conservative conversions (eq. 1
// with three velocity components).
#pragma once

#include "lf_aux.cuh"
#include "lf_device3d.cuh"
#include "lf_internal3d.h"

namespace lf {

template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
wave_speed3d_kernel(const Mesh3Desc m, const T* __restrict__ U, Scalars* sc) {
  const Phys<T> P(mesh_view(m, 0));
  const T rdz = T(m.rdz);
  const long long rows = (long long)m.ny * m.nz, n = rows * m.nx;
  T smax = T(0);
  bool bad = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / m.nx, i = k - r * m.nx;
    const long long idx = r * m.pitch + i;
    T Uc[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) Uc[l] = U[l * m.plane + idx];
    bool ok;
    smax = fmax(smax, cell_speed3<T>(P, rdz, Uc, ok));
    bad |= !ok;
  }
  constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(FULL, smax, o));
  const bool any_bad = __any_sync(FULL, bad);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_speed(&sc->smax[sc->parity], double(smax));
    if (any_bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
  }
}

// q: dense planes (rho, u, v, w, p, y_k), nx*ny*nz each; U: pitched state.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
prim_to_cons3d_kernel(const Mesh3Desc m, const T* q, T* U) {
  const T gm1 = T(m.gamma - 1.0);
  const long long rows = (long long)m.ny * m.nz, n = rows * m.nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / m.nx, i = k - r * m.nx;
    const long long idx = r * m.pitch + i;
    const T rho = q[k], u = q[n + k], v = q[2 * n + k], w = q[3 * n + k], p = q[4 * n + k];
    U[idx] = rho;
    U[m.plane + idx] = rho * u;
    U[2 * m.plane + idx] = rho * v;
    U[3 * m.plane + idx] = rho * w;
    U[4 * m.plane + idx] = p / gm1 + T(0.5) * rho * (u * u + v * v + w * w);
    for (int s = 0; s < m.nspecies; ++s) U[(5 + s) * m.plane + idx] = rho * q[(5 + s) * n + k];
  }
}

template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
cons_to_prim3d_kernel(const Mesh3Desc m, const T* U, T* q) {
  const T gm1 = T(m.gamma - 1.0);
  const long long rows = (long long)m.ny * m.nz, n = rows * m.nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / m.nx, i = k - r * m.nx;
    const long long idx = r * m.pitch + i;
    const T rho = U[idx], mx = U[m.plane + idx], my = U[2 * m.plane + idx], mz = U[3 * m.plane + idx];
    const T E = U[4 * m.plane + idx];
    const T u = mx / rho, v = my / rho, w = mz / rho;
    q[k] = rho;
    q[n + k] = u;
    q[2 * n + k] = v;
    q[3 * n + k] = w;
    q[4 * n + k] = gm1 * (E - T(0.5) * (mx * u + my * v + mz * w));
    for (int s = 0; s < m.nspecies; ++s) q[(5 + s) * n + k] = U[(5 + s) * m.plane + idx] / rho;
  }
}

// Species planes only: rho y_k = rho * y_k from dense fractions y, and back.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
species_to_cons3d_kernel(const Mesh3Desc m, const T* y, T* U) {
  const long long n = (long long)m.ny * m.nz * m.nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / m.nx, i = k - r * m.nx;
    const long long idx = r * m.pitch + i;
    const T rho = U[idx];
    for (int s = 0; s < m.nspecies; ++s) U[(5 + s) * m.plane + idx] = rho * y[s * n + k];
  }
}

template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
cons_to_species3d_kernel(const Mesh3Desc m, const T* U, T* y) {
  const long long n = (long long)m.ny * m.nz * m.nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / m.nx, i = k - r * m.nx;
    const long long idx = r * m.pitch + i;
    const T rho = U[idx];
    for (int s = 0; s < m.nspecies; ++s) y[s * n + k] = U[(5 + s) * m.plane + idx] / rho;
  }
}

inline int aux_blocks3(const Mesh3Desc& m) {
  long long b = ((long long)m.nx * m.ny * m.nz + AUX_THREADS - 1) / AUX_THREADS;
  if (b > 152 * 16) b = 152 * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace lf
