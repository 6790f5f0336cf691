// Small kernels around the fused stage: the CFL wave-speed reduction of a
// state (Sec. 4, Heun step 1), conversions between primitive and
// conservative variables (eq. 1), and compensated conservation sums.
#pragma once

#include "lf_device.cuh"

namespace lf {

constexpr int AUX_THREADS = 256;
constexpr int SUMS_BLOCKS = 1216;  // 8 x 152 SMs

template <typename T, int DIM>
__global__ void __launch_bounds__(AUX_THREADS)
wave_speed_kernel(const MeshDesc m, const T* __restrict__ U, Scalars* sc) {
  const Phys<T> P(m);
  const long long n = (long long)m.nx * m.ny;
  T smax = T(0);
  bool bad = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
    T Uc[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) Uc[l] = U[l * m.plane + idx];
    bool ok;
    smax = fmax(smax, cell_speed<T, DIM>(P, Uc, ok));
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

// src planes are dense (nx*ny, x fastest, stride src_plane between planes);
// U is the pitched internal layout.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
prim_to_cons_kernel(const MeshDesc m, const T* rho, const T* u, const T* v, const T* p, T* U) {
  const T gm1 = T(m.gamma - 1.0);
  const long long n = (long long)m.nx * m.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
    const T r = rho[k], uu = u[k], vv = v ? v[k] : T(0), pp = p[k];
    U[idx] = r;
    U[m.plane + idx] = r * uu;
    U[2 * m.plane + idx] = r * vv;
    U[3 * m.plane + idx] = pp / gm1 + T(0.5) * r * (uu * uu + vv * vv);
  }
}

template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
cons_to_prim_kernel(const MeshDesc m, const T* U, T* rho, T* u, T* v, T* p) {
  const T gm1 = T(m.gamma - 1.0);
  const long long n = (long long)m.nx * m.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
    const T r = U[idx], mx = U[m.plane + idx], my = U[2 * m.plane + idx], E = U[3 * m.plane + idx];
    const T uu = mx / r, vv = my / r;
    rho[k] = r;
    u[k] = uu;
    if (v) v[k] = vv;
    p[k] = gm1 * (E - T(0.5) * (mx * uu + my * vv));
  }
}

// Neumaier's compensated summation: the running sum s and the accumulated
// rounding error c, with s + c the compensated total.
struct KahanNeumaier {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
};

// Pass 1: every block sums a fixed, strided slice of the cells for NS fields
// starting at plane l0; the block's compensated partial for field l0 + l
// goes to partials[((l0 + l) * gridDim.x + block) * 2].
template <typename T, int NS>
__global__ void __launch_bounds__(AUX_THREADS)
sums_partial_kernel(const MeshDesc m, const T* __restrict__ U, int l0, double* partials) {
  __shared__ double sh_s[NS][AUX_THREADS];
  __shared__ double sh_c[NS][AUX_THREADS];
  KahanNeumaier acc[NS];
  const long long n = (long long)m.nx * m.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
#pragma unroll
    for (int l = 0; l < NS; ++l) acc[l].add(double(U[(l0 + l) * m.plane + idx]));
  }
#pragma unroll
  for (int l = 0; l < NS; ++l) {
    sh_s[l][threadIdx.x] = acc[l].s;
    sh_c[l][threadIdx.x] = acc[l].c;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    const int l = threadIdx.x;
    KahanNeumaier tot;
    for (int t = 0; t < AUX_THREADS; ++t) {
      tot.add(sh_s[l][t]);
      tot.add(sh_c[l][t]);
    }
    partials[((l0 + l) * gridDim.x + blockIdx.x) * 2] = tot.s;
    partials[((l0 + l) * gridDim.x + blockIdx.x) * 2 + 1] = tot.c;
  }
}

// Pass 2: one thread per field adds the block partials in block order.
__global__ void sums_final_kernel(const double* partials, int nblocks, int nfields, double* out);

// rho y_k = rho * y_k (y: dense planes, U: pitched state with its density set).
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
species_to_cons_kernel(const MeshDesc m, const T* y, T* U) {
  const long long n = (long long)m.nx * m.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
    const T r = U[idx];
    for (int s = 0; s < m.nspecies; ++s) U[(4 + s) * m.plane + idx] = r * y[s * n + k];
  }
}

// y_k = (rho y_k) / rho into dense planes.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS)
cons_to_species_kernel(const MeshDesc m, const T* U, T* y) {
  const long long n = (long long)m.nx * m.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / m.nx, i = k - j * m.nx;
    const long long idx = j * m.pitch + i;
    const T r = U[idx];
    for (int s = 0; s < m.nspecies; ++s) y[s * n + k] = U[(4 + s) * m.plane + idx] / r;
  }
}

}  // namespace lf
