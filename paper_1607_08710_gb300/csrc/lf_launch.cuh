// Host launchers of the per-precision kernels.  Included by one translation
// unit per precision, which instantiates them with LF_INSTANTIATE_LAUNCHERS.
#pragma once

#include "lf_adjoint.cuh"
#include "lf_aux.cuh"
#include "lf_batch_stage.cuh"
#include "lf_stage.cuh"

namespace lf {

inline int aux_blocks(long long n) {
  long long b = (n + AUX_THREADS - 1) / AUX_THREADS;
  if (b > 152 * 16) b = 152 * 16;
  return b < 1 ? 1 : (int)b;
}

template <typename T>
cudaError_t launch_stage(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out, Scalars* sc,
                         cudaStream_t s) {
  if (m.nspecies > 0) return launch_stage_species(stage, m, Uin, Un, out, sc, s);
  return launch_stage_nf<T, 4>(stage, m, Uin, Un, out, sc, s);
}

template <typename T>
cudaError_t launch_batch_stage(int stage, const BatchDesc& b, const T* Uin, const T* Un, T* out, Scalars* sc,
                               int* counter, cudaStream_t s) {
  return launch_batch_stage_impl<T>(stage, b, Uin, Un, out, sc, counter, s);
}

template <typename T>
int batch_blocks_per_sm(int stage, int limiter) {
  return batch_blocks_impl<T>(stage, limiter);
}

template <typename T>
cudaError_t launch_wave_speed(const MeshDesc& m, const T* U, Scalars* sc, cudaStream_t s) {
  const int nb = aux_blocks((long long)m.nx * m.ny);
  if (m.dim == 1) wave_speed_kernel<T, 1><<<nb, AUX_THREADS, 0, s>>>(m, U, sc);
  else wave_speed_kernel<T, 2><<<nb, AUX_THREADS, 0, s>>>(m, U, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prim_to_cons(const MeshDesc& m, const T* rho, const T* u, const T* v, const T* p,
                                long long, T* U, cudaStream_t s) {
  prim_to_cons_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, rho, u, v, p, U);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cons_to_prim(const MeshDesc& m, const T* U, T* rho, T* u, T* v, T* p, cudaStream_t s) {
  cons_to_prim_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, U, rho, u, v, p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_species_to_cons(const MeshDesc& m, const T* y, T* U, cudaStream_t s) {
  species_to_cons_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, y, U);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cons_to_species(const MeshDesc& m, const T* U, T* y, cudaStream_t s) {
  cons_to_species_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, U, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sums(const MeshDesc& m, const T* U, double* partials, int nblocks, double* out,
                        cudaStream_t s) {
  sums_partial_kernel<T, 4><<<nblocks, AUX_THREADS, 0, s>>>(m, U, 0, partials);
  // planes past the first four: species, or rho E and the species of a 3D state
  if (m.nspecies == 1) sums_partial_kernel<T, 1><<<nblocks, AUX_THREADS, 0, s>>>(m, U, 4, partials);
  else if (m.nspecies == 2) sums_partial_kernel<T, 2><<<nblocks, AUX_THREADS, 0, s>>>(m, U, 4, partials);
  else if (m.nspecies == 3) sums_partial_kernel<T, 3><<<nblocks, AUX_THREADS, 0, s>>>(m, U, 4, partials);
  static_assert(MAX_SPECIES == 2, "extra summed planes: nspecies <= 2, plus rho E in 3D");
  sums_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, 4 + m.nspecies, out);
  return cudaGetLastError();
}

template <typename T, int LIM>
cudaError_t launch_slope_tables_lim(const MeshDesc& m, const T* Q, T* tabx, T* taby, cudaStream_t s) {
  slope_table_kernel<T, LIM, 0><<<aux_blocks((long long)(m.nx + 2) * m.ny), AUX_THREADS, 0, s>>>(m, Q, tabx);
  slope_table_kernel<T, LIM, 1><<<aux_blocks((long long)(m.ny + 2) * m.nx), AUX_THREADS, 0, s>>>(m, Q, taby);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_prep(const MeshDesc& m, const T* U, T* Q, T* tabx, T* taby, cudaStream_t s) {
  prim_planes_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, U, Q);
  switch (m.limiter) {
    case LIM_MINMOD: return launch_slope_tables_lim<T, LIM_MINMOD>(m, Q, tabx, taby, s);
    case LIM_SWEBY: return launch_slope_tables_lim<T, LIM_SWEBY>(m, Q, tabx, taby, s);
    default: return launch_slope_tables_lim<T, LIM_VANLEER>(m, Q, tabx, taby, s);
  }
}

template <typename T>
cudaError_t launch_face_vjp(const MeshDesc& m, int dir, const T* Q, const T* tab, const T* mu, T* Fq,
                            cudaStream_t s) {
  const long long nfaces = dir == 0 ? (long long)(m.nx + 1) * m.ny : (long long)(m.ny + 1) * m.nx;
  const int nb = aux_blocks(nfaces);
  if (dir == 0) face_vjp_kernel<T, 0><<<nb, AUX_THREADS, 0, s>>>(m, Q, tab, mu, Fq);
  else face_vjp_kernel<T, 1><<<nb, AUX_THREADS, 0, s>>>(m, Q, tab, mu, Fq);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cell_vjp(const MeshDesc& m, const T* Q, const T* Fx, const T* Fy, const T* tabx, const T* taby,
                            const T* X, double alpha, const T* Y, double beta, double c, T* out, cudaStream_t s) {
  cell_vjp_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, Q, Fx, Fy, tabx, taby, X, T(alpha),
                                                                               Y, T(beta), T(c), out);
  return cudaGetLastError();
}

template <typename T, int LIM>
cudaError_t launch_face_vjp_direct_lim(const MeshDesc& m, int dir, const T* U, const T* mu, T* Fq, cudaStream_t s) {
  const long long nfaces = dir == 0 ? (long long)(m.nx + 1) * m.ny : (long long)(m.ny + 1) * m.nx;
  const int nb = aux_blocks(nfaces);
  if (dir == 0) face_vjp_direct_kernel<T, LIM, 0><<<nb, AUX_THREADS, 0, s>>>(m, U, mu, Fq);
  else face_vjp_direct_kernel<T, LIM, 1><<<nb, AUX_THREADS, 0, s>>>(m, U, mu, Fq);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_face_vjp_direct(const MeshDesc& m, int dir, const T* U, const T* mu, T* Fq, cudaStream_t s) {
  switch (m.limiter) {
    case LIM_MINMOD: return launch_face_vjp_direct_lim<T, LIM_MINMOD>(m, dir, U, mu, Fq, s);
    case LIM_SWEBY: return launch_face_vjp_direct_lim<T, LIM_SWEBY>(m, dir, U, mu, Fq, s);
    default: return launch_face_vjp_direct_lim<T, LIM_VANLEER>(m, dir, U, mu, Fq, s);
  }
}

template <typename T>
cudaError_t launch_cell_vjp_direct(const MeshDesc& m, const T* U, const T* Fx, const T* Fy, const T* X, double alpha,
                                   const T* Y, double beta, double c, T* out, cudaStream_t s) {
  const int nb = aux_blocks((long long)m.nx * m.ny);
  switch (m.limiter) {
    case LIM_MINMOD:
      cell_vjp_direct_kernel<T, LIM_MINMOD><<<nb, AUX_THREADS, 0, s>>>(m, U, Fx, Fy, X, T(alpha), Y, T(beta), T(c), out);
      break;
    case LIM_SWEBY:
      cell_vjp_direct_kernel<T, LIM_SWEBY><<<nb, AUX_THREADS, 0, s>>>(m, U, Fx, Fy, X, T(alpha), Y, T(beta), T(c), out);
      break;
    default:
      cell_vjp_direct_kernel<T, LIM_VANLEER><<<nb, AUX_THREADS, 0, s>>>(m, U, Fx, Fy, X, T(alpha), Y, T(beta), T(c),
                                                                       out);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_prim(const MeshDesc& m, const T* U0, const T* lam, T* gq, cudaStream_t s) {
  grad_prim_kernel<T><<<aux_blocks((long long)m.nx * m.ny), AUX_THREADS, 0, s>>>(m, U0, lam, gq);
  return cudaGetLastError();
}

#define LF_INSTANTIATE_LAUNCHERS(T)                                                                    \
  template cudaError_t launch_stage<T>(int, const MeshDesc&, const T*, const T*, T*, Scalars*,         \
                                       cudaStream_t);                                                  \
  template cudaError_t launch_wave_speed<T>(const MeshDesc&, const T*, Scalars*, cudaStream_t);        \
  template cudaError_t launch_batch_stage<T>(int, const BatchDesc&, const T*, const T*, T*, Scalars*, int*,  \
                                             cudaStream_t);                                            \
  template int batch_blocks_per_sm<T>(int, int);                                                       \
  template cudaError_t launch_prim_to_cons<T>(const MeshDesc&, const T*, const T*, const T*, const T*, \
                                              long long, T*, cudaStream_t);                            \
  template cudaError_t launch_cons_to_prim<T>(const MeshDesc&, const T*, T*, T*, T*, T*, cudaStream_t); \
  template cudaError_t launch_sums<T>(const MeshDesc&, const T*, double*, int, double*, cudaStream_t);      \
  template cudaError_t launch_species_to_cons<T>(const MeshDesc&, const T*, T*, cudaStream_t);           \
  template cudaError_t launch_cons_to_species<T>(const MeshDesc&, const T*, T*, cudaStream_t);           \
  template cudaError_t launch_adjoint_prep<T>(const MeshDesc&, const T*, T*, T*, T*, cudaStream_t);           \
  template cudaError_t launch_face_vjp<T>(const MeshDesc&, int, const T*, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_cell_vjp<T>(const MeshDesc&, const T*, const T*, const T*, const T*, const T*,     \
                                          const T*, double, const T*, double, double, T*, cudaStream_t);         \
  template cudaError_t launch_face_vjp_direct<T>(const MeshDesc&, int, const T*, const T*, T*, cudaStream_t);    \
  template cudaError_t launch_cell_vjp_direct<T>(const MeshDesc&, const T*, const T*, const T*, const T*,        \
                                                 double, const T*, double, double, T*, cudaStream_t);            \
  template cudaError_t launch_grad_prim<T>(const MeshDesc&, const T*, const T*, T*, cudaStream_t);

}  // namespace lf
