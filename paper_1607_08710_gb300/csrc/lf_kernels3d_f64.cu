// FP64 instantiation of the 3D stage and element-wise kernels.
#include "lf_aux3d.cuh"
#include "lf_stage3d.cuh"

namespace lf {

cudaError_t launch_stage3d(int stage, const Mesh3Desc& m, const double* Uin, const double* Un, double* out, Scalars* sc,
                           cudaStream_t s) {
  return launch_stage3d_impl<double>(stage, m, Uin, Un, out, sc, s);
}

cudaError_t launch_wave_speed3d(const Mesh3Desc& m, const double* U, Scalars* sc, cudaStream_t s) {
  wave_speed3d_kernel<double><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, sc);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons3d(const Mesh3Desc& m, const double* q, double* U, cudaStream_t s) {
  prim_to_cons3d_kernel<double><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, q, U);
  return cudaGetLastError();
}

cudaError_t launch_cons_to_prim3d(const Mesh3Desc& m, const double* U, double* q, cudaStream_t s) {
  cons_to_prim3d_kernel<double><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, q);
  return cudaGetLastError();
}

cudaError_t launch_species_to_cons3d(const Mesh3Desc& m, const double* y, double* U, cudaStream_t s) {
  species_to_cons3d_kernel<double><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, y, U);
  return cudaGetLastError();
}

cudaError_t launch_cons_to_species3d(const Mesh3Desc& m, const double* U, double* y, cudaStream_t s) {
  cons_to_species3d_kernel<double><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, y);
  return cudaGetLastError();
}

}  // namespace lf
