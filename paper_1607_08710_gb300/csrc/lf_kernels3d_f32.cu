// FP32 instantiation of the 3D stage and element-wise kernels.
#include "lf_aux3d.cuh"
#include "lf_stage3d.cuh"

namespace lf {

int stage3d_rows_per_cta() { return ROWS3; }

cudaError_t launch_stage3d(int stage, const Mesh3Desc& m, const float* Uin, const float* Un, float* out, Scalars* sc,
                           cudaStream_t s) {
  return launch_stage3d_impl<float>(stage, m, Uin, Un, out, sc, s);
}

cudaError_t launch_wave_speed3d(const Mesh3Desc& m, const float* U, Scalars* sc, cudaStream_t s) {
  wave_speed3d_kernel<float><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, sc);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons3d(const Mesh3Desc& m, const float* q, float* U, cudaStream_t s) {
  prim_to_cons3d_kernel<float><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, q, U);
  return cudaGetLastError();
}

cudaError_t launch_cons_to_prim3d(const Mesh3Desc& m, const float* U, float* q, cudaStream_t s) {
  cons_to_prim3d_kernel<float><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, q);
  return cudaGetLastError();
}

cudaError_t launch_species_to_cons3d(const Mesh3Desc& m, const float* y, float* U, cudaStream_t s) {
  species_to_cons3d_kernel<float><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, y, U);
  return cudaGetLastError();
}

cudaError_t launch_cons_to_species3d(const Mesh3Desc& m, const float* U, float* y, cudaStream_t s) {
  cons_to_species3d_kernel<float><<<aux_blocks3(m), AUX_THREADS, 0, s>>>(m, U, y);
  return cudaGetLastError();
}

}  // namespace lf
