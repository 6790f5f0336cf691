// FP64 stage kernels for meshes carrying transported mass fractions (Sec. 5):
// 4 + nspecies fields per cell, nspecies = 1 .. MAX_SPECIES.
#include "lf_stage.cuh"

namespace lf {
cudaError_t launch_stage_species(int stage, const MeshDesc& m, const double* Uin, const double* Un, double* out,
                                 Scalars* sc, cudaStream_t s) {
  switch (m.nspecies) {
    case 1: return launch_stage_nf<double, 5>(stage, m, Uin, Un, out, sc, s);
    case 2: return launch_stage_nf<double, 6>(stage, m, Uin, Un, out, sc, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace lf
