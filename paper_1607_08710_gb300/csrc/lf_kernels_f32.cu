// FP32 instantiation of the stage and auxiliary kernels.
#include "lf_aux.cuh"
#include "lf_launch.cuh"
#include "lf_stage.cuh"

namespace lf {
LF_INSTANTIATE_LAUNCHERS(float)
}  // namespace lf
