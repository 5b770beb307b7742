// FP32 kernel set (fields stored and updated in FP32; restriction sums as
// error-free FP32 pairs rounded once; conservation sums in FP64).
#include "amr_launch.cuh"
#include "amr_mlp_kernels.cuh"

namespace amr {
template struct Kernels<float>;
}
