// FP64 kernel set. Compiled with -fmad=false so that every multiply and add
// rounds separately, in the order the expressions are written.
#include "amr_launch.cuh"
#include "amr_mlp_kernels.cuh"

namespace amr {
template struct Kernels<double>;
}
