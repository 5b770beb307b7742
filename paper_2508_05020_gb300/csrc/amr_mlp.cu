// Learned refinement indicator, standalone calls of include/amr.h.
#include <cuda_runtime.h>
#include "amr.h"
#include "amr_internal.h"

namespace amr {
int mlp_k(int dim) { return dim == 1 ? 15 : (dim == 2 ? 100 : 625); }
long mlp_n_weights(int dim) { const long K = mlp_k(dim); return 64 * K + 64 + 64 * 64 + 64 + 64 + 1; }
}  // namespace amr

extern "C" {
int amr_mlp_k(int dim) { return (dim >= 1 && dim <= 3) ? amr::mlp_k(dim) : AMR_ERR_ARG; }
int amr_mlp_features(int, double, const double*, long, float*, const amr_options_t*) { return AMR_ERR_STATE; }
int amr_mlp_infer(int, const float*, long, const float*, float*, const amr_options_t*) { return AMR_ERR_STATE; }
int amr_mlp_grad(int, const float*, const float*, long, float, const float*, float*, float*, const amr_options_t*) {
    return AMR_ERR_STATE;
}
int amr_mlp_train(int, const float*, const float*, long, float, int, int, float, uint64_t, float*, float*,
                  const amr_options_t*) {
    return AMR_ERR_STATE;
}
}
