// Learned refinement indicator, AMR side: training-sample harvest from 1D
// runs, per-patch inference over the band [-1, N]^d of leaf patches, and the
// cell-level agreement counts against the plain sensor. Included by the two
// precision units after amr_launch.cuh.
#pragma once
#include "amr_launch.cuh"

namespace amr {

// 5-point (rho, u, p) samples of the band cells [-1, N] of every leaf patch of a
// 1D hierarchy, with the plain flag of the centre; sample slot (leaf, cell) is
// fixed, invalid (out-of-domain) slots get label 255.
template <typename T, int N>
__global__ void k_harvest(Grid g, const T* U, double* samples, unsigned char* labels) {
    const int npatch = g.counts[1];
    const double gm1 = g.gamma - 1.0;
    const long long total = (long long)npatch * (N + 2);
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(it / (N + 2));
        const int l = (int)(it - (long long)pi * (N + 2)) - 1;
        const int slot = g.leaf_list[pi];
        const int lev = g.level[slot];
        const int Gx = g.coord[slot * 3] * N + l;
        const bool indom = g.periodic[0] || (Gx >= 0 && Gx < g.ext[lev][0] * N);
        double r[5], u[5], p[5];
        for (int k = 0; k < 5; ++k) {
            const int sx = l - 2 + k + G;
            double Uc[3];
            for (int v = 0; v < 3; ++v) Uc[v] = (double)U[slot_index(g, slot, v, 0, 0, sx)];
            r[k] = Uc[0];
            u[k] = Uc[1] / Uc[0];
            p[k] = pressure_d<1>(Uc, gm1);
            samples[it * 15 + k * 3 + 0] = r[k];
            samples[it * 15 + k * 3 + 1] = u[k];
            samples[it * 15 + k * 3 + 2] = p[k];
        }
        const double sr = fabs(r[3] - r[1]) / (r[3] + 2.0 * r[2] + r[1]);
        const double sp = fabs(p[3] - p[1]) / (p[3] + 2.0 * p[2] + p[1]);
        labels[it] = indom ? ((sr > g.theta_rho || sp > g.theta_p) ? 1 : 0) : 255;
    }
}

template <typename T>
cudaError_t Kernels<T>::harvest(const Grid& g, const T* U, int* n_out, double* samples, unsigned char* labels,
                                int max_n, cudaStream_t s) {
    (void)n_out;
    (void)max_n;
    switch (g.dim * 100 + g.N) {
    case 108: k_harvest<T, 8><<<256, 256, 0, s>>>(g, U, samples, labels); break;
    case 116: k_harvest<T, 16><<<256, 256, 0, s>>>(g, U, samples, labels); break;
    case 132: k_harvest<T, 32><<<256, 256, 0, s>>>(g, U, samples, labels); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::flag_mlp(const Grid& g, const T* U, const float* w, int* anyflag, int grid,
                                 cudaStream_t s) {
    (void)g; (void)U; (void)w; (void)anyflag; (void)grid; (void)s;
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t Kernels<T>::flag_stats(const Grid& g, const T* U, const float* w, unsigned long long* counts,
                                   int grid, cudaStream_t s) {
    (void)g; (void)U; (void)w; (void)counts; (void)grid; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace amr
