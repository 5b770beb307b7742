// Learned refinement indicator, AMR side: training-sample harvest from 1D
// runs, per-patch inference over the band [-1, N]^d of leaf patches, and the
// cell-level agreement counts against the plain sensor. Included by the two
// precision units after amr_launch.cuh.
#pragma once
#include "amr_launch.cuh"
#include "amr_mlp_core.cuh"

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
        const bool fr = fabs(r[3] - r[1]) > g.theta_rho * (r[3] + 2.0 * r[2] + r[1]);
        const bool fp = fabs(p[3] - p[1]) > g.theta_p * (p[3] + 2.0 * p[2] + p[1]);
        labels[it] = indom ? ((fr || fp) ? 1 : 0) : 255;
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

// ---------------------------------------------------------------------------
// K10: learned indicator on the band [-1, N]^d of every leaf patch. One work
// item is a leaf patch (1D/2D) or a slab of DZ band planes of it (3D). The
// primitives (rho, u.., p) of the slab and its +-2 halo are staged in shared
// memory in FP32; each warp takes 16 band cells at a time and builds the
// normalised 5^d stencil features straight into the BF16 A fragments of the
// tensor-core MLP (mlp_tile). A patch is flagged if any in-domain band cell
// has a positive logit; slabs of an already flagged patch are skipped.
// With `stats`, the plain sensor of every band cell is evaluated too (FP64,
// as in k_flag_plain) and the agreement counts TP, FP, FN, TN accumulated.
// ---------------------------------------------------------------------------
template <int D, int N> struct MlpBand {
    static constexpr int B = N + 2;                       // band cells per dimension
    static constexpr int S = N + 2 * G;                   // slot cells per dimension
    static constexpr int DZ = D == 3 ? 2 : 1;
    static constexpr int NSLAB = D == 3 ? B / DZ : 1;
    static constexpr int PX = S, PY = D >= 2 ? S : 1, PZ = D == 3 ? DZ + 4 : 1;
    static constexpr int PLANE = PX * PY * PZ;            // floats per primitive field
    static constexpr int CELLS = D == 1 ? B : (D == 2 ? B * B : B * B * DZ);
    static constexpr int F = D + 2;
};

template <int D, int N>
constexpr size_t mlp_flag_smem() {
    using P = MlpBand<D, N>;
    return (sizeof(MlpSmem<D>) + 15) / 16 * 16 + sizeof(int) * mlp_kpad(D) + sizeof(float) * P::F * P::PLANE + 16;
}

template <typename T, int D, int N>
__device__ bool plain_flag_cell(const Grid& g, const T* U, int slot, const int* l) {
    constexpr int NV = D + 2;
    const T gm1 = T(g.gamma) - T(1);
    auto rho_p = [&](int dx, int dy, int dz, T& r, T& p) {
        T Uc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            Uc[v] = U[slot_index(g, slot, v, sc<D>(2, l[2] + dz), sc<D>(1, l[1] + dy), sc<D>(0, l[0] + dx))];
        T u[D], Tt;
        primitives<T, D>(Uc, gm1, r, u, p, Tt);
    };
    T r0, p0;
    rho_p(0, 0, 0, r0, p0);
    bool f = false;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int ex = d == 0, ey = d == 1, ez = d == 2;
        T rm, pm, rp, pp;
        rho_p(-ex, -ey, -ez, rm, pm);
        rho_p(ex, ey, ez, rp, pp);
        f = f || (fabs(rp - rm) > T(g.theta_rho) * (rp + T(2) * r0 + rm)) ||
            (fabs(pp - pm) > T(g.theta_p) * (pp + T(2) * p0 + pm));
    }
    return f;
}

template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_flag_mlp(Grid g, const T* __restrict__ U, const float* __restrict__ w,
                                                  int* anyflag, unsigned long long* stats) {
    using P = MlpBand<D, N>;
    constexpr int K = mlp_kin(D), KP = mlp_kpad(D), F = P::F;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem<D>& ms = *reinterpret_cast<MlpSmem<D>*>(smem_raw);
    int* koff = reinterpret_cast<int*>(smem_raw + (sizeof(MlpSmem<D>) + 15) / 16 * 16);
    float* prim = reinterpret_cast<float*>(koff + KP);
    __shared__ int skip;
    mlp_stage_weights<D>(ms, w);
    // feature k -> (field, offset of the stencil point relative to the centre cell)
    for (int k = threadIdx.x; k < KP; k += blockDim.x) {
        if (k >= K) { koff[k] = -1; continue; }
        const int j = k / F, f = k - j * F;
        const int ox = j % 5 - 2, oy = D >= 2 ? (j / 5) % 5 - 2 : 0, oz = D == 3 ? j / 25 - 2 : 0;
        const int kind = f == 0 ? 0 : (f == F - 1 ? 2 : 1);                   // rho, velocity, p
        koff[k] = (kind << 28) | (f * P::PLANE + (oz * P::PY + oy) * P::PX + ox + (1 << 20));
    }
    __syncthreads();
    const T gm1 = T(g.gamma) - T(1);
    const int npatch = g.counts[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int gq = lane >> 2;
    for (int item = blockIdx.x; item < npatch * P::NSLAB; item += gridDim.x) {
        const int pi = item / P::NSLAB, slab = item - pi * P::NSLAB;
        const int slot = g.leaf_list[pi];
        if (threadIdx.x == 0) skip = (!stats && *((volatile int*)&anyflag[slot])) ? 1 : 0;
        __syncthreads();
        if (skip) continue;
        const int lev = g.level[slot];
        const int c[3] = {g.coord[slot * 3], g.coord[slot * 3 + 1], g.coord[slot * 3 + 2]};
        const int zb0 = D == 3 ? slab * P::DZ - 1 : 0;            // first band plane (local z)
        // primitives of the slab and its halo: local z in [zb0 - 2, zb0 + DZ + 2)
        for (int idx = threadIdx.x; idx < P::PLANE; idx += blockDim.x) {
            const int px = idx % P::PX, py = (idx / P::PX) % P::PY, pz = idx / (P::PX * P::PY);
            const int sz = D == 3 ? zb0 - 2 + pz + G : 0;
            T Uc[D + 2];
#pragma unroll
            for (int v = 0; v < D + 2; ++v) Uc[v] = U[slot_index(g, slot, v, sz, py, px)];
            T rho, u[D], p, Tt;
            primitives<T, D>(Uc, gm1, rho, u, p, Tt);
            prim[idx] = (float)rho;
#pragma unroll
            for (int d = 0; d < D; ++d) prim[(1 + d) * P::PLANE + idx] = (float)u[d];
            prim[(F - 1) * P::PLANE + idx] = (float)p;
        }
        __syncthreads();
        constexpr int TILES = (P::CELLS + 15) / 16;
        for (int tile = warp; tile < TILES; tile += nw) {
            int cen[2], lc[2][3];
            bool valid[2];
            float ir[2], ic[2], ip[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = tile * 16 + gq + 8 * h;
                valid[h] = r < P::CELLS;
                const int rr = valid[h] ? r : P::CELLS - 1;
                const int bx = rr % P::B, by = D >= 2 ? (rr / P::B) % P::B : 0, bz = D == 3 ? rr / (P::B * P::B) : 0;
                lc[h][0] = bx - 1;
                lc[h][1] = D >= 2 ? by - 1 : 0;
                lc[h][2] = D == 3 ? zb0 + bz : 0;
                const int qx = lc[h][0] + G, qy = D >= 2 ? lc[h][1] + G : 0, qz = D == 3 ? bz + 2 : 0;
                cen[h] = (qz * P::PY + qy) * P::PX + qx;
                const float r0 = prim[cen[h]], p0 = prim[(F - 1) * P::PLANE + cen[h]];
                ir[h] = 1.f / r0;
                ip[h] = 1.f / p0;
                ic[h] = rsqrtf((float)g.gamma * p0 * ir[h]);
                bool indom = true;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (g.periodic[d]) continue;
                    const int Gd = c[d] * N + lc[h][d];
                    indom = indom && Gd >= 0 && Gd < g.ext[lev][d] * N;
                }
                valid[h] = valid[h] && indom;
            }
            auto feat = [&](int h, int k) -> float {
                const int o = koff[k];
                if (o < 0) return 0.f;
                const int kind = o >> 28;
                const float v = prim[cen[h] + (o & 0x0FFFFFFF) - (1 << 20)];
                return kind == 0 ? v * ir[h] - 1.f : (kind == 2 ? v * ip[h] - 1.f : v * ic[h]);
            };
            const float2 z = mlp_tile<D>(ms, feat);
            const bool m0 = valid[0] && z.x > 0.f, m1 = valid[1] && z.y > 0.f;
            const bool any = __any_sync(0xffffffffu, m0 || m1);
            if (any && lane == 0) atomicOr(&anyflag[slot], 1);
            if (stats) {
                unsigned long long cnt[4] = {0, 0, 0, 0};
                if ((lane & 3) == 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!valid[h]) continue;
                        const bool pf = plain_flag_cell<T, D, N>(g, U, slot, lc[h]);
                        const bool lf = h ? m1 : m0;
                        cnt[pf ? (lf ? 0 : 2) : (lf ? 1 : 3)] += 1;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    unsigned long long v = cnt[q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && v) atomicAdd(&stats[q], v);
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int D, int N>
static cudaError_t flag_mlp_launch(const Grid& g, const T* U, const float* w, int* anyflag,
                                   unsigned long long* stats, int grid, cudaStream_t s) {
    constexpr size_t smem = mlp_flag_smem<D, N>();
    k_flag_mlp<T, D, N><<<grid, 256, smem, s>>>(g, U, w, anyflag, stats);
    return cudaGetLastError();
}

template <typename T, int D, int N>
static cudaError_t flag_mlp_prepare() {
    constexpr size_t smem = mlp_flag_smem<D, N>();
    return cudaFuncSetAttribute(k_flag_mlp<T, D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t Kernels<T>::flag_mlp(const Grid& g, const T* U, const float* w, int* anyflag, int grid,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(anyflag, 0, sizeof(int) * (size_t)g.cap, s);
    if (e != cudaSuccess) return e;
    AMR_DISPATCH(g, return (flag_mlp_launch<T, D, N>(g, U, w, anyflag, nullptr, grid, s)));
    return cudaSuccess;
}

template <typename T>
cudaError_t Kernels<T>::flag_stats(const Grid& g, const T* U, const float* w, unsigned long long* counts,
                                   int grid, cudaStream_t s) {
    // the per-patch flags land in a scratch area after the four counters
    int* scratch = reinterpret_cast<int*>(counts + 4);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * (size_t)g.cap, s);
    if (e != cudaSuccess) return e;
    AMR_DISPATCH(g, return (flag_mlp_launch<T, D, N>(g, U, w, scratch, counts, grid, s)));
    return cudaSuccess;
}

template <typename T>
cudaError_t Kernels<T>::prepare_mlp(const Grid& g) {
    AMR_DISPATCH(g, return (flag_mlp_prepare<T, D, N>()));
    return cudaSuccess;
}

}  // namespace amr
