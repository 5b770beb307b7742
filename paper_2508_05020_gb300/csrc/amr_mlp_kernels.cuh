// Learned refinement indicator, AMR side: training-sample harvest from 1D
// runs, per-patch inference over the band [-1, N]^d of leaf patches, and the
// cell-level agreement counts against the plain sensor. Included by the two
// precision units after amr_launch.cuh.
#pragma once
#include "amr_launch.cuh"
#include "amr_mlp_core.cuh"
#include "amr_mlp_tc.cuh"

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

// ---------------------------------------------------------------------------
// K10: learned indicator on the band [-1, N]^d of every leaf patch. One work
// item is a leaf patch (1D/2D) or a slab of DZ band planes of it (3D). The
// primitives (rho, u.., p) of the slab and its +-2 halo are staged in shared
// memory in FP32. Band cells are taken 128 at a time (a GEMM tile, 16 rows per
// warp): all threads write the centre-normalised 5^d stencil features of the
// tile into a double-buffered 64-wide K chunk in shared memory (BF16, padded
// rows), and each warp accumulates layer 1 on the tensor cores from that chunk
// (ldmatrix + mma.sync). Layer 2 and the output follow in registers. A patch is
// flagged if any in-domain band cell has a positive logit; items of an already
// flagged patch are skipped. With `stats` the plain sensor of every band cell
// is evaluated too and the agreement counts TP, FP, FN, TN accumulated.
// ---------------------------------------------------------------------------
template <int D, int N> struct MlpBand {
    static constexpr int B = N + 2;                       // band cells per dimension
    static constexpr int S = N + 2 * G;                   // slot cells per dimension
    static constexpr int DZ = D == 3 ? 3 : 1;
    static constexpr int NSLAB = D == 3 ? B / DZ : 1;
    static constexpr int PX = S, PY = D >= 2 ? S : 1, PZ = D == 3 ? DZ + 4 : 1;
    static constexpr int PLANE = PX * PY * PZ;            // floats per primitive field
    static constexpr int CELLS = D == 1 ? B : (D == 2 ? B * B : B * B * DZ);
    static constexpr int F = D + 2;
    static constexpr int NTH = 512;                       // 16 warps
    static constexpr int M = TC_M;                        // rows of a tile (TMEM lanes)
    static constexpr int TILES = (CELLS + M - 1) / M;
};

template <int D, int N> struct MlpFlagLayout {
    using P = MlpBand<D, N>;
    static constexpr size_t W = 0;
    static constexpr size_t KREL = (sizeof(MlpTcSmem<D>) + 127) / 128 * 128;
    static constexpr size_t PRIM = KREL + sizeof(int) * mlp_pts(D);
    static constexpr size_t ABUF = (PRIM + sizeof(float) * P::F * P::PLANE + 127) / 128 * 128;
    static constexpr size_t HBUF = ABUF + 2 * sizeof(__nv_bfloat16) * TC_M * TC_KC;
    static constexpr size_t ROWS = HBUF + sizeof(__nv_bfloat16) * TC_M * MLP_H;
    static constexpr size_t SLOTS = ROWS + sizeof(int) * 8 * TC_M;
    static constexpr size_t TOTAL = SLOTS + 4 * sizeof(uint64_t);
};

template <int D, int N>
constexpr size_t mlp_flag_smem() { return MlpFlagLayout<D, N>::TOTAL + 128; }

template <typename T, int D, int N>
__global__ void __launch_bounds__(512, 1) k_flag_mlp(Grid g, const T* __restrict__ U, const float* __restrict__ w,
                                                     int* anyflag, unsigned long long* stats) {
    using P = MlpBand<D, N>;
    using Lay = MlpFlagLayout<D, N>;
    constexpr int F = P::F, M = P::M, NP = mlp_npts(D), PTS = mlp_pts(D), KP = mlp_kpad(D);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    MlpTcSmem<D>& ms = *reinterpret_cast<MlpTcSmem<D>*>(base + Lay::W);
    int* krel = reinterpret_cast<int*>(base + Lay::KREL);
    float* prim = reinterpret_cast<float*>(base + Lay::PRIM);
    __nv_bfloat16* abuf = reinterpret_cast<__nv_bfloat16*>(base + Lay::ABUF);
    __nv_bfloat16* hbuf = reinterpret_cast<__nv_bfloat16*>(base + Lay::HBUF);
    int* rcen = reinterpret_cast<int*>(base + Lay::ROWS);
    float* rsc = reinterpret_cast<float*>(rcen + M);      // [3][M]: 1/rho0, 1/c0, 1/p0
    int* rval = reinterpret_cast<int*>(rsc + 3 * M);
    int* rlc = rval + M;                                  // [3][M]: local cell
    uint64_t* slots = reinterpret_cast<uint64_t*>(base + Lay::SLOTS);
    __shared__ int skip;
    mlp_tc_stage_weights<D>(ms, w);
    // stencil point j -> offset of its cell from the centre cell (padding points: 0)
    for (int j = threadIdx.x; j < PTS; j += blockDim.x) {
        const int ox = j % 5 - 2, oy = D >= 2 ? (j / 5) % 5 - 2 : 0, oz = D == 3 ? j / 25 - 2 : 0;
        krel[j] = j < NP ? (oz * P::PY + oy) * P::PX + ox : 0;
    }
    TcState st;
    tc_setup(st, slots);                                   // includes a CTA barrier
    const T gm1 = T(g.gamma) - T(1);
    const int npatch = g.counts[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // feature-fill role: row of the tile and a 16-wide K slice of the chunk
    const int frow = (warp & 3) * 32 + lane, fslice = warp >> 2;
    bool alive = true;
    for (int item = blockIdx.x; item < npatch * P::NSLAB && alive; item += gridDim.x) {
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
        for (int tile = 0; tile < P::TILES; ++tile) {
            if (threadIdx.x < M) {                         // per-row data of the tile
                const int r = tile * M + threadIdx.x;
                const bool inb = r < P::CELLS;
                const int rr = inb ? r : P::CELLS - 1;
                const int bx = rr % P::B, by = D >= 2 ? (rr / P::B) % P::B : 0, bz = D == 3 ? rr / (P::B * P::B) : 0;
                const int l0 = bx - 1, l1 = D >= 2 ? by - 1 : 0, l2 = D == 3 ? zb0 + bz : 0;
                const int qx = l0 + G, qy = D >= 2 ? l1 + G : 0, qz = D == 3 ? bz + 2 : 0;
                const int cen = (qz * P::PY + qy) * P::PX + qx;
                const float r0 = prim[cen], p0 = prim[(F - 1) * P::PLANE + cen];
                const float ir = 1.f / r0;
                bool indom = inb;
                const int lcv[3] = {l0, l1, l2};
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (g.periodic[d]) continue;
                    const int Gd = c[d] * N + lcv[d];
                    indom = indom && Gd >= 0 && Gd < g.ext[lev][d] * N;
                }
                rcen[threadIdx.x] = cen;
                rsc[threadIdx.x] = ir;
                rsc[M + threadIdx.x] = rsqrtf((float)g.gamma * p0 * ir);
                rsc[2 * M + threadIdx.x] = 1.f / p0;
                rval[threadIdx.x] = indom ? 1 : 0;
                rlc[threadIdx.x] = l0;
                rlc[M + threadIdx.x] = l1;
                rlc[2 * M + threadIdx.x] = l2;
            }
            __syncthreads();
            const int mcen = rcen[frow];
            const float sc0 = rsc[frow], sc1 = rsc[M + frow], sc2 = rsc[2 * M + frow];
            // 16 features (one field, 16 consecutive stencil points) of chunk cc
            auto fill = [&](int cc, __nv_bfloat16* dst) {
                const int k0 = cc * TC_KC + fslice * 16;
                uint32_t wv[8];
                if (k0 < KP) {
                    const int f = k0 / PTS, j0 = k0 - f * PTS;
                    const float sc = f == 0 ? sc0 : (f == F - 1 ? sc2 : sc1);
                    const float sh = (f == 0 || f == F - 1) ? -1.f : 0.f;
                    const float* pf = prim + f * P::PLANE + mcen;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x0 = pf[krel[j0 + 2 * e]], x1 = pf[krel[j0 + 2 * e + 1]];
                        wv[e] = pack_bf16(x0 * sc + sh, x1 * sc + sh);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) wv[e] = 0u;
                }
                *reinterpret_cast<uint4*>(dst + canon_off(frow, fslice * 16, TC_KC)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                *reinterpret_cast<uint4*>(dst + canon_off(frow, fslice * 16 + 8, TC_KC)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
            };
            const float z = mlp_tile_tc<D>(st, ms, abuf, hbuf, fill);
            if (!__syncthreads_and(st.ok ? 1 : 0)) {       // a bounded wait gave up somewhere
                if (threadIdx.x == 0) atomicOr(&g.time->err, ERR_TIMEOUT);
                alive = false;
                break;
            }
            if (warp < 4) {
                const int row = warp * 32 + lane;
                const bool m = rval[row] && z > 0.f;
                if (__any_sync(0xffffffffu, m) && lane == 0) atomicOr(&anyflag[slot], 1);
                if (stats) {
                    unsigned long long cnt[4] = {0, 0, 0, 0};
                    if (rval[row]) {
                        const int lc[3] = {rlc[row], rlc[M + row], rlc[2 * M + row]};
                        const bool pf = plain_flag_cell<T, D, N>(g, U, slot, lc);
                        cnt[pf ? (m ? 0 : 2) : (m ? 1 : 3)] += 1;
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
            if (!stats) {                                    // the rest of a flagged patch is skipped
                if (threadIdx.x == 0) skip = *((volatile int*)&anyflag[slot]);
                __syncthreads();
                if (skip) break;
            }
        }
        __syncthreads();
    }
    tc_teardown(st);
}

template <typename T, int D, int N>
static cudaError_t flag_mlp_launch(const Grid& g, const T* U, const float* w, int* anyflag,
                                   unsigned long long* stats, int grid, cudaStream_t s) {
    constexpr size_t smem = mlp_flag_smem<D, N>();
    k_flag_mlp<T, D, N><<<grid, MlpBand<D, N>::NTH, smem, s>>>(g, U, w, anyflag, stats);
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
