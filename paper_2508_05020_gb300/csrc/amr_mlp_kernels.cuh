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
// K10: learned indicator on the band [-1, N]^d of every leaf patch. A work
// item is a leaf patch (1D/2D) or a slab of DZ band planes of it (3D); items
// are taken from a global counter in slab-major order, items of a patch that
// is already flagged are skipped, and the next item's state is prefetched into
// L2 while the current one is evaluated. Band cells are evaluated 128 at a time
// (a tile, one row per TMEM lane). Inside the kernel the K axis is ordered by
// stencil plane (3D: the offset oz; 1D/2D: a single plane), then field, then
// point of the plane, each plane padded to PK columns; a K chunk is one plane.
// The CTA is warp-specialised:
//  - 8 producer warps stage the primitives (rho, u.., p) of the item and its
//    +-2 halo in shared memory (FP32), then compute the centre-normalised
//    features of one stencil plane of a tile (each warp: 32 rows x PK/2
//    columns; every column's cell offset and field are compile-time), convert
//    them to BF16 and store them with tcgen05.st into a ring of NS chunk
//    buffers in tensor memory (row = TMEM lane, two features per 32-bit
//    column), then arrive on the buffer's `full` barrier;
//  - one thread of the MMA warp waits for each chunk, issues the layer-1
//    tcgen05.mma (M = 128, N = 64, K = 16 per slice, A from tensor memory, W1
//    from shared memory) into the tile's accumulator and commits to the
//    buffer's `empty` barrier; at the end of a tile it commits to `acc_full`
//    and, once the epilogue has written the hidden layer (again into tensor
//    memory), issues the layer-2 MMA (K = 64, into the same accumulator
//    columns) and commits to `l2_full`;
//  - 4 epilogue warps (TMEM lanes 0-127) turn the layer-1 accumulator into the
//    BF16 hidden layer (bias + ReLU), then form the logit from the layer-2
//    accumulator, and flag the patch if an in-domain band cell has a positive
//    logit.
// The accumulators are double-buffered, so the epilogue of one tile overlaps
// the layer-1 MMAs of the next. Rows are ordered x fastest, then z, then y
// (3D), and the staged primitives use padded x and plane pitches for which the
// shared-memory words of 32 consecutive rows fall in 32 distinct banks, for
// every stencil offset. With `stats` the plain sensor of every band cell is
// evaluated too and the agreement counts TP, FP, FN, TN accumulated.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pad_mod32(int n, int r) { return n + (((r - n) % 32) + 32) % 32; }

// plane-major K order of the fused kernel
template <int D> struct MlpPlanes {
    static constexpr int F = D + 2;
    static constexpr int NPL = D == 3 ? 5 : 1;            // stencil planes = K chunks per tile
    static constexpr int PPL = D == 1 ? 5 : 25;           // stencil points per plane
    static constexpr int PF = F * PPL;                    // features per plane
    static constexpr int SG = 2;                          // producer warps per row group
    static constexpr int PK = (PF + 16 * SG - 1) / (16 * SG) * (16 * SG);   // K per plane, padded
    static constexpr int SPG = PK / (16 * SG);            // 16-wide slices per producer warp
    static constexpr int KF = NPL * PK;
};

template <int D> struct MlpFlagW {
    __nv_bfloat16 w1[MLP_H * MlpPlanes<D>::KF];           // canonical K-major, plane-major K
    __nv_bfloat16 w2[MLP_H * MLP_H];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
};

// flat float weights (W1 with k = j (d + 2) + f, stencil point j) -> shared memory
template <int D>
__device__ void mlp_flag_stage_weights(MlpFlagW<D>& s, const float* __restrict__ w) {
    using PL = MlpPlanes<D>;
    constexpr int K = mlp_kin(D), F = PL::F;
    const float* W1 = w;
    const float* B1 = W1 + MLP_H * K;
    const float* W2 = B1 + MLP_H;
    const float* B2 = W2 + MLP_H * MLP_H;
    const float* W3 = B2 + MLP_H;
    const float* B3 = W3 + MLP_H;
    for (int i = threadIdx.x; i < MLP_H * PL::KF; i += blockDim.x) {
        const int o = i / PL::KF, kf = i - o * PL::KF;
        const int pl = kf / PL::PK, p = kf - pl * PL::PK;
        float v = 0.f;
        if (p < PL::PF) {
            const int f = p / PL::PPL, j = pl * PL::PPL + p % PL::PPL;
            v = W1[o * K + j * F + f];
        }
        s.w1[canon_off(o, kf, PL::KF)] = __float2bfloat16_rn(v);
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) {
        const int o = i / MLP_H, k = i - o * MLP_H;
        s.w2[canon_off(o, k, MLP_H)] = __float2bfloat16_rn(W2[i]);
    }
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        s.b1[i] = B1[i];
        s.b2[i] = B2[i];
        s.w3[i] = W3[i];
    }
    if (threadIdx.x == 0) s.b3 = B3[0];
}

template <int D, int N> struct MlpBand {
    using PL = MlpPlanes<D>;
    static constexpr int B = N + 2;                       // band cells per dimension
    static constexpr int S = N + 2 * G;                   // slot cells per dimension
    static constexpr int DZ = D == 3 ? (B % 3 == 0 ? 3 : 2) : 1;
    static constexpr int NSLAB = D == 3 ? B / DZ : 1;
    static_assert(D != 3 || B % DZ == 0, "the slabs tile the band");
    // staged primitives: x pitch PX, plane pitch PP, PZ planes (3D)
    static constexpr int PX = D == 1 ? S : (D == 2 ? pad_mod32(S, B % 32) : pad_mod32(S, (B * DZ) % 32));
    static constexpr int PY = D >= 2 ? S : 1;
    static constexpr int PP = D == 3 ? pad_mod32(PX * S, B % 32) : PX * PY;
    static constexpr int PZ = D == 3 ? DZ + 4 : 1;
    static constexpr int PLANE = PP * PZ;                 // floats per primitive field
    static constexpr int CELLS = D == 1 ? B : (D == 2 ? B * B : B * B * DZ);
    static constexpr int F = D + 2;
    static constexpr int M = TC_M;                        // rows of a tile (TMEM lanes)
    static constexpr int TILES = (CELLS + M - 1) / M;
    static constexpr int NS = 5;                          // chunk ring depth (tensor memory)
    static constexpr int EPI_WARPS = 4, MMA_WARP = 4, PROD_WARP0 = 5, PROD_WARPS = 4 * PL::SG;
    static constexpr int NPROD = PROD_WARPS * 32;
    static constexpr int NTH = (PROD_WARP0 + PROD_WARPS) * 32;
    // tensor memory columns: accumulator of tile parity a at 64 a (layer 1,
    // then layer 2), the hidden layer (layer-2 A), the chunk ring
    static constexpr int TM_H = 2 * MLP_H, TM_RING = TM_H + MLP_H / 2, TMEM_COLS = 512;
    static constexpr int STAGE_COLS = PL::PK / 2;
    static_assert(TM_RING + NS * STAGE_COLS <= TMEM_COLS, "tensor memory budget");
    // band cell of row r (1D: x; 2D: x, y; 3D: x, z, y)
    __device__ static void cell(int r, int& bx, int& by, int& bz) {
        bx = r % B;
        if (D == 1) { by = 0; bz = 0; }
        else if (D == 2) { by = r / B; bz = 0; }
        else { bz = (r / B) % DZ; by = r / (B * DZ); }
    }
};

// features of one stencil plane for producer group SGI: columns
// SGI * SPG * 16 .. + SPG * 16 of the plane, packed two per word; `c` points at
// the row's centre cell in the plane (field 0), scale/shift per field kind
template <int D, int N, int SGI>
__device__ __forceinline__ void plane_features(const float* c, float s_rho, float s_u, float s_p,
                                               uint32_t (&wv)[MlpPlanes<D>::SPG * 8]) {
    using PL = MlpPlanes<D>;
    using P = MlpBand<D, N>;
#pragma unroll
    for (int i = 0; i < PL::SPG * 16; i += 2) {
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int p = SGI * PL::SPG * 16 + i + h;
            if (p < PL::PF) {
                const int f = p / PL::PPL, jj = p % PL::PPL;
                const int off = f * P::PLANE + (D >= 2 ? (jj / 5 - 2) * P::PX : 0) + jj % 5 - 2;
                const float x = c[off];
                v[h] = f == 0 ? fmaf(x, s_rho, -1.f) : (f == PL::F - 1 ? fmaf(x, s_p, -1.f) : x * s_u);
            } else {
                v[h] = 0.f;
            }
        }
        wv[i / 2] = pack_bf16(v[0], v[1]);
    }
}

template <int D, int N> struct MlpFlagLayout {
    using P = MlpBand<D, N>;
    static constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
    static constexpr size_t W = 0;
    static constexpr size_t PRIM = al(sizeof(MlpFlagW<D>));
    static constexpr size_t CTL = al(PRIM + sizeof(float) * P::F * P::PLANE);     // int4 stage_ctl[NS], tile_ctl[2]
    static constexpr size_t BARS = CTL + sizeof(int4) * (P::NS + 2);
    // full[NS], empty[NS], acc_full[2], acc_empty[2], h_full, l2_full, fin
    static constexpr int NBAR = 2 * P::NS + 7;
    static constexpr size_t MISC = BARS + sizeof(uint64_t) * NBAR;                // tmem base, abort, items
    static constexpr size_t TOTAL = MISC + 16;
};

template <int D, int N>
constexpr size_t mlp_flag_smem() { return MlpFlagLayout<D, N>::TOTAL + 128; }

__device__ __forceinline__ void producer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}

template <typename T, int D, int N, bool STATS>
__global__ void __launch_bounds__(MlpBand<D, N>::NTH, 1)
    k_flag_mlp(Grid g, const T* __restrict__ U, const float* __restrict__ w, int* anyflag,
               unsigned long long* stats) {
    using P = MlpBand<D, N>;
    using PL = MlpPlanes<D>;
    using Lay = MlpFlagLayout<D, N>;
    constexpr int F = P::F, M = P::M, NS = P::NS, NPL = PL::NPL, PK = PL::PK, KF = PL::KF;
    static_assert(Lay::TOTAL + 128 <= 232448, "shared memory of one CTA");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    MlpFlagW<D>& ms = *reinterpret_cast<MlpFlagW<D>*>(base + Lay::W);
    float* prim = reinterpret_cast<float*>(base + Lay::PRIM);
    int4* stage_ctl = reinterpret_cast<int4*>(base + Lay::CTL);
    int4* tile_ctl = stage_ctl + NS;
    uint32_t* misc = reinterpret_cast<uint32_t*>(base + Lay::MISC);
    volatile int* abort_f = reinterpret_cast<volatile int*>(misc + 1);
    volatile int* s_item = reinterpret_cast<volatile int*>(misc + 2);      // current, next item
    const uint32_t b_full = smem_u32(base + Lay::BARS), b_empty = b_full + 8 * NS, b_accf = b_empty + 8 * NS;
    const uint32_t b_acce = b_accf + 16, b_h = b_acce + 16, b_l2 = b_h + 8, b_fin = b_l2 + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    mlp_flag_stage_weights<D>(ms, w);
    if (warp == 0) tmem_alloc(smem_u32(misc), P::TMEM_COLS);
    if (threadIdx.x == 32) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(b_full + 8 * s, P::PROD_WARPS);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(b_accf + 8 * a, 2);                 // the MMAs' commit + the tile record
            mbar_init(b_acce + 8 * a, P::EPI_WARPS);
        }
        mbar_init(b_h, P::EPI_WARPS);
        mbar_init(b_l2, 1);
        mbar_init(b_fin, 1);
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(misc);
    const int total = g.counts[1] * P::NSLAB;
    int* counter = anyflag + g.cap;                        // zeroed with the flags by the launcher

    if (warp >= P::PROD_WARP0) {
        // ---------------- producers ----------------
        // TMEM lane quarter of a warp is warp % 4: the row group follows it
        const int ptid = threadIdx.x - P::PROD_WARP0 * 32;
        const int frow = (warp & 3) * 32 + lane, sg = (warp - P::PROD_WARP0) >> 2;
        const uint32_t tm_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + P::TM_RING + sg * PL::SPG * 8;
        const T gm1 = T(g.gamma) - T(1);
        const int npatch = g.counts[1];
        // items are slab-major (slab = item / npatch): the slabs of a patch are
        // far apart in the order, so a patch decided by an earlier slab is
        // seen as decided when its later slabs come up and they are skipped.
        // Decided: the refine bit below the finest level (it implies the keep
        // bit), the keep bit on the finest level (which cannot refine)
        auto decided = [&](int it) -> bool {
            const int slot = g.leaf_list[it % npatch];
            const int need = g.level[slot] == g.L - 1 ? 2 : 1;
            return (*((volatile int*)&anyflag[slot]) & need) != 0;
        };
        auto grab = [&]() -> int {
            for (;;) {
                const int it = atomicAdd(counter, 1);
                if (it >= total || *abort_f) return -1;
                if constexpr (STATS) return it;
                if (!decided(it)) return it;
            }
        };
        int s = 0, nxt = -2;                               // nxt: the item prefetched (-2: none taken yet)
        uint32_t ph = 0;                                   // ring position and pass parity
        for (;;) {
            producer_sync(P::NPROD);                       // the previous item's primitives are no longer read
            if (ptid == 0) {
                int it = nxt == -2 ? grab() : nxt;
                if constexpr (!STATS) {                    // flagged since it was taken: skip it
                    if (it >= 0 && decided(it)) it = grab();
                }
                s_item[0] = it;
                s_item[1] = it >= 0 ? grab() : -1;
            }
            producer_sync(P::NPROD);
            const int item = s_item[0];
            nxt = s_item[1];
            if (item < 0) {                                // end record in the next chunk buffer
                mbar_wait_ab(b_empty + 8 * s, ph ^ 1, abort_f, g.tc_wait);
                if (ptid == 0) stage_ctl[s] = make_int4(-1, 0, 0, 0);
                __syncwarp();
                if (lane == 0) mbar_arrive(b_full + 8 * s);
                break;
            }
            if (nxt >= 0) {                                // the next item's state into L2 meanwhile
                const int nslot = g.leaf_list[nxt % npatch], nslab = nxt / npatch;
                const int nz0 = D == 3 ? nslab * P::DZ - 3 + G : 0;
                constexpr int LINE_ELEMS = 128 / sizeof(T);
                const long long span = (long long)P::PZ * g.SY * g.SX;
                const int lines = (int)((span + LINE_ELEMS - 1) / LINE_ELEMS);
                for (int i = ptid; i < F * lines; i += P::NPROD) {
                    const int v = i / lines, ln = i - v * lines;
                    const T* a = U + slot_index(g, nslot, v, nz0, 0, 0) + (long long)ln * LINE_ELEMS;
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
                }
            }
            const int pi = item % npatch, slab = item / npatch;
            const int slot = g.leaf_list[pi];
            const int zb0 = D == 3 ? slab * P::DZ - 1 : 0;  // first band plane (local z)
            // primitives of the slab and its halo: local z in [zb0 - 2, zb0 + DZ + 2),
            // loaded as 16-byte vectors along x (slot rows are 16-byte aligned)
            {
                // aligned vectors of the padded row covering slot x in [0, S):
                // vector xv starts at slot x xv VE - XP (negative: the row pad)
                constexpr int VE = 16 / sizeof(T);
                constexpr int XP = PatchShape<T, N>::XP;
                constexpr int XV0 = XP / VE, NXV = (XP + P::S + VE - 1) / VE - XV0;
                constexpr int NVEC = NXV * P::PY * P::PZ;
                for (int iv = ptid; iv < NVEC; iv += P::NPROD) {
                    const int xv = iv % NXV, py = (iv / NXV) % P::PY, pz = iv / (NXV * P::PY);
                    const int sz = D == 3 ? zb0 - 2 + pz + G : 0;
                    const int x0 = (xv + XV0) * VE - XP;
                    T Uv[D + 2][VE];
#pragma unroll
                    for (int v = 0; v < D + 2; ++v) {
                        const T* src = U + slot_index(g, slot, v, sz, py, x0);
                        if constexpr (sizeof(T) == 4) {
                            const float4 q = *reinterpret_cast<const float4*>(src);
                            Uv[v][0] = q.x; Uv[v][1] = q.y; Uv[v][2] = q.z; Uv[v][3] = q.w;
                        } else {
                            const double2 q = *reinterpret_cast<const double2*>(src);
                            Uv[v][0] = q.x; Uv[v][1] = q.y;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < VE; ++e) {
                        const int px = x0 + e;
                        if (px < 0 || px >= P::S) continue;
                        T Uc[D + 2];
#pragma unroll
                        for (int v = 0; v < D + 2; ++v) Uc[v] = Uv[v][e];
                        T rho, u[D], p, Tt;
                        primitives<T, D>(Uc, gm1, rho, u, p, Tt);
                        const int idx = pz * P::PP + py * P::PX + px;
                        prim[idx] = (float)rho;
#pragma unroll
                        for (int d = 0; d < D; ++d) prim[(1 + d) * P::PLANE + idx] = (float)u[d];
                        prim[(F - 1) * P::PLANE + idx] = (float)p;
                    }
                }
            }
            producer_sync(P::NPROD);
            for (int tile = 0; tile < P::TILES; ++tile) {
                // the row's centre cell and its normalisation: 1/rho0, 1/c0, 1/p0
                const int r = tile * M + frow;
                int bx, by, bz;
                P::cell(r < P::CELLS ? r : P::CELLS - 1, bx, by, bz);
                const int mcen = (D == 3 ? (bz + 2) * P::PP : 0) + (D >= 2 ? (by - 1 + G) * P::PX : 0) + bx - 1 + G;
                const float r0 = prim[mcen], p0 = prim[(F - 1) * P::PLANE + mcen];
                const float s_rho = 1.f / r0;
                const float s_u = rsqrtf((float)g.gamma * p0 * s_rho), s_p = 1.f / p0;
#pragma unroll 1
                for (int pl = 0; pl < NPL; ++pl) {
                    uint32_t wv[PL::SPG * 8];
                    const float* c = prim + mcen + (D == 3 ? (pl - 2) * P::PP : 0);
                    if (sg == 0) plane_features<D, N, 0>(c, s_rho, s_u, s_p, wv);
                    else plane_features<D, N, 1>(c, s_rho, s_u, s_p, wv);
                    mbar_wait_ab(b_empty + 8 * s, ph ^ 1, abort_f, g.tc_wait);
                    tc_fence_after();
                    if (pl == 0 && ptid == 0) stage_ctl[s] = make_int4(slot, zb0, tile, 0);
                    const uint32_t ta = tm_lane + s * P::STAGE_COLS;
                    if constexpr (PL::SPG == 4) {
                        tmem_st32(ta, wv);
                    } else {
#pragma unroll
                        for (int q = 0; q < PL::SPG; ++q) {
                            uint32_t w8[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) w8[e] = wv[q * 8 + e];
                            tmem_st8(ta + q * 8, w8);
                        }
                    }
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_full + 8 * s);
                    if (++s == NS) { s = 0; ph ^= 1; }
                }
            }
        }
    } else if (warp == P::MMA_WARP) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            constexpr uint32_t IDESC = umma_idesc_bf16(TC_M, MLP_H);
            // descriptors advance by k 16-byte units per k columns (canonical K-major)
            const uint64_t bd1 = umma_desc(smem_u32(ms.w1), 128, (KF >> 3) * 128);
            const uint64_t bd2 = umma_desc(smem_u32(ms.w2), 128, (MLP_H >> 3) * 128);
            auto layer2 = [&](int tt) -> bool {           // hidden layer of tile tt written -> its layer-2 MMA
                if (!mbar_wait_ab(b_h, tt & 1, abort_f, g.tc_wait)) return false;
                tc_fence_after();
                const uint32_t d = tmem + (tt & 1) * MLP_H;
#pragma unroll
                for (int kk = 0; kk < MLP_H; kk += 16)
                    umma_bf16_ts(d, tmem + P::TM_H + kk / 2, bd2 + (uint64_t)kk, IDESC, kk > 0 ? 1u : 0u);
                umma_commit(b_l2);
                return true;
            };
            int s = 0, t = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (;;) {
                if (!mbar_wait_ab(b_full + 8 * s, ph, abort_f, g.tc_wait)) { ok = false; break; }
                const int4 info = stage_ctl[s];
                if (info.x < 0) break;                     // no more items
                const int a = t & 1;
                if (t >= 2 && !mbar_wait_ab(b_acce + 8 * a, ((t >> 1) - 1) & 1, abort_f, g.tc_wait)) { ok = false; break; }
                const uint32_t d = tmem + a * MLP_H;
#pragma unroll 1
                for (int pl = 0; pl < NPL; ++pl) {
                    if (pl > 0 && !mbar_wait_ab(b_full + 8 * s, ph, abort_f, g.tc_wait)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t aa = tmem + P::TM_RING + s * P::STAGE_COLS;
                    const uint64_t bb = bd1 + (uint64_t)(pl * PK);
#pragma unroll
                    for (int q = 0; q < PK / 16; ++q)
                        umma_bf16_ts(d, aa + q * 8, bb + (uint64_t)(q * 16), IDESC, (pl | q) ? 1u : 0u);
                    umma_commit(b_empty + 8 * s);
                    if (++s == NS) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                if (!g.tc_test) {                          // (a timeout test withholds the signal)
                    umma_commit(b_accf + 8 * a);
                    tile_ctl[a] = info;
                    mbar_arrive(b_accf + 8 * a);
                }
                if (t > 0 && !layer2(t - 1)) { ok = false; break; }
                ++t;
            }
            if (ok && t > 0) ok = layer2(t - 1);
            if (ok) {                                      // end record for the epilogue
                const int a = t & 1;
                if (t < 2 || mbar_wait_ab(b_acce + 8 * a, ((t >> 1) - 1) & 1, abort_f, g.tc_wait)) {
                    tile_ctl[a] = make_int4(-1, 0, 0, 0);
                    mbar_arrive_n(b_accf + 8 * a, 2);
                }
            }
            umma_commit(b_fin);                            // every MMA issued has completed
            if (!mbar_wait_cycles(b_fin, 0)) *abort_f = 1;
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (TMEM lanes 0-127) ----------------
        const int row = warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int t = 0;; ++t) {
            const int a = t & 1;
            if (!mbar_wait_ab(b_accf + 8 * a, (t >> 1) & 1, abort_f, g.tc_wait)) break;
            const int4 info = tile_ctl[a];
            if (info.x < 0) break;
            tc_fence_after();
            const uint32_t d = tmem + lane_base + a * MLP_H;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tmem_ld16(d + q * 16, v);
                uint32_t pk[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int cc = q * 16 + 2 * e;
                    pk[e] = pack_bf16(fmaxf(v[2 * e] + ms.b1[cc], 0.f), fmaxf(v[2 * e + 1] + ms.b1[cc + 1], 0.f));
                }
                tmem_st8(tmem + lane_base + P::TM_H + q * 8, pk);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_h);
            if (!mbar_wait_ab(b_l2, t & 1, abort_f, g.tc_wait)) break;
            tc_fence_after();
            float z = ms.b3;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tmem_ld16(d + q * 16, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) z += fmaxf(v[e] + ms.b2[q * 16 + e], 0.f) * ms.w3[q * 16 + e];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_acce + 8 * a);
            // the row's band cell, in-domain test, flag
            const int slot = info.x, zb0 = info.y, r = info.z * M + row;
            const bool inb = r < P::CELLS;
            int bx, by, bz;
            P::cell(inb ? r : P::CELLS - 1, bx, by, bz);
            const int lc[3] = {bx - 1, D >= 2 ? by - 1 : 0, D == 3 ? zb0 + bz : 0};
            const int lev = g.level[slot];
            bool indom = inb;
#pragma unroll
            for (int dd = 0; dd < D; ++dd) {
                if (g.periodic[dd]) continue;
                const int Gd = g.coord[slot * 3 + dd] * N + lc[dd];
                indom = indom && Gd >= 0 && Gd < g.ext[lev][dd] * N;
            }
            // bit 0: refine (logit > -R); bit 1: keep, blocks coarsening (logit > -H)
            const bool m = indom && z > -g.mlp_refine;
            const bool k = indom && z > -g.mlp_keep;
            const int bits = (__any_sync(0xffffffffu, m) ? 1 : 0) | (__any_sync(0xffffffffu, k) ? 2 : 0);
            if (bits && lane == 0) atomicOr(&anyflag[slot], bits);
            if constexpr (STATS) {
                unsigned long long cnt[4] = {0, 0, 0, 0};
                if (indom) {
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
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, P::TMEM_COLS);
    if (threadIdx.x == 0 && *abort_f) atomicOr(&g.time->err, ERR_TIMEOUT);
}

template <typename T, int D, int N>
static cudaError_t flag_mlp_launch(const Grid& g, const T* U, const float* w, int* anyflag,
                                   unsigned long long* stats, int grid, cudaStream_t s) {
    constexpr size_t smem = mlp_flag_smem<D, N>();
    if (stats) k_flag_mlp<T, D, N, true><<<grid, MlpBand<D, N>::NTH, smem, s>>>(g, U, w, anyflag, stats);
    else k_flag_mlp<T, D, N, false><<<grid, MlpBand<D, N>::NTH, smem, s>>>(g, U, w, anyflag, stats);
    return cudaGetLastError();
}

template <typename T, int D, int N>
static cudaError_t flag_mlp_prepare() {
    constexpr size_t smem = mlp_flag_smem<D, N>();
    cudaError_t e = cudaFuncSetAttribute(k_flag_mlp<T, D, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_flag_mlp<T, D, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t Kernels<T>::flag_mlp(const Grid& g, const T* U, const float* w, int* anyflag, int grid,
                                 cudaStream_t s) {
    // per-slot flags and, after them, the work-item counter
    cudaError_t e = cudaMemsetAsync(anyflag, 0, sizeof(int) * ((size_t)g.cap + 1), s);
    if (e != cudaSuccess) return e;
    AMR_DISPATCH(g, return (flag_mlp_launch<T, D, N>(g, U, w, anyflag, nullptr, grid, s)));
    return cudaSuccess;
}

template <typename T>
cudaError_t Kernels<T>::flag_stats(const Grid& g, const T* U, const float* w, unsigned long long* counts,
                                   int grid, cudaStream_t s) {
    // the per-patch flags and the work-item counter land in a scratch area
    // after the four counters
    int* scratch = reinterpret_cast<int*>(counts + 4);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * ((size_t)g.cap + 1), s);
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
