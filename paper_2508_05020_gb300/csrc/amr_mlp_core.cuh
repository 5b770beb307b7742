// Learned refinement indicator: the K -> 64 -> 64 -> 1 network (ReLU) on BF16
// tensor cores with FP32 accumulation, one warp per 16-row tile.
//
// Layer 1 and layer 2 use mma.sync m16n8k16 (A row-major 16x16 BF16, B the
// weight matrix W (n x k, row-major) read as a 16x8 column-major operand, C
// 16x8 FP32). The layer-1 accumulators are turned into the layer-2 A operand in
// registers (two adjacent 16x8 C tiles hold one 16x16 A tile), and the output
// neuron is a dot product reduced over each lane quad.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace amr {

constexpr int MLP_H = 64;

__host__ __device__ constexpr int mlp_kin(int d) { return d == 1 ? 15 : (d == 2 ? 100 : 625); }
// Inside the kernels the K axis is field-major: k' = f * PTS + j (field f of
// the d + 2 primitive fields, stencil point j padded to PTS, a multiple of 16),
// so every 16-wide K slice holds one field. The flat weight layout of the ABI
// (k = j (d + 2) + f) is permuted when the weights are staged.
__host__ __device__ constexpr int mlp_npts(int d) { return d == 1 ? 5 : (d == 2 ? 25 : 125); }
__host__ __device__ constexpr int mlp_pts(int d) { return (mlp_npts(d) + 15) / 16 * 16; }
__host__ __device__ constexpr int mlp_kpad(int d) { return (d + 2) * mlp_pts(d); }

// weights as staged in shared memory (BF16, zero-padded K, padded row pitch
// so the 8 rows a lane group touches fall in distinct banks)
template <int D> struct MlpSmem {
    static constexpr int K = mlp_kin(D);
    static constexpr int KP = mlp_kpad(D);
    static constexpr int P1 = KP + 8;          // W1 row pitch (bf16)
    static constexpr int P2 = MLP_H + 8;       // W2 row pitch
    __nv_bfloat16 w1[MLP_H * P1];
    __nv_bfloat16 w2[MLP_H * P2];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
};

// flat float weights: W1 (64 x K) | b1 | W2 (64 x 64) | b2 | W3 (64) | b3
template <int D>
__device__ void mlp_stage_weights(MlpSmem<D>& s, const float* __restrict__ w) {
    constexpr int K = MlpSmem<D>::K, KP = MlpSmem<D>::KP, P1 = MlpSmem<D>::P1, P2 = MlpSmem<D>::P2;
    const float* W1 = w;
    const float* B1 = W1 + MLP_H * K;
    const float* W2 = B1 + MLP_H;
    const float* B2 = W2 + MLP_H * MLP_H;
    const float* W3 = B2 + MLP_H;
    const float* B3 = W3 + MLP_H;
    constexpr int F = D + 2, NP = mlp_npts(D), PTS = mlp_pts(D);
    for (int i = threadIdx.x; i < MLP_H * KP; i += blockDim.x) {
        const int o = i / KP, kp = i - o * KP;
        const int f = kp / PTS, j = kp - f * PTS;
        s.w1[o * P1 + kp] = __float2bfloat16_rn(j < NP ? W1[o * K + j * F + f] : 0.f);
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) {
        const int o = i / MLP_H, k = i - o * MLP_H;
        s.w2[o * P2 + k] = __float2bfloat16_rn(W2[i]);
    }
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        s.b1[i] = B1[i];
        s.b2[i] = B2[i];
        s.w3[i] = W3[i];
    }
    if (threadIdx.x == 0) s.b3 = B3[0];
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// B fragments of two 16x8 n-tiles (rows n0 .. n0 + 15 of W, k .. k + 15) with
// one ldmatrix.x4: b[0], b[1] for rows n0..n0+7, b[2], b[3] for n0+8..n0+15.
__device__ __forceinline__ void ldmatrix_b(uint32_t (&b)[4], const __nv_bfloat16* W, int pitch, int n0, int k) {
    const int lane = threadIdx.x & 31;
    const int row = n0 + (lane & 7) + ((lane >> 4) << 3);
    const int col = k + (((lane >> 3) & 1) << 3);
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(W + row * pitch + col);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(addr));
}

// Layer 2 and the output neuron from the layer-1 accumulators of a warp's
// 16-row tile (bias + ReLU, re-packed in registers as the layer-2 A operand).
// Returns the logits of rows g (x) and g + 8 (y), valid in every lane.
template <int D>
__device__ __forceinline__ float2 mlp_epilogue(const MlpSmem<D>& s, const float (&acc)[8][4]) {
    constexpr int P2 = MlpSmem<D>::P2;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint32_t h[8][2];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int c = n * 8 + 2 * t;
        const float x0 = fmaxf(acc[n][0] + s.b1[c], 0.f), x1 = fmaxf(acc[n][1] + s.b1[c + 1], 0.f);
        const float y0 = fmaxf(acc[n][2] + s.b1[c], 0.f), y1 = fmaxf(acc[n][3] + s.b1[c + 1], 0.f);
        h[n][0] = pack_bf16(x0, x1);
        h[n][1] = pack_bf16(y0, y1);
    }
    float acc2[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) acc2[n][0] = acc2[n][1] = acc2[n][2] = acc2[n][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t a0 = h[2 * kk][0], a1 = h[2 * kk][1], a2 = h[2 * kk + 1][0], a3 = h[2 * kk + 1][1];
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            ldmatrix_b(b, s.w2, P2, np * 16, kk * 16);
            mma_bf16(acc2[2 * np], a0, a1, a2, a3, b[0], b[1]);
            mma_bf16(acc2[2 * np + 1], a0, a1, a2, a3, b[2], b[3]);
        }
    }
    float zx = 0.f, zy = 0.f;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int c = n * 8 + 2 * t;
        zx += fmaxf(acc2[n][0] + s.b2[c], 0.f) * s.w3[c] + fmaxf(acc2[n][1] + s.b2[c + 1], 0.f) * s.w3[c + 1];
        zy += fmaxf(acc2[n][2] + s.b2[c], 0.f) * s.w3[c] + fmaxf(acc2[n][3] + s.b2[c + 1], 0.f) * s.w3[c + 1];
    }
    zx += __shfl_xor_sync(0xffffffffu, zx, 1);
    zx += __shfl_xor_sync(0xffffffffu, zx, 2);
    zy += __shfl_xor_sync(0xffffffffu, zy, 1);
    zy += __shfl_xor_sync(0xffffffffu, zy, 2);
    return make_float2(zx + s.b3, zy + s.b3);
}

// Layer-1 accumulation of one 16-row x 16-k step of a warp from an A tile in
// shared memory (row-major BF16, row pitch `pitch` elements, 16-byte aligned
// rows): ldmatrix.x4 gives the A fragment, the weights come from s.w1 at k.
template <int D>
__device__ __forceinline__ void mma_l1_step(const MlpSmem<D>& s, const __nv_bfloat16* a_rows, int pitch, int kk,
                                            int k, float (&acc)[8][4]) {
    constexpr int P1 = MlpSmem<D>::P1;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* ap = a_rows + (lane & 15) * pitch + kk + (lane >> 4) * 8;
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(ap);
    uint32_t a0, a1, a2, a3;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                 : "r"(addr));
#pragma unroll
    for (int np = 0; np < 4; ++np) {
        uint32_t b[4];
        ldmatrix_b(b, s.w1, P1, np * 16, k);
        mma_bf16(acc[2 * np], a0, a1, a2, a3, b[0], b[1]);
        mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b[2], b[3]);
    }
}

// Logits of the 16 rows of one tile. feat(h, k) returns the feature k of the
// lane's row g + 8 h (g = lane / 4). Returns the logit of rows g (x) and
// g + 8 (y), valid in every lane.
template <int D, class Feat>
__device__ __forceinline__ float2 mlp_tile(const MlpSmem<D>& s, Feat feat) {
    constexpr int KP = MlpSmem<D>::KP, P1 = MlpSmem<D>::P1, P2 = MlpSmem<D>::P2;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll 2
    for (int kb = 0; kb < KP; kb += 16) {
        const int k0 = kb + 2 * t;
        const uint32_t a0 = pack_bf16(feat(0, k0), feat(0, k0 + 1));
        const uint32_t a1 = pack_bf16(feat(1, k0), feat(1, k0 + 1));
        const uint32_t a2 = pack_bf16(feat(0, k0 + 8), feat(0, k0 + 9));
        const uint32_t a3 = pack_bf16(feat(1, k0 + 8), feat(1, k0 + 9));
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const __nv_bfloat16* wr = s.w1 + (n * 8 + g) * P1 + k0;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 8);
            mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
        }
    }
    return mlp_epilogue<D>(s, acc);
}

}  // namespace amr
