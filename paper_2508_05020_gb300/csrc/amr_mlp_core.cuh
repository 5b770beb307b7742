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
__host__ __device__ constexpr int mlp_kpad(int d) { return (mlp_kin(d) + 15) / 16 * 16; }

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
    for (int i = threadIdx.x; i < MLP_H * KP; i += blockDim.x) {
        const int o = i / KP, k = i - o * KP;
        s.w1[o * P1 + k] = __float2bfloat16_rn(k < K ? W1[o * K + k] : 0.f);
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
    // bias + ReLU, re-packed as the layer-2 A operand
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
        for (int n = 0; n < 8; ++n) {
            const __nv_bfloat16* wr = s.w2 + (n * 8 + g) * P2 + kk * 16 + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 8);
            mma_bf16(acc2[n], a0, a1, a2, a3, b0, b1);
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

}  // namespace amr
