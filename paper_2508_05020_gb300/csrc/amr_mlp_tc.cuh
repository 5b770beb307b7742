// Learned refinement indicator on the 5th-generation tensor cores (tcgen05).
//
// A CTA evaluates 128-row tiles of the K -> 64 -> 64 -> 1 network. Layer 1:
// all warps write the BF16 features of a 64-wide K chunk into shared memory in
// the K-major, non-swizzled canonical layout (8-row x 16-byte core matrices);
// one thread issues tcgen05.mma (M = 128, N = 64, K = 16, BF16 x BF16 -> FP32)
// with shared-memory descriptors for the chunk and for the staged weights,
// accumulating in tensor memory, and tcgen05.commit arrives on an mbarrier
// when the chunk's MMAs are done (so the chunk buffer can be refilled). The
// four warps that own TMEM lanes 0-127 read the accumulator with tcgen05.ld,
// add bias + ReLU, write the hidden layer back as the layer-2 A operand, and
// a second MMA (K = 64) gives layer 2; the output neuron is a per-row dot
// product. Every mbarrier wait is bounded: on timeout the kernel records an
// error bit, still deallocates its tensor memory, and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "amr_mlp_core.cuh"

namespace amr {

constexpr int TC_M = 128;                // rows of a tile (TMEM lanes)
constexpr int TC_KC = 64;                // K chunk
constexpr int TC_TMEM_COLS = 512;        // whole tensor memory of the SM (headroom for any N decoding)
constexpr unsigned TC_SPIN_LIMIT = 1u << 26;

// weights in the canonical K-major layout: element (n, k) at
// (n / 8) * SBO + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2 bytes, SBO = (K / 8) * 128
template <int D> struct MlpTcSmem {
    static constexpr int KP = mlp_kpad(D);
    __nv_bfloat16 w1[MLP_H * KP];
    __nv_bfloat16 w2[MLP_H * MLP_H];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
};

__device__ __forceinline__ int canon_off(int r, int k, int kdim) {
    return (r >> 3) * (kdim >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);   // in bf16 elements
}

template <int D>
__device__ void mlp_tc_stage_weights(MlpTcSmem<D>& s, const float* __restrict__ w) {
    constexpr int K = mlp_kin(D), KP = mlp_kpad(D), F = D + 2, NP = mlp_npts(D), PTS = mlp_pts(D);
    const float* W1 = w;
    const float* B1 = W1 + MLP_H * K;
    const float* W2 = B1 + MLP_H;
    const float* B2 = W2 + MLP_H * MLP_H;
    const float* W3 = B2 + MLP_H;
    const float* B3 = W3 + MLP_H;
    for (int i = threadIdx.x; i < MLP_H * KP; i += blockDim.x) {
        const int o = i / KP, kp = i - o * KP;
        const int f = kp / PTS, j = kp - f * PTS;          // field-major K
        s.w1[canon_off(o, kp, KP)] = __float2bfloat16_rn(j < NP ? W1[o * K + j * F + f] : 0.f);
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

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for the completion of phase `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (unsigned it = 0; it < TC_SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA tensor-core state: TMEM base, mbarriers and their phases.
struct TcState {
    uint32_t tmem;          // TMEM base address (lane 0, first allocated column)
    uint32_t mbar_chunk[2]; // one per A-chunk buffer
    uint32_t mbar_l2;       // layer-2 completion
    uint32_t ph_chunk[2];
    uint32_t ph_l2;
    uint32_t pending[2];    // a commit on this buffer has not been waited for
    bool ok;                // no wait has timed out
};

// set-up by the whole CTA: warp 0 allocates TMEM, thread 0 initialises the
// mbarriers. `slots` is 8-byte aligned shared memory: [0..2] mbarriers, [3] TMEM address.
__device__ __forceinline__ void tc_setup(TcState& st, uint64_t* slots) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slots + 3)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(slots + 0), 1);
        mbar_init(smem_u32(slots + 1), 1);
        mbar_init(smem_u32(slots + 2), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    st.tmem = *reinterpret_cast<volatile uint32_t*>(slots + 3);
    st.mbar_chunk[0] = smem_u32(slots + 0);
    st.mbar_chunk[1] = smem_u32(slots + 1);
    st.mbar_l2 = smem_u32(slots + 2);
    st.ph_chunk[0] = st.ph_chunk[1] = 0;
    st.ph_l2 = 0;
    st.pending[0] = st.pending[1] = 0;
    st.ok = true;
}

// wait (bounded) for the outstanding commit of chunk buffer b
__device__ __forceinline__ void tc_drain(TcState& st, int b) {
    if (st.pending[b]) {
        if (!mbar_wait(st.mbar_chunk[b], st.ph_chunk[b])) st.ok = false;
        st.ph_chunk[b] ^= 1u;
        st.pending[b] = 0;
    }
}

// tear-down by the whole CTA: every commit waited for, then warp 0 frees TMEM
__device__ __forceinline__ void tc_teardown(TcState& st) {
    tc_drain(st, 0);
    tc_drain(st, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(st.tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// Logit of one 128-row tile. fill(cc, dst) writes the features of K chunk cc
// (TC_KC columns, canonical K-major layout with SBO = TC_KC / 8 * 128 bytes)
// into dst; every thread of the CTA takes part. abuf holds two chunk buffers,
// hbuf the 128 x 64 layer-2 operand. Returns the logit of row
// 32 warp + lane for warps 0-3 (other warps return 0).
template <int D, class Fill>
__device__ float mlp_tile_tc(TcState& st, const MlpTcSmem<D>& s, __nv_bfloat16* abuf, __nv_bfloat16* hbuf,
                             Fill fill) {
    constexpr int KP = mlp_kpad(D);
    constexpr int NCHUNK = (KP + TC_KC - 1) / TC_KC;
    constexpr uint32_t IDESC = umma_idesc_bf16(TC_M, MLP_H);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t d1 = st.tmem;                 // layer-1 accumulator: columns [0, 64)
    const uint32_t d2 = st.tmem + MLP_H;         // layer-2 accumulator: columns [64, 128)
    const uint32_t w1a = smem_u32(s.w1), w2a = smem_u32(s.w2);
    for (int cc = 0; cc < NCHUNK; ++cc) {
        const int b = cc & 1;
        tc_drain(st, b);                          // the MMAs that read this buffer are done
        __nv_bfloat16* dst = abuf + (size_t)b * TC_M * TC_KC;
        fill(cc, dst);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t aa = smem_u32(dst);
#pragma unroll
            for (int kk = 0; kk < TC_KC; kk += 16) {
                const int k = cc * TC_KC + kk;
                if (k < KP) {
                    const uint64_t ad = umma_desc(aa + (kk >> 3) * 128, 128, (TC_KC >> 3) * 128);
                    const uint64_t bd = umma_desc(w1a + (k >> 3) * 128, 128, (KP >> 3) * 128);
                    umma_bf16(d1, ad, bd, IDESC, k > 0 ? 1u : 0u);
                }
            }
            umma_commit(st.mbar_chunk[b]);
        }
        st.pending[b] = 1;
    }
    tc_drain(st, (NCHUNK - 1) & 1);               // the last commit covers every earlier MMA
    tc_drain(st, NCHUNK & 1);
    tc_fence_after();
    float z = 0.f;
    if (warp < 4) {
        const int row = warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[16];
            tmem_ld16(d1 + lane_base + q * 16, v);
            uint32_t pk[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = q * 16 + 2 * e;
                pk[e] = pack_bf16(fmaxf(v[2 * e] + s.b1[c], 0.f), fmaxf(v[2 * e + 1] + s.b1[c + 1], 0.f));
            }
            // columns q*16 .. q*16+15 = two 8-wide core-matrix rows of the layer-2 operand
            *reinterpret_cast<uint4*>(hbuf + canon_off(row, q * 16, MLP_H)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(hbuf + canon_off(row, q * 16 + 8, MLP_H)) =
                make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t ha = smem_u32(hbuf);
#pragma unroll
        for (int kk = 0; kk < MLP_H; kk += 16) {
            const uint64_t ad = umma_desc(ha + (kk >> 3) * 128, 128, (MLP_H >> 3) * 128);
            const uint64_t bd = umma_desc(w2a + (kk >> 3) * 128, 128, (MLP_H >> 3) * 128);
            umma_bf16(d2, ad, bd, IDESC, kk > 0 ? 1u : 0u);
        }
        umma_commit(st.mbar_l2);
    }
    if (!mbar_wait(st.mbar_l2, st.ph_l2)) st.ok = false;
    st.ph_l2 ^= 1u;
    tc_fence_after();
    if (warp < 4) {
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float acc = s.b3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[16];
            tmem_ld16(d2 + lane_base + q * 16, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) acc += fmaxf(v[e] + s.b2[q * 16 + e], 0.f) * s.w3[q * 16 + e];
        }
        z = acc;
    }
    tc_fence_before();
    __syncthreads();                               // TMEM and hbuf free for the next tile
    tc_fence_after();
    return z;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// Pipeline primitives of the warp-specialised flag kernel: mbarrier arrivals,
// a non-blocking test, and a wait bounded both in clock cycles and by a shared
// abort word (any role that times out sets it, and every other role's waits
// then return at once, so that the CTA reaches its tear-down).
// ---------------------------------------------------------------------------
namespace amr {

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_n(uint32_t mbar, uint32_t n) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar), "r"(n)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for the completion of phase `parity`; false once *abort is set or
// after `limit` SM cycles (which sets *abort)
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, volatile int* abort, long long limit) {
    if (mbar_try(mbar, parity)) return true;               // the common case: no clock read
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if (*abort) return false;
        if ((it & 63u) == 0u && clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
}

// the same wait without the abort word and at the full limit (tear-down:
// in-flight MMAs)
__device__ __forceinline__ bool mbar_wait_cycles(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    for (unsigned it = 0;; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 63u) == 63u && clock64() - t0 > TC_WAIT_CYCLES) return false;
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols) : "memory");
}

}  // namespace amr

namespace amr {

// tcgen05.mma with the A operand in tensor memory (M rows = TMEM lanes, K
// packed two BF16 per 32-bit column) and B from a shared-memory descriptor
__device__ __forceinline__ void umma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// 32 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

}  // namespace amr
