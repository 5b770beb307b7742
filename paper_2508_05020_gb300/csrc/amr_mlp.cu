// Learned refinement indicator, standalone calls of include/amr.h: feature
// embedding of 1D samples, BF16 tensor-core inference, FP32 gradient and Adam
// training. The paper leaves the refinement criterion to the runtime program
// (Sec. 4.2); this network is one such program. Training is deterministic:
// every reduction is a fixed-order loop, no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "amr.h"
#include "amr_internal.h"
#include "amr_mlp_core.cuh"
#include "amr_mlp_tc.cuh"

namespace amr {
int mlp_k(int dim) { return mlp_kin(dim); }
long mlp_n_weights(int dim) {
    const long K = mlp_kin(dim);
    return MLP_H * K + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
}
}  // namespace amr

using namespace amr;

namespace {

// ---------------------------------------------------------------------------
// features: 1D 5-point samples (rho, u, p) embedded along axis a with sign s
// (point at offset o takes sample index 2 + s o_a, velocity component a = s u),
// normalised by the centre: rho/rho0 - 1, u/c0, p/p0 - 1, c0 = sqrt(gamma p0/rho0).
// Row 2 d i + 2 a + (s > 0); per point (z, y, x lexicographic) features (rho, u.., p).
// ---------------------------------------------------------------------------
__global__ void k_features(int D, double gamma, const double* __restrict__ smp, long n, float* __restrict__ X) {
    const int K = mlp_kin(D), F = D + 2;
    const long rows = n * 2 * D;
    for (long it = blockIdx.x * (long)blockDim.x + threadIdx.x; it < rows * K; it += (long)gridDim.x * blockDim.x) {
        const long row = it / K;
        const int k = (int)(it - row * K);
        const long i = row / (2 * D);
        const int r = (int)(row - i * 2 * D);
        const int a = r >> 1;
        const int s = (r & 1) ? 1 : -1;
        const int j = k / F, f = k - j * F;
        const int o[3] = {j % 5 - 2, D >= 2 ? (j / 5) % 5 - 2 : 0, D == 3 ? j / 25 - 2 : 0};
        const int idx = 2 + s * o[a];
        const double* S = smp + i * 15;
        const double r0 = S[2 * 3 + 0], p0 = S[2 * 3 + 2];
        const double c0 = sqrt(gamma * p0 / r0);
        double v;
        if (f == 0) v = S[idx * 3 + 0] / r0 - 1.0;
        else if (f == F - 1) v = S[idx * 3 + 2] / p0 - 1.0;
        else v = (f - 1 == a ? S[idx * 3 + 1] * s : 0.0) / c0;
        X[it] = (float)v;
    }
}

// standalone inference on feature rows (n x K floats, ABI feature order) on
// the tcgen05 core: 128-row tiles, features copied (BF16) into the canonical
// field-major chunk layout. Rows a timed-out CTA did not reach stay NaN.
template <int D> struct InferLayout {
    static constexpr size_t ABUF = (sizeof(MlpTcSmem<D>) + 127) / 128 * 128;
    static constexpr size_t HBUF = ABUF + 2 * sizeof(__nv_bfloat16) * TC_M * TC_KC;
    static constexpr size_t SLOTS = HBUF + sizeof(__nv_bfloat16) * TC_M * MLP_H;
    static constexpr size_t TOTAL = SLOTS + 4 * sizeof(uint64_t) + 128;
};

template <int D>
__global__ void __launch_bounds__(512, 1) k_infer(const float* __restrict__ X, long n, const float* __restrict__ w,
                                                  float* __restrict__ z, int* err) {
    using Lay = InferLayout<D>;
    constexpr int K = mlp_kin(D), KP = mlp_kpad(D), F = D + 2, NP = mlp_npts(D), PTS = mlp_pts(D);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    MlpTcSmem<D>& s = *reinterpret_cast<MlpTcSmem<D>*>(base);
    __nv_bfloat16* abuf = reinterpret_cast<__nv_bfloat16*>(base + Lay::ABUF);
    __nv_bfloat16* hbuf = reinterpret_cast<__nv_bfloat16*>(base + Lay::HBUF);
    uint64_t* slots = reinterpret_cast<uint64_t*>(base + Lay::SLOTS);
    mlp_tc_stage_weights<D>(s, w);
    TcState st;
    tc_setup(st, slots);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int frow = (warp & 3) * 32 + lane, fslice = warp >> 2;
    const long tiles = (n + TC_M - 1) / TC_M;
    for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long r = tile * TC_M + frow;
        const float* x = X + (r < n ? r : n - 1) * K;
        auto fill = [&](int cc, __nv_bfloat16* dst) {
            const int k0 = cc * TC_KC + fslice * 16;
            uint32_t wv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float v2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kp = k0 + 2 * e + h;
                    const int f = kp / PTS, j = kp - f * PTS;
                    v2[h] = (kp < KP && j < NP) ? x[j * F + f] : 0.f;
                }
                wv[e] = pack_bf16(v2[0], v2[1]);
            }
            *reinterpret_cast<uint4*>(dst + canon_off(frow, fslice * 16, TC_KC)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            *reinterpret_cast<uint4*>(dst + canon_off(frow, fslice * 16 + 8, TC_KC)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
        };
        const float zz = mlp_tile_tc<D>(st, s, abuf, hbuf, fill);
        if (!__syncthreads_and(st.ok ? 1 : 0)) {
            if (threadIdx.x == 0) atomicOr(err, 1);
            break;
        }
        if (warp < 4) {
            const long ro = tile * TC_M + warp * 32 + lane;
            if (ro < n) z[ro] = zz;
        }
    }
    tc_teardown(st);
}

// ---------------------------------------------------------------------------
// FP32 training kernels (rows of a minibatch selected by idx)
// ---------------------------------------------------------------------------
__global__ void k_dense_relu(const float* __restrict__ In, const int* __restrict__ idx, int n, int I,
                             const float* __restrict__ W, const float* __restrict__ b, float* __restrict__ H) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * MLP_H) return;
    const int r = (int)(t / MLP_H), o = (int)(t % MLP_H);
    const float* x = In + (long)(idx ? idx[r] : r) * I;
    const float* wr = W + (long)o * I;
    float acc = b[o];
    for (int k = 0; k < I; ++k) acc += x[k] * wr[k];
    H[t] = fmaxf(acc, 0.f);
}

__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

__global__ void k_out(const float* __restrict__ H2, int n, const float* __restrict__ w3, const float* __restrict__ b3,
                      const float* __restrict__ y, const int* __restrict__ idx, float pw, float* __restrict__ dz,
                      float* __restrict__ lossv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float z = b3[0];
    for (int j = 0; j < MLP_H; ++j) z += H2[(long)r * MLP_H + j] * w3[j];
    const float yy = y[idx ? idx[r] : r];
    const float sg = 0.5f * (1.f + tanhf(0.5f * z));
    lossv[r] = pw * yy * softplus(-z) + (1.f - yy) * softplus(z);
    dz[r] = (pw * yy * (sg - 1.f) + (1.f - yy) * sg) / (float)n;
}

// dH = (dOut @ W) * (H > 0); dOut (n x O), W (O x 64)
__global__ void k_back_hidden(const float* __restrict__ dOut, int n, int O, const float* __restrict__ W,
                              const float* __restrict__ H, float* __restrict__ dH) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * MLP_H) return;
    const int r = (int)(t / MLP_H), j = (int)(t % MLP_H);
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc += dOut[(long)r * O + o] * W[(long)o * MLP_H + j];
    dH[t] = H[t] > 0.f ? acc : 0.f;
}

// dW[o][i] = sum_r dOut[r][o] In[row(r)][i]  (i < I), db[o] = sum_r dOut[r][o]
__global__ void k_wgrad(const float* __restrict__ dOut, int n, int O, const float* __restrict__ In,
                        const int* __restrict__ idx, int I, float* __restrict__ dW, float* __restrict__ db) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)O * (I + 1)) return;
    const int o = (int)(t / (I + 1)), i = (int)(t % (I + 1));
    float acc = 0.f;
    if (i < I) {
        for (int r = 0; r < n; ++r) acc += dOut[(long)r * O + o] * In[(long)(idx ? idx[r] : r) * I + i];
        dW[(long)o * I + i] = acc;
    } else {
        for (int r = 0; r < n; ++r) acc += dOut[(long)r * O + o];
        db[o] = acc;
    }
}

__global__ void k_sum(const float* __restrict__ v, int n, float* __restrict__ out, float scale) {
    __shared__ float red[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] += red[0] * scale;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, long n, float lr, float c1, float c2) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gr[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// minibatch rows of an epoch: an affine permutation r -> (a r + b) mod n
__global__ void k_perm(int* idx, long n, long a, long b) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) idx[i] = (int)((a * i + b) % n);
}

struct Dev {
    std::vector<void*> p;
    const amr_options_t* opt;
    ~Dev() {
        for (void* q : p) {
            if (opt && opt->dev_free) opt->dev_free(q, opt->user);
            else if (!(opt && opt->dev_alloc)) cudaFree(q);
        }
    }
    template <typename T> T* get(size_t n) {
        void* q = nullptr;
        const size_t bytes = (n * sizeof(T) + 255) / 256 * 256;
        if (opt && opt->dev_alloc) q = opt->dev_alloc(bytes, opt->user);
        else if (cudaMalloc(&q, bytes) != cudaSuccess) q = nullptr;
        if (q) p.push_back(q);
        return reinterpret_cast<T*>(q);
    }
};

cudaStream_t stream_of(const amr_options_t* o) { return o ? reinterpret_cast<cudaStream_t>(o->stream) : nullptr; }

int blocks(long n, int b = 256) { return (int)((n + b - 1) / b); }

// one forward + backward pass over `n` rows; gradient to g (flat layout)
int fwd_bwd(int D, const float* X, const int* idx, const float* y, int n, float pw, const float* w, float* g,
            float* loss_acc, float loss_scale, float* H1, float* H2, float* dz, float* lossv, float* dH1, float* dH2,
            cudaStream_t s) {
    const int K = mlp_kin(D);
    const float* W1 = w;
    const float* b1 = W1 + MLP_H * K;
    const float* W2 = b1 + MLP_H;
    const float* b2 = W2 + MLP_H * MLP_H;
    const float* w3 = b2 + MLP_H;
    const float* b3 = w3 + MLP_H;
    float* gW1 = g;
    float* gb1 = gW1 + MLP_H * K;
    float* gW2 = gb1 + MLP_H;
    float* gb2 = gW2 + MLP_H * MLP_H;
    float* gw3 = gb2 + MLP_H;
    float* gb3 = gw3 + MLP_H;
    const long nh = (long)n * MLP_H;
    k_dense_relu<<<blocks(nh), 256, 0, s>>>(X, idx, n, K, W1, b1, H1);
    k_dense_relu<<<blocks(nh), 256, 0, s>>>(H1, nullptr, n, MLP_H, W2, b2, H2);
    k_out<<<blocks(n), 256, 0, s>>>(H2, n, w3, b3, y, idx, pw, dz, lossv);
    k_wgrad<<<blocks(MLP_H + 1), 256, 0, s>>>(dz, n, 1, H2, nullptr, MLP_H, gw3, gb3);
    k_back_hidden<<<blocks(nh), 256, 0, s>>>(dz, n, 1, w3, H2, dH2);
    k_wgrad<<<blocks((long)MLP_H * (MLP_H + 1)), 256, 0, s>>>(dH2, n, MLP_H, H1, nullptr, MLP_H, gW2, gb2);
    k_back_hidden<<<blocks(nh), 256, 0, s>>>(dH2, n, MLP_H, W2, H1, dH1);
    k_wgrad<<<blocks((long)MLP_H * (K + 1)), 256, 0, s>>>(dH1, n, MLP_H, X, idx, K, gW1, gb1);
    if (loss_acc) k_sum<<<1, 256, 0, s>>>(lossv, n, loss_acc, loss_scale);
    return cudaGetLastError() == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

template <int D>
cudaError_t launch_infer(const float* X, long n, const float* w, float* z, int* err, cudaStream_t s) {
    const size_t smem = InferLayout<D>::TOTAL;
    cudaError_t e = cudaFuncSetAttribute(k_infer<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long tiles = (n + TC_M - 1) / TC_M;
    const int grid = (int)std::min<long>(tiles, (long)nsm);
    k_infer<D><<<grid, 512, smem, s>>>(X, n, w, z, err);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int amr_mlp_k(int dim) { return (dim >= 1 && dim <= 3) ? mlp_kin(dim) : AMR_ERR_ARG; }

int amr_mlp_features(int dim, double gamma, const double* samples, long n, float* X, const amr_options_t* opt) {
    if (dim < 1 || dim > 3 || !samples || !X || n <= 0) return AMR_ERR_ARG;
    cudaStream_t s = stream_of(opt);
    Dev dv{{}, opt};
    const long rows = n * 2 * dim;
    const int K = mlp_kin(dim);
    double* ds = dv.get<double>(n * 15);
    float* dx = dv.get<float>(rows * K);
    if (!ds || !dx) return AMR_ERR_CUDA;
    if (cudaMemcpyAsync(ds, samples, n * 15 * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return AMR_ERR_CUDA;
    k_features<<<(int)std::min<long>(blocks(rows * K), 65536), 256, 0, s>>>(dim, gamma, ds, n, dx);
    if (cudaGetLastError() != cudaSuccess) return AMR_ERR_CUDA;
    if (cudaMemcpyAsync(X, dx, rows * K * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return AMR_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

int amr_mlp_infer(int dim, const float* X, long n, const float* weights, float* logits, const amr_options_t* opt) {
    if (dim < 1 || dim > 3 || !X || !weights || !logits || n <= 0) return AMR_ERR_ARG;
    cudaStream_t s = stream_of(opt);
    Dev dv{{}, opt};
    const int K = mlp_kin(dim);
    const long nw = mlp_n_weights(dim);
    float* dx = dv.get<float>(n * K);
    float* dw = dv.get<float>(nw);
    float* dz = dv.get<float>(n);
    int* derr = dv.get<int>(1);
    if (!dx || !dw || !dz || !derr) return AMR_ERR_CUDA;
    cudaMemcpyAsync(dx, X, n * K * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dw, weights, nw * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(dz, 0xFF, n * sizeof(float), s);           // NaN until written
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    cudaError_t e = dim == 1 ? launch_infer<1>(dx, n, dw, dz, derr, s)
                  : dim == 2 ? launch_infer<2>(dx, n, dw, dz, derr, s) : launch_infer<3>(dx, n, dw, dz, derr, s);
    if (e != cudaSuccess) return AMR_ERR_CUDA;
    int herr = 0;
    cudaMemcpyAsync(logits, dz, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMR_ERR_CUDA;
    return herr ? AMR_ERR_TIMEOUT : AMR_OK;
}

int amr_mlp_grad(int dim, const float* X, const float* y, long n, float pw, const float* weights, float* grad,
                 float* loss, const amr_options_t* opt) {
    if (dim < 1 || dim > 3 || !X || !y || !weights || !grad || n <= 0 || n > (1 << 24)) return AMR_ERR_ARG;
    cudaStream_t s = stream_of(opt);
    Dev dv{{}, opt};
    const int K = mlp_kin(dim);
    const long nw = mlp_n_weights(dim);
    float* dx = dv.get<float>(n * K);
    float* dy = dv.get<float>(n);
    float* dw = dv.get<float>(nw);
    float* dg = dv.get<float>(nw);
    float* H1 = dv.get<float>(n * MLP_H);
    float* H2 = dv.get<float>(n * MLP_H);
    float* dH1 = dv.get<float>(n * MLP_H);
    float* dH2 = dv.get<float>(n * MLP_H);
    float* dz = dv.get<float>(n);
    float* lv = dv.get<float>(n);
    float* la = dv.get<float>(1);
    if (!dx || !dy || !dw || !dg || !H1 || !H2 || !dH1 || !dH2 || !dz || !lv || !la) return AMR_ERR_CUDA;
    cudaMemcpyAsync(dx, X, n * K * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dy, y, n * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dw, weights, nw * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(la, 0, sizeof(float), s);
    if (fwd_bwd(dim, dx, nullptr, dy, (int)n, pw, dw, dg, la, 1.0f / (float)n, H1, H2, dz, lv, dH1, dH2, s))
        return AMR_ERR_CUDA;
    cudaMemcpyAsync(grad, dg, nw * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (loss) cudaMemcpyAsync(loss, la, sizeof(float), cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

int amr_mlp_train(int dim, const float* X, const float* y, long n, float pw, int epochs, int batch, float lr,
                  uint64_t seed, float* weights, float* loss_hist, const amr_options_t* opt) {
    if (dim < 1 || dim > 3 || !X || !y || !weights || n <= 0 || epochs <= 0 || batch <= 0 || n > (1L << 30))
        return AMR_ERR_ARG;
    cudaStream_t s = stream_of(opt);
    Dev dv{{}, opt};
    const int K = mlp_kin(dim);
    const long nw = mlp_n_weights(dim);
    const int B = (int)std::min<long>(batch, n);
    float* dx = dv.get<float>(n * K);
    float* dy = dv.get<float>(n);
    float* dw = dv.get<float>(nw);
    float* dg = dv.get<float>(nw);
    float* m = dv.get<float>(nw);
    float* v = dv.get<float>(nw);
    int* idx = dv.get<int>(n);
    float* H1 = dv.get<float>((long)B * MLP_H);
    float* H2 = dv.get<float>((long)B * MLP_H);
    float* dH1 = dv.get<float>((long)B * MLP_H);
    float* dH2 = dv.get<float>((long)B * MLP_H);
    float* dz = dv.get<float>(B);
    float* lv = dv.get<float>(B);
    float* la = dv.get<float>(epochs);
    if (!dx || !dy || !dw || !dg || !m || !v || !idx || !H1 || !H2 || !dH1 || !dH2 || !dz || !lv || !la)
        return AMR_ERR_CUDA;
    cudaMemcpyAsync(dx, X, n * K * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dy, y, n * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dw, weights, nw * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(m, 0, nw * sizeof(float), s);
    cudaMemsetAsync(v, 0, nw * sizeof(float), s);
    cudaMemsetAsync(la, 0, epochs * sizeof(float), s);
    long step = 0;
    const long nb = n / B;            // full minibatches per epoch
    for (int ep = 0; ep < epochs; ++ep) {
        // affine permutation with a multiplier coprime to n, from a SplitMix64 stream
        uint64_t z = seed + (uint64_t)(ep + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        long a = (long)(z % (uint64_t)n) | 1;
        auto gcd = [](long p, long q) { while (q) { long r = p % q; p = q; q = r; } return p; };
        while (gcd(a, n) != 1) a += 2;
        const long b = (long)((z >> 32) % (uint64_t)n);
        k_perm<<<blocks(n), 256, 0, s>>>(idx, n, a % n, b);
        for (long bi = 0; bi < nb; ++bi) {
            if (fwd_bwd(dim, dx, idx + bi * B, dy, B, pw, dw, dg, la + ep, 1.0f / (float)(B * nb), H1, H2, dz, lv,
                        dH1, dH2, s))
                return AMR_ERR_CUDA;
            ++step;
            const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
            k_adam<<<blocks(nw), 256, 0, s>>>(dw, dg, m, v, nw, lr, c1, c2);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return AMR_ERR_CUDA;
    cudaMemcpyAsync(weights, dw, nw * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (loss_hist) cudaMemcpyAsync(loss_hist, la, epochs * sizeof(float), cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free gradient: amr_mlp_grad_noalloc.
//
// Some callers cannot allocate device memory: code running inside a task-based
// runtime that owns the whole device memory (a task there only gets the
// buffers the runtime maps for it, and an allocation behind the runtime's back
// can fail or fragment its pool), code issuing work while a CUDA stream
// capture is in progress (allocation is not allowed there), and real-time
// loops where an allocation may synchronise the device. For them the hidden
// activations of the forward/backward pass live in the fixed array below,
// which every GPU that loads this library holds until the process exits:
// 4 x 2048 x 64 + 2 x 2048 + 64 floats (about 2.1 MB).
// ---------------------------------------------------------------------------
namespace {
constexpr long NOALLOC_ROWS = AMR_MLP_NOALLOC_MAX_ROWS;
constexpr size_t NOALLOC_FLOATS = 4 * NOALLOC_ROWS * MLP_H + 2 * NOALLOC_ROWS + 64;
}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

namespace {
std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on device `dev` (current). In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress and cached.
float* noalloc_scratch(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev >= 0 && dev < NOALLOC_MAX_DEVICES && g_noalloc_ptr[dev]) return g_noalloc_ptr[dev];
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    if (dev >= 0 && dev < NOALLOC_MAX_DEVICES) g_noalloc_ptr[dev] = reinterpret_cast<float*>(p);
    return reinterpret_cast<float*>(p);
}
}  // namespace

extern "C" int amr_mlp_grad_noalloc(int dim, const float* X, const float* y, long n, float pos_weight,
                                    const float* weights, float* grad, float* loss, void* stream) {
    if (dim < 1 || dim > 3 || !X || !y || !weights || !grad || !loss || n <= 0) return AMR_ERR_ARG;
    if (n > AMR_MLP_NOALLOC_MAX_ROWS) return AMR_ERR_ARG;      // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AMR_ERR_CUDA;
    float* base = noalloc_scratch(dev);
    if (!base) return AMR_ERR_CUDA;
    const size_t hs = (size_t)NOALLOC_ROWS * MLP_H;
    float* H1 = base;
    float* H2 = base + hs;
    float* dH1 = base + 2 * hs;
    float* dH2 = base + 3 * hs;
    float* dz = base + 4 * hs;
    float* lv = dz + NOALLOC_ROWS;
    float* lacc = lv + NOALLOC_ROWS;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the loss accumulator keeps the previous call's value: clear it
    if (cudaMemsetAsync(lacc, 0, sizeof(float), s) != cudaSuccess) return AMR_ERR_CUDA;
    if (fwd_bwd(dim, X, nullptr, y, (int)n, pos_weight, weights, grad, lacc, 1.0f / (float)n, H1, H2, dz, lv, dH1,
                dH2, s))
        return AMR_ERR_CUDA;
    if (cudaMemcpyAsync(loss, lacc, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return AMR_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}
