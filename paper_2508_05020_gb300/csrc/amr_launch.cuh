// Kernel launchers of one storage precision: dispatch on (dimension, patch
// size) to the template instances of amr_kernels.cuh. Included once by each
// precision unit (amr_f32.cu, amr_f64.cu) with AMR_T set to its type.
#pragma once
#include "amr_kernels.cuh"

namespace amr {

// chunk depth (3D), block size and resident CTAs per SM of the fused RHS
// kernel: candidate V of a precision, dimension and patch size
template <typename T, int D, int N, int V = 0> struct RhsCfg {
    // 3D FP32 with 16^3 patches: four-plane chunks (113 KB of staging and face
    // buffer), two CTAs of at most 128 registers per SM; otherwise two-plane
    // chunks
    static constexpr int DZ = D == 3 ? (sizeof(T) == 4 && N == 16 ? 4 : 2) : 1;
    static constexpr int NTH = D == 1 ? 64 : 256;
    static constexpr int MINB = (D == 3 && sizeof(T) == 4) ? (N == 16 ? 2 : 3) : 1;
    static constexpr bool TMA = false;
};
// the other candidates of FP32 3D 16^3 patches: two-plane chunks (72 KB) at
// three CTAs of at most 80 registers per SM (more warps to hide the staging
// loads), and eight-plane chunks (195 KB) of 512 threads at one CTA per SM
// (fewer halo planes staged per interior plane); candidates 3 and 4 are 0 and 2
// with the halo planes brought in by tensor copies (TMA) while the threads
// stage the centre planes
template <> struct RhsCfg<float, 3, 16, 1> {
    static constexpr int DZ = 2, NTH = 256, MINB = 3;
    static constexpr bool TMA = false;
};
template <> struct RhsCfg<float, 3, 16, 2> {
    static constexpr int DZ = 8, NTH = 512, MINB = 1;
    static constexpr bool TMA = false;
};
template <> struct RhsCfg<float, 3, 16, 3> {
    static constexpr int DZ = 4, NTH = 256, MINB = 2;
    static constexpr bool TMA = true;
};
template <> struct RhsCfg<float, 3, 16, 4> {
    static constexpr int DZ = 8, NTH = 512, MINB = 1;
    static constexpr bool TMA = true;
};
template <typename T, int D, int N, int FLUX> struct RhsShapes {
    static constexpr int n = (sizeof(T) == 4 && D == 3 && N == 16 && FLUX == AMR_FLUX_RUSANOV) ? 5 : 1;
};

#define AMR_DISPATCH(g, CALL)                                   \
    switch ((g).dim * 100 + (g).N) {                            \
    case 108: { constexpr int D = 1, N = 8; CALL; } break;      \
    case 116: { constexpr int D = 1, N = 16; CALL; } break;     \
    case 132: { constexpr int D = 1, N = 32; CALL; } break;     \
    case 208: { constexpr int D = 2, N = 8; CALL; } break;      \
    case 216: { constexpr int D = 2, N = 16; CALL; } break;     \
    case 232: { constexpr int D = 2, N = 32; CALL; } break;     \
    case 308: { constexpr int D = 3, N = 8; CALL; } break;      \
    case 316: { constexpr int D = 3, N = 16; CALL; } break;     \
    default: return cudaErrorInvalidValue;                      \
    }

inline double4 d4(const double* v) { return make_double4(v[0], v[1], v[2], v[3]); }

template <typename T, int D, int N, int FLUX, int V>
static cudaError_t rhs_launch_v(const Grid& g, const T* Us, const T* U0, T* Uout, T* faces, int stage, int grid,
                                cudaStream_t s, int one_slot, int fuse, const CUtensorMap* tmap) {
    using C = RhsCfg<T, D, N, V>;
    static const CUtensorMap none{};                     // the kernels without tensor copies ignore it
    if (C::TMA && !tmap) return cudaErrorInvalidValue;   // no tensor map of this state array
    k_rhs<T, D, N, C::DZ, C::NTH, C::MINB, FLUX, C::TMA>
        <<<grid, C::NTH, rhs_smem_bytes<T, D, N, C::DZ, FLUX, C::TMA>(), s>>>(g, Us, U0, Uout, faces, stage,
                                                                          one_slot, fuse, tmap ? *tmap : none);
    return cudaSuccess;
}

template <typename T, int D, int N, int FLUX>
static cudaError_t rhs_launch_f(const Grid& g, const T* Us, const T* U0, T* Uout, T* faces, int stage, int grid,
                                cudaStream_t s, int one_slot, int fuse, const CUtensorMap* tmap) {
    if constexpr (RhsShapes<T, D, N, FLUX>::n == 5) {
        switch (g.rhs_shape) {
        case 1: return rhs_launch_v<T, D, N, FLUX, 1>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
        case 2: return rhs_launch_v<T, D, N, FLUX, 2>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
        case 3: return rhs_launch_v<T, D, N, FLUX, 3>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
        case 4: return rhs_launch_v<T, D, N, FLUX, 4>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
        default: break;
        }
    }
    return rhs_launch_v<T, D, N, FLUX, 0>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
}

template <typename T, int D, int N>
static cudaError_t rhs_launch(const Grid& g, const T* Us, const T* U0, T* Uout, T* faces, int stage, int grid,
                              cudaStream_t s, int one_slot, int fuse, const CUtensorMap* tmap) {
    // one instantiation per flux: the Rusanov kernel carries no HLLC code
    cudaError_t e;
    if (g.flux == AMR_FLUX_CENTRAL)
        e = rhs_launch_f<T, D, N, AMR_FLUX_CENTRAL>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
    else if (g.flux == AMR_FLUX_HYBRID)
        e = rhs_launch_f<T, D, N, AMR_FLUX_HYBRID>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
    else if (g.flux == AMR_FLUX_HLLC)
        e = rhs_launch_f<T, D, N, AMR_FLUX_HLLC>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
    else
        e = rhs_launch_f<T, D, N, AMR_FLUX_RUSANOV>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse, tmap);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int D, int N, int FLUX, int V>
static cudaError_t rhs_prepare_v() {
    using C = RhsCfg<T, D, N, V>;
    return cudaFuncSetAttribute(k_rhs<T, D, N, C::DZ, C::NTH, C::MINB, FLUX, C::TMA>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rhs_smem_bytes<T, D, N, C::DZ, FLUX, C::TMA>());
}

template <typename T, int D, int N, int FLUX>
static cudaError_t rhs_prepare_f() {
    cudaError_t e = rhs_prepare_v<T, D, N, FLUX, 0>();
    if constexpr (RhsShapes<T, D, N, FLUX>::n == 5) {
        if (e == cudaSuccess) e = rhs_prepare_v<T, D, N, FLUX, 1>();
        if (e == cudaSuccess) e = rhs_prepare_v<T, D, N, FLUX, 2>();
        if (e == cudaSuccess) e = rhs_prepare_v<T, D, N, FLUX, 3>();
        if (e == cudaSuccess) e = rhs_prepare_v<T, D, N, FLUX, 4>();
    }
    return e;
}

template <typename T, int D, int N>
static cudaError_t rhs_prepare() {
    cudaError_t e = rhs_prepare_f<T, D, N, AMR_FLUX_RUSANOV>();
    if (e == cudaSuccess) e = rhs_prepare_f<T, D, N, AMR_FLUX_HLLC>();
    if (e == cudaSuccess) e = rhs_prepare_f<T, D, N, AMR_FLUX_HYBRID>();
    if (e == cudaSuccess) e = rhs_prepare_f<T, D, N, AMR_FLUX_CENTRAL>();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_flag_plain<T, D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)flag_smem_bytes<T, D, N>());
}

template <typename T, int D, int N>
static int rhs_shapes_of(int flux) {
    switch (flux) {
    case AMR_FLUX_RUSANOV: return RhsShapes<T, D, N, AMR_FLUX_RUSANOV>::n;
    case AMR_FLUX_HLLC: return RhsShapes<T, D, N, AMR_FLUX_HLLC>::n;
    case AMR_FLUX_HYBRID: return RhsShapes<T, D, N, AMR_FLUX_HYBRID>::n;
    default: return RhsShapes<T, D, N, AMR_FLUX_CENTRAL>::n;
    }
}

template <typename T>
int Kernels<T>::rhs_shapes(const Grid& g) {
    switch (g.dim * 100 + g.N) {
    case 108: return rhs_shapes_of<T, 1, 8>(g.flux);
    case 116: return rhs_shapes_of<T, 1, 16>(g.flux);
    case 132: return rhs_shapes_of<T, 1, 32>(g.flux);
    case 208: return rhs_shapes_of<T, 2, 8>(g.flux);
    case 216: return rhs_shapes_of<T, 2, 16>(g.flux);
    case 232: return rhs_shapes_of<T, 2, 32>(g.flux);
    case 308: return rhs_shapes_of<T, 3, 8>(g.flux);
    case 316: return rhs_shapes_of<T, 3, 16>(g.flux);
    default: return 1;
    }
}

template <typename T>
cudaError_t Kernels<T>::prepare(const Grid& g) {
    AMR_DISPATCH(g, return (rhs_prepare<T, D, N>()));
    return cudaSuccess;
}

template <typename T>
cudaError_t Kernels<T>::ghost_fill(const Grid& g, T* U, int level, double tfrac, int grid, cudaStream_t s,
                                   int one_slot, int chunk, bool stage_only) {
    if (chunk < 32) return cudaErrorInvalidValue;
    const int n_cells = stage_only ? g.n_ghost_face : g.n_ghost;
    if (stage_only) {
        AMR_DISPATCH(g, (k_ghost<T, D, N, true><<<grid, 256, 0, s>>>(g, U, level, tfrac, one_slot, d4(g.dmr_pre),
                                                                      d4(g.dmr_post), chunk, n_cells)));
    } else {
        AMR_DISPATCH(g, (k_ghost<T, D, N, false><<<grid, 256, 0, s>>>(g, U, level, tfrac, one_slot, d4(g.dmr_pre),
                                                                       d4(g.dmr_post), chunk, n_cells)));
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::rhs_stage(const Grid& g, const T* Us, const T* U0, T* Uout, T* faces, int stage, int grid,
                                  cudaStream_t s, int one_slot, int fuse_restrict, const void* tmap) {
    AMR_DISPATCH(g, return (rhs_launch<T, D, N>(g, Us, U0, Uout, faces, stage, grid, s, one_slot, fuse_restrict,
                                                static_cast<const CUtensorMap*>(tmap))));
    return cudaSuccess;
}

template <typename T>
cudaError_t Kernels<T>::reflux(const Grid& g, T* Uout, const T* faces, int stage, int grid, cudaStream_t s,
                               int one_item) {
    AMR_DISPATCH(g, (k_reflux<T, D, N><<<grid, 256, 0, s>>>(g, Uout, faces, stage, one_item)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::restrict_level(const Grid& g, T* U, int level, int grid, cudaStream_t s, int one_slot) {
    AMR_DISPATCH(g, (k_restrict<T, D, N><<<grid, 256, 0, s>>>(g, U, level, one_slot)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::cfl(const Grid& g, const T* U, int grid, cudaStream_t s, int one_slot) {
    AMR_DISPATCH(g, (k_cfl<T, D, N><<<grid, 256, 0, s>>>(g, U, one_slot)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::init_ic(const Grid& g, T* U, const int* list, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)(((long long)n * 4096 + 255) / 256 < 65536 ? ((long long)n * 4096 + 255) / 256 : 65536);
    AMR_DISPATCH(g, (k_init_ic<T, D, N><<<grid, 256, 0, s>>>(g, U, list, n, d4(g.dmr_pre), d4(g.dmr_post))));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::prolong_new(const Grid& g, T* U, const int* list, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = n < 65536 ? n : 65536;
    AMR_DISPATCH(g, (k_prolong_new<T, D, N><<<grid, 256, 0, s>>>(g, U, list, n)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::flag_plain(const Grid& g, const T* U, int* anyflag, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(anyflag, 0, sizeof(int) * (size_t)g.cap, s);   // OR over the items
    if (e != cudaSuccess) return e;
    AMR_DISPATCH(g, (k_flag_plain<T, D, N><<<grid, 256, flag_smem_bytes<T, D, N>(), s>>>(g, U, anyflag)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::cons_sums(const Grid& g, const T* U, double* partial, double* out, cudaStream_t s) {
    AMR_DISPATCH(g, (k_cons_partial<T, D, N><<<1024, 256, 0, s>>>(g, U, partial)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (g.nv) {
    case 3: k_cons_total<3><<<1, 256, 0, s>>>(g.counts, partial, out); break;
    case 4: k_cons_total<4><<<1, 256, 0, s>>>(g.counts, partial, out); break;
    default: k_cons_total<5><<<1, 256, 0, s>>>(g.counts, partial, out); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::unpack_interiors(const Grid& g, const T* U, const int* slots, int n, double* out,
                                         cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    AMR_DISPATCH(g, (k_unpack<T, D, N><<<1024, 256, 0, s>>>(g, U, slots, n, out)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::pack_interiors(const Grid& g, T* U, const int* slots, int n, const double* in,
                                       cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    AMR_DISPATCH(g, (k_pack<T, D, N><<<1024, 256, 0, s>>>(g, U, slots, n, in)));
    return cudaGetLastError();
}

}  // namespace amr
