// Precision-independent kernels: time-step finalisation and the compaction of
// refinement requests / coarsening candidates.
#include <cuda_runtime.h>
#include "amr_internal.h"

namespace amr {

// dt = CFL / lambda_max (Sec. 3.1: the sound speed sets the step), clipped to
// t_end; the maximum is reset for the next step.
__global__ void k_finalize_dt(DevTime* tm, double cfl, double t_end) {
    if (tm->cancel) return;
    const double lam = __longlong_as_double((long long)tm->lam);
    if (!(lam > 0.0) || !(lam <= 1.0e300)) {
        tm->err |= ERR_NONFINITE;
        tm->dt = 0.0;
    } else {
        double dt = cfl / lam;
        if (t_end > 0.0) dt = fmin(dt, t_end - tm->t);
        tm->dt = dt;
    }
    tm->lam = 0ull;
}

__global__ void k_set_dt(DevTime* tm, double dt) {
    if (!tm->cancel) tm->dt = dt;
}

__global__ void k_advance_time(DevTime* tm) {
    if (!tm->cancel) tm->t = tm->t + tm->dt;
}

cudaError_t launch_finalize_dt(const Grid& g, cudaStream_t s) {
    k_finalize_dt<<<1, 1, 0, s>>>(g.time, g.cfl, g.t_end);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(DevTime* t, double dt, cudaStream_t s) {
    k_set_dt<<<1, 1, 0, s>>>(t, dt);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(DevTime* t, cudaStream_t s) {
    k_advance_time<<<1, 1, 0, s>>>(t);
    return cudaGetLastError();
}

// Requests in canonical order: refine = leaf, below the finest level, refine
// bit (1) set; coarsen = has children, all children leaves, none with the keep
// bit (2) set (the plain sensor sets both bits together). One block; an
// exclusive scan per 1024-patch chunk (warp shuffles + shared totals) keeps
// the canonical order of the compacted lists.
__global__ void __launch_bounds__(1024) k_requests(Grid g, const int* anyflag, const int* rejected,
                                                   int* out_refine, int* out_coarsen, int* out_counts) {
    __shared__ int wsum[2][32];
    __shared__ int base[2];
    const int n = g.counts[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) { base[0] = 0; base[1] = 0; }
    __syncthreads();
    for (int start = 0; start < n; start += blockDim.x) {
        const int i = start + threadIdx.x;
        int r = 0, c = 0, slot = -1;
        if (i < n) {
            slot = g.all_list[i];
            const int pf = g.pflag[slot];
            const int lev = g.level[slot];
            if (!(pf & 1)) {
                r = (lev < g.L - 1 && (anyflag[slot] & 1)) ? 1 : 0;
            } else {
                const int nch = 1 << g.dim;
                bool ok = true;
                for (int k = 0; k < nch; ++k) {
                    const int ch = g.child[slot * 8 + k];
                    if (ch < 0 || (g.pflag[ch] & 1) || (anyflag[ch] & 2)) { ok = false; break; }
                }
                c = ok ? 1 : 0;
            }
        }
        // inclusive warp scans
        int sr = r, scn = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, sr, o);
            const int b = __shfl_up_sync(0xffffffffu, scn, o);
            if (lane >= o) { sr += a; scn += b; }
        }
        if (lane == 31) { wsum[0][wid] = sr; wsum[1][wid] = scn; }
        __syncthreads();
        if (wid == 0) {
            int a = lane < (int)(blockDim.x >> 5) ? wsum[0][lane] : 0;
            int b = lane < (int)(blockDim.x >> 5) ? wsum[1][lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, a, o);
                const int y = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) { a += x; b += y; }
            }
            wsum[0][lane] = a;
            wsum[1][lane] = b;
        }
        __syncthreads();
        const int off_r = base[0] + (wid > 0 ? wsum[0][wid - 1] : 0) + sr - r;
        const int off_c = base[1] + (wid > 0 ? wsum[1][wid - 1] : 0) + scn - c;
        if (r) out_refine[off_r] = slot;
        if (c) out_coarsen[off_c] = slot;
        __syncthreads();
        if (threadIdx.x == 0) {
            base[0] += wsum[0][(blockDim.x >> 5) - 1];
            base[1] += wsum[1][(blockDim.x >> 5) - 1];
        }
        __syncthreads();
    }
    // a step issued next is void if the mesh may change: on refinement requests, or
    // coarsening candidates other than the list the host last found it could not
    // coarsen on this same hierarchy (rejected[0] = its length, -1: none)
    const int nr = base[0], nc = base[1];
    int cancel = nr > 0 ? 1 : 0;
    if (!cancel && nc > 0) {
        if (!rejected || rejected[0] != nc) {
            cancel = 1;
        } else {
            bool differ = false;
            for (int i = threadIdx.x; i < nc; i += blockDim.x) differ = differ || out_coarsen[i] != rejected[1 + i];
            cancel = __syncthreads_or(differ) ? 1 : 0;
        }
    }
    if (threadIdx.x == 0) {
        out_counts[0] = nr;
        out_counts[1] = nc;
        g.time->cancel = cancel;
    }
}

cudaError_t launch_requests(const Grid& g, const int* anyflag, const int* rejected, int* out_refine,
                            int* out_coarsen, int* out_counts, cudaStream_t s) {
    k_requests<<<1, 1024, 0, s>>>(g, anyflag, rejected, out_refine, out_coarsen, out_counts);
    return cudaGetLastError();
}

}  // namespace amr
