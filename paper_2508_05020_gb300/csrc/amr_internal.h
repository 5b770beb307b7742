// Internal declarations shared by the translation units of libamr.
//
// Device layout of the patch pool (the patch region of Sec. 4.2, which spans
// interior and ghost points): one array per state,
//     U[slot][var][z][y][x],  z in [0, SZ), y in [0, SY), x in [0, SX),
// with SZ = N + 6 in 3D (else 1), SY = N + 6 in 2D/3D (else 1). A row holds
// XP pad elements, then the N + 6 cells of the row (3 ghosts, N interior, 3
// ghosts), then pad up to the x pitch SX, a multiple of 8 elements. XP puts
// the first interior cell of every row on a 32-byte boundary (FP32: XP = 5,
// FP64: XP = 1), so a row's N interior cells fill whole 32-byte sectors and
// are read as aligned 16-byte vectors. Local cell index l in [-3, N+3) maps to
// slot index l + 3 (the x element l + 3 + XP). A patch's data is contiguous
// (nv * SZ * SY * SX elements).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace amr {

constexpr int G = 3;            // ghost layers: the WENO5 pencil reaches i-2 .. i+3
constexpr int MAXL = 8;         // maximum number of levels
constexpr int NBR = 27;         // neighbour table entries per slot ({-1,0,1}^3)

// device error bits (DevTime::err)
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_MESH = 2;
constexpr int ERR_TIMEOUT = 4;        // a bounded device wait gave up

// limit of a bounded wait of the tensor-core pipeline, in SM clock cycles
// (about two seconds)
constexpr long long TC_WAIT_CYCLES = 1ll << 32;

// Per-step scalars kept on the device so that a captured step needs no host input.
struct DevTime {
    double t;                   // time at the start of the step
    double dt;                  // step in use
    unsigned long long lam;     // bit pattern of the max wave-speed sum (non-negative double)
    int err;                    // ERR_* bits
    int cancel;                 // nonzero: the kernels of a step return at once (set by the request
                                // compaction when the mesh may change; a step issued ahead of that
                                // decision is then void and issued again)
};

// Read-only description of the grid and the metadata tables, passed by value.
struct Grid {
    int dim, N, L, nv;
    int SX, SY, SZ;
    int XP;                     // pad elements before the first ghost of a row
    long long slot_elems;       // SZ * SY * SX
    long long patch_elems;      // nv * slot_elems
    int cap;                    // pool capacity (slots)
    int ext[MAXL][3];           // patches per dimension at each level
    double dx[MAXL][3];         // cell size per level and dimension
    double lo[3];
    int periodic[3];
    int bc[3][2];               // AMR_BC_* per dimension and side
    double gamma;
    double cfl, t_end;
    double theta_rho, theta_p;
    int ic;
    int flux;                   // AMR_FLUX_*
    double theta_sw;            // AMR_FLUX_HYBRID: threshold of the face's shock sensor
    int rhs_shape;              // tile-shape candidate of the fused RHS (AMR_TUNE_RHS_SHAPE)
    float mlp_keep;             // learned flagger: a logit above -mlp_keep sets the keep bit
    float mlp_refine;           // learned flagger: a logit above -mlp_refine sets the refine bit
    long long tc_wait;          // learned flagger: limit of a role's pipeline wait (SM cycles)
    int tc_test;                // learned flagger, tests of the timeout path only: nonzero makes
                                //   the MMA thread withhold the epilogue's accumulator signal, so
                                //   the epilogue's first wait cannot complete
    unsigned long long seed;
    double amp;
    int base_cells[3];
    double dmr_pre[4], dmr_post[4];   // double-Mach (rho, u, v, p) ahead of / behind the shock
    // metadata, indexed by slot
    const int* level;           // [cap]
    const int* coord;           // [cap * 3]
    const int* nbr;             // [cap * 27]: slot at offset (ox,oy,oz), index (oz+1)*9+(oy+1)*3+(ox+1);
                                //   -1 = in-domain position without a patch, -2 = outside the domain
    const int* parent;          // [cap]
    const int* child;           // [cap * 8]: children in (z, y, x)-lexicographic order, -1 if none
    const int* pflag;           // [cap]: bit 0 has children; bits 8.. save-face mask (bit 8 + 2 d + side)
    // work lists (device), canonical order
    const int* all_list;        // every active slot; level l occupies [level_off[l], level_off[l+1])
    const int* level_off;       // [L + 1]
    const int* leaf_list;       // leaf slots
    const int* counts;          // [0] n_all, [1] n_leaf, [2] n_reflux, [3] n_new
    const int* reflux_list;     // leaf slots with at least one coarse-fine face
    const int* reflux_fine;     // [n_reflux * 6 * 4]: fine slots across each face (-1 if none)
    const int* new_list;        // slots created by the last regrid
    const int* ghost_tab;       // packed local (x,y,z)+3 of every ghost cell of a slot (slot order),
                                //   followed by the n_ghost_face face ghosts box by box
    int n_ghost;                // ghost cells of a slot
    int n_ghost_face;           // of them outside the interior along one dimension only (face ghosts)
    DevTime* time;
};

// Kernel set of one storage precision. Implemented for float and double in
// amr_f32.cu / amr_f64.cu; the FP64 unit is compiled without FMA contraction.
template <typename T>
struct Kernels {
    // one-time kernel attributes (dynamic shared memory); call before any capture
    static cudaError_t prepare(const Grid& g);
    static cudaError_t prepare_mlp(const Grid& g);
    // ghost cells of every patch of `level` (same-level copy, prolongation,
    // physical boundaries) at time t + tfrac * dt
    // stage_only: the face ghosts without a same-level neighbour across their
    // face (all a stage reads from a slot's ghost region: the RHS and the
    // prolongation read same-level neighbours' interiors directly); else every
    // ghost cell (what the flag stencils read)
    static cudaError_t ghost_fill(const Grid& g, T* U, int level, double tfrac, int grid,
                                  cudaStream_t s, int one_slot, int chunk = 512, bool stage_only = false);
    // compiled tile-shape candidates of the fused RHS for this grid and flux
    static int rhs_shapes(const Grid& g);
    // RHS + SSP-RK3 stage of every patch (or one patch if one_slot >= 0);
    // fuse_restrict: patches of the finest level L - 1 also restrict their
    // output into their parents (the restriction of level L - 1 is then done)
    // tmap: the tensor map (CUtensorMap) of the state array Us, needed by the
    // tile shapes that copy halo planes with TMA (else cudaErrorInvalidValue)
    static cudaError_t rhs_stage(const Grid& g, const T* Us, const T* U0, T* Uout, T* faces,
                                 int stage, int grid, cudaStream_t s, int one_slot, int fuse_restrict = 0,
                                 const void* tmap = nullptr);
    static cudaError_t reflux(const Grid& g, T* Uout, const T* faces, int stage, int grid,
                              cudaStream_t s, int one_slot);
    // covered cells of level-1 patches from the children of level `level`
    static cudaError_t restrict_level(const Grid& g, T* U, int level, int grid, cudaStream_t s,
                                      int one_slot);
    static cudaError_t cfl(const Grid& g, const T* U, int grid, cudaStream_t s, int one_slot);
    static cudaError_t init_ic(const Grid& g, T* U, const int* list, int n, cudaStream_t s);
    static cudaError_t prolong_new(const Grid& g, T* U, const int* list, int n, cudaStream_t s);
    static cudaError_t flag_plain(const Grid& g, const T* U, int* anyflag, int grid,
                                  cudaStream_t s);
    static cudaError_t cons_sums(const Grid& g, const T* U, double* partial, double* out,
                                 cudaStream_t s);
    static cudaError_t unpack_interiors(const Grid& g, const T* U, const int* slots, int n,
                                        double* out, cudaStream_t s);
    static cudaError_t pack_interiors(const Grid& g, T* U, const int* slots, int n,
                                      const double* in, cudaStream_t s);
    // learned indicator: per-patch any(logit > 0) on the band [-1, N]^d of leaf patches
    static cudaError_t flag_mlp(const Grid& g, const T* U, const float* w, int* anyflag,
                                int grid, cudaStream_t s);
    // per-cell plain and learned flags on the band [-1, N]^d: counts[4]
    static cudaError_t flag_stats(const Grid& g, const T* U, const float* w,
                                  unsigned long long* counts, int grid, cudaStream_t s);
    static cudaError_t harvest(const Grid& g, const T* U, int* n_out, double* samples,
                               unsigned char* labels, int max_n, cudaStream_t s);
};

// dt finalisation and request compaction (precision-independent, amr_common.cu)
cudaError_t launch_finalize_dt(const Grid& g, cudaStream_t s);
cudaError_t launch_set_dt(DevTime* t, double dt, cudaStream_t s);
cudaError_t launch_advance_time(DevTime* t, cudaStream_t s);
cudaError_t launch_requests(const Grid& g, const int* anyflag, const int* rejected, int* out_refine, int* out_coarsen,
                            int* out_counts, cudaStream_t s);

// MLP pieces (amr_mlp.cu)
int mlp_k(int dim);
long mlp_n_weights(int dim);

}  // namespace amr
