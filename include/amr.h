/*
 * amr.h -- C ABI of the GB300 patch-based AMR Euler library (libamr).
 *
 * The library advances the compressible Euler equations of a calorically
 * perfect gas (Sec. 3.1, Eqs. 1-7) on a patch hierarchy (Sec. 4.2): every
 * patch has the same N^d cells plus 3 ghost layers per side, level-0 patches
 * form a Cartesian layout and each is the root of a binary tree / quadtree /
 * octree with refinement ratio 2 (Sec. 4.3). One call to amr_step advances
 * the hierarchy by one SSP-RK3 step (Sec. 3.2), all levels with the same dt:
 * every leaf patch with the characteristic WENO5-JS interpolation and the
 * Rusanov flux (Eqs. 10-12; options: the HLLC flux, or the central schemes
 * of Eqs. 8-9 for shock-free flows), every patch with children by
 * restriction from them after each stage; amr_regrid applies the refinement
 * requests under rules R1/R2 with Algorithm 1 and the coarsening rule of
 * Sec. 4.3.
 *
 * Conventions for every entry point:
 *   - return value: AMR_OK (0) or a negative AMR_ERR_* code; no exception or
 *     longjmp crosses the ABI. On error amr_last_error(ctx) holds a message.
 *   - a call that fails leaves the hierarchy and the state as they were,
 *     except AMR_ERR_CUDA and AMR_ERR_NONFINITE, after which only
 *     amr_get_*, amr_last_error and amr_destroy may be called.
 *   - lists are in canonical order: level, then lexicographic (z, y, x)
 *     patch coordinates. Slot (pool) indices are never exposed.
 *   - host buffers are owned by the caller; a NULL output pointer with a
 *     non-NULL count pointer asks for the size only (two-call protocol).
 *   - device memory comes from the caller's allocator hook (opt->dev_alloc)
 *     or cudaMalloc when the hook is NULL; work is issued on opt->stream.
 *   - the library is not thread-safe per context.
 */
#ifndef AMR_H
#define AMR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define AMR_OK             0
#define AMR_ERR_ARG       -1   /* invalid argument */
#define AMR_ERR_POOL      -2   /* patch pool capacity exceeded (regrid left unchanged) */
#define AMR_ERR_CUDA      -3   /* a CUDA call failed */
#define AMR_ERR_NONFINITE -4   /* non-positive density or pressure, or a non-finite wave speed */
#define AMR_ERR_TIMEOUT   -5   /* a bounded device wait gave up */
#define AMR_ERR_STATE     -6   /* call not allowed in the current state */
#define AMR_ERR_MESH      -7   /* a patch set that breaks R1/R2 or the tree structure */
#define AMR_ERR_IO        -8   /* a checkpoint file could not be written or read, or does not match */

/* boundary kinds, per dimension and side */
#define AMR_BC_OUTFLOW     0   /* ghost = nearest interior layer */
#define AMR_BC_REFLECT     1   /* mirror ghost k <-> interior -1-k, normal momentum negated */
#define AMR_BC_PERIODIC    2   /* both sides of a dimension must be periodic */
#define AMR_BC_DMR_INFLOW  3   /* double Mach reflection: post-shock state */
#define AMR_BC_DMR_BOTTOM  4   /* post-shock for x < 1/6, reflecting wall beyond */
#define AMR_BC_DMR_TOP     5   /* post-/pre-shock by the exact shock x_s(t) = 1/6 + (1+20t)/sqrt(3) */

/* initial conditions (point-sampled at cell centres) */
#define AMR_IC_SOD          0  /* x < 0.5: (1, 0, 1), else (0.125, 0, 0.1) */
#define AMR_IC_SHU_OSHER    1  /* x < -4: (3.857143, 2.629369, 10.33333), else (1 + 0.2 sin 5x, 0, 1) */
#define AMR_IC_RIEMANN2D    2  /* four quadrants split at x = y = 0.5 */
#define AMR_IC_DMR          3  /* Mach-10 shock x = 1/6 + y/sqrt(3) into (1.4, 0, 0, 1) */
#define AMR_IC_BLAST3D      4  /* p = 100 inside r < 0.1 of the box centre, 0.1 outside; seeded rho perturbation */
#define AMR_IC_IMPLOSION    5  /* Sec. 6, Eq. 13: |x| + |y| < 0.15: (0.125, 0.140), else (1, 1) */
#define AMR_IC_DENSITY_WAVE 6  /* rho = 1 + 0.2 sin(2 pi x), u_x = 1, p = 1 */
#define AMR_IC_CONSTANT     7  /* rho = 1, u = (0.3, -0.2, 0.1), p = 1 */
#define AMR_IC_SHEAR_LAYER  8  /* Sec. 6: periodic shear layers at y = -+0.15 in (-0.3, 0.3)^2: band rho 1, outer
                                  rho 2, p 1, u = -+dU/2 with dU = 0.7 (c1 + c2), tanh profiles of width 0.01;
                                  v = 0.05 sin(2 pi 5 (x + 0.3) / 0.6) times Gaussians of width 0.02 at the layers */

/* refinement indicators */
#define AMR_FLAG_PLAIN 0       /* relative-jump sensor on rho and p over the patch band [-2, N+1]^d */
#define AMR_FLAG_MLP   1       /* learned indicator (BF16 tensor cores) over the band [-1, N]^d */

/* execution modes */
#define AMR_MODE_BATCHED   0   /* one persistent launch per kernel over all patches, CUDA graph */
#define AMR_MODE_PER_PATCH 1   /* one launch per patch per operation (task-per-patch baseline) */

typedef struct amr_ctx amr_ctx;

/* Computational domain: dim in {1,2,3}; [lo, hi] per dimension (unused
 * dimensions ignored); boundary kind per dimension and side (AMR_BC_*). */
typedef struct {
    int dim;
    double lo[3], hi[3];
    int bc_lo[3], bc_hi[3];
} amr_domain_t;

/* Options. Zero-initialise and set what you need; amr_default_options fills
 * the defaults (FP64, CFL 0.5, plain flags, thresholds 0.05, batched). */
typedef struct {
    int precision;        /* 64 (FP64 storage and arithmetic) or 32 (FP32 storage, stencil
                             arithmetic, CFL and flag tests; restriction sums carried error-free
                             as FP32 pairs and rounded once; FP64 conservation sums and CFL
                             maximum) */
    double cfl;           /* CFL number of the step (Sec. 3.1: c sets the step size) */
    double t_end;         /* > 0: the step is clipped so t never exceeds t_end */
    int flagger;          /* AMR_FLAG_PLAIN or AMR_FLAG_MLP */
    double theta_rho;     /* sensor thresholds: a cell is flagged if the relative jump */
    double theta_p;       /*   |phi+ - phi-| / (phi+ + 2 phi0 + phi-) exceeds theta */
    int max_patches;      /* pool capacity; <= 0 means every level fully refined */
    uint64_t seed;        /* seed of the blast density perturbation */
    double amp;           /* amplitude of that perturbation (0.01 for the blast problem) */
    int mode;             /* AMR_MODE_BATCHED or AMR_MODE_PER_PATCH */
    int use_graph;        /* 1: capture the step of the batched mode in a CUDA graph */
    void* (*dev_alloc)(size_t bytes, void* user);   /* device allocator hook, or NULL */
    void (*dev_free)(void* ptr, void* user);
    void* user;
    void* stream;         /* cudaStream_t the library issues its work on (NULL: legacy stream) */
    const float* mlp_weights;  /* host weights of the learned indicator (layout of amr_set_mlp), copied
                                  at init; NULL: the initial hierarchy uses the plain sensor and
                                  amr_set_mlp must precede the first amr_regrid */
    long mlp_n_weights;
    int autotune;         /* 1: amr_init ends with amr_autotune on the initial hierarchy */
    int flux;             /* AMR_FLUX_RUSANOV (Sec. 3.2, Eqs. 11-12; default), AMR_FLUX_HLLC (an
                             option the method leaves open: Toro's HLLC from the same face states) or
                             AMR_FLUX_CENTRAL (Sec. 3.2's shock-free schemes: 4th-order central mid-point
                             interpolation of p, u, T (Eq. 8), the Euler flux of that edge state, and the
                             4th-order staggered divergence (Eq. 9) in conservative form) or
                             AMR_FLUX_HYBRID (face by face: the central scheme's conservative face
                             value where a shock sensor is quiet, WENO5 + Rusanov elsewhere; Sec. 3.2
                             gives the central schemes for shock-free flows and WENO for flows with
                             shocks, the per-face switch is this library's extension) */
    double mlp_keep_margin;  /* H >= 0, learned flagger only: a patch requests refinement if a band
                                cell's logit is > -R (R = mlp_refine_margin, default 0) and blocks the
                                coarsening of its parent if one is > -H (hysteresis between the two
                                decisions; H = R: the same test) */
    double theta_switch;  /* AMR_FLUX_HYBRID only: a face i+1/2 takes the WENO5 + Rusanov flux if, at
                             any pencil node k = i-1 .. i+2 and for phi = rho (= p / T) or p,
                             |phi_{k+1} - phi_{k-1}| > theta_switch (phi_{k+1} + 2 phi_k + phi_{k-1})
                             (the relative jump of the refinement sensor along the face normal);
                             else the central value. Default 0.05 */
    double mlp_refine_margin;  /* R in [0, H], learned flagger only: a patch requests refinement if a
                                  band cell's logit is > -R (0: the network's own decision, logit > 0;
                                  a larger R refines more, trading precision for recall against the
                                  plain sensor); H is mlp_keep_margin */
} amr_options_t;

#define AMR_FLUX_RUSANOV 0
#define AMR_FLUX_HLLC 1
#define AMR_FLUX_CENTRAL 2
#define AMR_FLUX_HYBRID 3

/* Launch parameters of the batched step (amr_get_tuning), in this order:
 * CTAs per SM of the ghost fill, ghost cells per ghost-fill work item, CTAs per
 * SM of the fused RHS, the reflux, the restriction, the CFL reduction and the
 * plain flagging. */
#define AMR_TUNE_GHOST_GRID 0
#define AMR_TUNE_GHOST_CHUNK 1
#define AMR_TUNE_RHS_GRID 2
#define AMR_TUNE_REFLUX_GRID 3
#define AMR_TUNE_RESTRICT_GRID 4
#define AMR_TUNE_CFL_GRID 5
#define AMR_TUNE_FLAG_GRID 6
#define AMR_TUNE_RHS_SHAPE 7    /* tile shape of the fused RHS: index of the compiled (z-chunk depth,
                                   threads per CTA, resident CTAs per SM) candidate, 0 where only one is
                                   compiled (FP32 3D 16^3 patches, Rusanov flux: 0 = four planes, 256
                                   threads, 2 CTAs; 1 = two planes, 256 threads, 3 CTAs; 2 = eight planes,
                                   512 threads, 1 CTA; 3 and 4 = shapes 0 and 2 with the halo planes
                                   copied by TMA (tensor copies on an mbarrier) while the threads stage
                                   the centre planes) */
#define AMR_TUNE_N 8

void amr_default_options(amr_options_t* opt);

/* Create a hierarchy (Sec. 4.2-4.3): level 0 is the Cartesian layout of
 * base_cells[d] / patch_size patches, filled with the initial condition
 * ic_id; then levels-1 rounds of flag -> regrid with the initial condition
 * re-sampled on new patches. ratio must be 2 (child[4] in Sec. 4.2);
 * base_cells[d] must be multiples of patch_size, patch_size in {8, 16, 32}
 * (3D: {8, 16}); levels in [1, 8]; (base_cells[d] / patch_size) << (levels - 1)
 * below 2^20; with max_patches <= 0, every level fully refined at most
 * 2^31 - 1 patches. gamma > 1. *out receives the context (also on failure,
 * for amr_last_error; destroy it). Invalid arguments give AMR_ERR_ARG before
 * any CUDA call; without a usable CUDA device the call returns AMR_ERR_CUDA
 * (there is no CPU fallback). */
int amr_init(amr_ctx** out, const amr_domain_t* dom, double gamma, const int base_cells[3],
             int levels, int ratio, int patch_size, int ic_id, const amr_options_t* opt);

/* One SSP-RK3 step (Sec. 3.2) of the hierarchy (leaves advanced, patches with
 * children restricted from them after each stage). dt <= 0 takes
 * dt = CFL / max over leaf cells of sum_d (|u_d| + c) / dx_d (clipped to
 * t_end); dt > 0 is used as given. dt_used (may be NULL) receives the step;
 * passing NULL avoids a device-to-host synchronisation. */
int amr_step(amr_ctx* ctx, double dt, double* dt_used);

/* n_steps CFL steps (amr_step with dt <= 0): the production loop, with no
 * return to the caller between steps. regrid is the regrid interval K: 0
 * never regrids; K >= 1 runs amr_regrid after every K-th step taken by
 * amr_advance since the context's last regrid (the count carries over
 * between calls and restarts at every regrid, amr_regrid included, so
 * repeated amr_advance(ctx, 1, K) calls regrid as one amr_advance(ctx, n, K)
 * does); K = 1 regrids after every step. The refinement criterion is not
 * evaluated between regrids, so with K > 1 a feature can move up to K steps
 * before the mesh follows it (Sec. 4.3 leaves the regrid frequency to the
 * runtime program). Stops at the first error and returns it (the steps before
 * it stand); n_steps < 0 or regrid < 0 is AMR_ERR_ARG. The only host
 * synchronisation is each regrid's read-back of the refinement requests. */
int amr_advance(amr_ctx* ctx, int n_steps, int regrid);

/* Flag (plain sensor or learned indicator), close the requests under R2
 * (Algorithm 1), coarsen by the Sec. 4.3 rule, and fill new patches by
 * limited-linear prolongation from their parents. */
int amr_regrid(amr_ctx* ctx);

/* Patches of one level: *n_patches receives their number; coords (may be
 * NULL) receives n x dim integer patch coordinates; data (may be NULL)
 * receives n x (dim+2) x N^d interior values as double, variables
 * (rho, rho u_0.., rho e), cells in (z, y, x) order. A data buffer in
 * page-locked host memory (cudaHostAlloc, cudaHostRegister, PyTorch's pinned
 * memory) is written by the device directly, in one kernel; any other buffer
 * through the library's device staging buffer. Either way the buffer must
 * hold the whole level. */
int amr_get_level(amr_ctx* ctx, int level, int* n_patches, int* coords, double* data);

/* Diagnostics: time, sum over leaf cells of U times the cell volume (FP64,
 * dim+2 entries), patches per level (8 entries, unused ones 0). Any pointer
 * may be NULL. */
int amr_get_diag(amr_ctx* ctx, double* t, double cons_sums[5], int patches_per_level[8]);

/* Replace the hierarchy and state: n patches given by level (n ints), coords
 * (n x dim ints) and interiors (n x (dim+2) x N^d doubles, layout of
 * amr_get_level), and the time t. The set must contain every level-0 patch,
 * complete sibling groups, and satisfy R2; otherwise AMR_ERR_MESH. Interiors
 * in page-locked host memory are read by the device in place; others are
 * copied through the staging buffer (as in amr_get_level). */
int amr_set_state(amr_ctx* ctx, int n, const int* levels, const int* coords,
                  const double* data, double t);

/* Checkpoint and restart. amr_checkpoint writes the hierarchy to a file: the
 * 8-byte tag "AMRCKPT1", then int32 dim, N, levels, dim+2, n (patches), the
 * double time t, int32 levels[n], int32 coords[n x dim] and double
 * interiors[n x (dim+2) x N^d] in canonical order (layout of amr_get_level),
 * host byte order. The values are exact images of the state (FP32 fields
 * widen exactly). amr_restore reads such a file into a context created with
 * the same dimension, patch size and number of levels (either precision; an
 * FP64 file restored into an FP32 context is rounded) and replaces its
 * hierarchy, state and time as amr_set_state does, so a run continued from
 * it repeats the original run's results. A file that cannot be opened, is
 * short, or has another tag or shape gives AMR_ERR_IO and leaves the context
 * unchanged. */
int amr_checkpoint(amr_ctx* ctx, const char* path);
int amr_restore(amr_ctx* ctx, const char* path);

/* Refinement requests and coarsening candidates of the current state without
 * changing it: keys are (level, cx, cy, cz) quadruples in canonical order.
 * Two-call protocol on each list (NULL list: size only). */
int amr_get_requests(amr_ctx* ctx, int* n_refine, int* refine_keys,
                     int* n_coarsen, int* coarsen_keys);

/* The refinement requests the plain relative-jump sensor makes on the current
 * hierarchy and state, whatever flagger the context regrids with: the leaf
 * patches below the finest level that the plain criterion would refine but
 * that are not refined. With the learned indicator, or with a regrid interval
 * above 1 (amr_advance), this counts how far the mesh lags the plain
 * criterion (unmet requests; the paper leaves the refinement criterion and its
 * frequency to the runtime program, Sec. 4.2-4.3). Fills the ghost cells of
 * the current state as a regrid does; changes neither the hierarchy nor the
 * interiors. *n_refine receives the count; NULL is AMR_ERR_ARG. */
int amr_plain_requests(amr_ctx* ctx, int* n_refine);

/* The mesh half of a regrid on a caller's hierarchy, on the host alone (no
 * context, no GPU; Sec. 4.3). Starting from the hierarchy `keys` (n rows of
 * (level, cx, cy, cz), any order, coordinates of unused dimensions 0),
 * Algorithm 1 is applied to each refinement request in canonical order (a
 * request for a patch that is absent, has children or lies on level
 * max_level is skipped), then the coarsening rule of Sec. 4.3 to the
 * candidates, repeated until it accepts none (children created by this call
 * stay): the steps amr_regrid takes once it has its requests, so a host-side
 * planner can foresee a regrid's outcome.
 * dim 1..3; base_patches: level-0 patches per dimension (entries beyond dim
 * ignored); periodic: 0 or 1 per dimension; max_level: the finest level
 * (levels - 1, at most 7), with base_patches[d] << max_level below 2^20.
 * refine_keys, candidate_keys: rows of 4 ints like keys. The resulting
 * hierarchy is written to out_keys (cap_out rows of 4 ints, canonical order);
 * *n_out receives its size, n_created and n_deleted (may be NULL) the
 * numbers of patches created and deleted. Caller-owned host arrays; nothing
 * is kept. Returns AMR_ERR_ARG for invalid sizes, a NULL array with a
 * positive count, or a key outside the level range or the domain;
 * AMR_ERR_MESH if `keys` repeats a key or breaks R1, R2 or the tree
 * structure; AMR_ERR_POOL if the result has more than cap_out rows (*n_out
 * set, out_keys untouched). */
int amr_mesh_close(int dim, const int base_patches[3], const int periodic[3], int max_level,
                   int n, const int* keys, int n_refine, const int* refine_keys,
                   int n_candidates, const int* candidate_keys,
                   int cap_out, int* n_out, int* out_keys, int* n_created, int* n_deleted);

/* The metadata tables the kernels read (Sec. 4.2: a patch's level,
 * coordinates, neighbours, parent and children), built for a caller's
 * hierarchy on the host alone (no context, no GPU), for inspection and
 * testing. keys: n >= 1 rows of (level, cx, cy, cz) forming a valid hierarchy
 * (as for amr_mesh_close); the patch of canonical index s gets slot s. The
 * tables are n_ints ints, in this order (cap = n):
 *   level[cap], coord[3 cap] (x, y, z per slot),
 *   nbr[27 cap] (entry (oz+1) 9 + (oy+1) 3 + (ox+1): the slot of the
 *     same-level patch at that offset, wrapped across periodic sides; -1 if
 *     absent, -2 outside the domain; the centre entry is the patch itself),
 *   parent[cap] (-1 on level 0), child[8 cap] (the children in (z, y, x)
 *     order, x fastest; -1 for a leaf and beyond 2^d),
 *   pflag[cap] (bit 0: has children; bit 8 + 2 d + side, side 0 low / 1
 *     high: the face takes part in a coarse-fine correction, i.e. a leaf whose
 *     neighbour across it has children, or a patch above level 0 with no
 *     same-level neighbour across it inside the domain),
 *   all_list[cap] (slots in canonical order), level_off[9] (start of each
 *     level in all_list; the total for levels beyond the last),
 *   leaf_list[cap] (leaf slots, canonical order), counts[4] (patches,
 *     leaves, correction items, new patches = 0),
 *   reflux_list[cap] (leaves with a face next to a patch with children,
 *     canonical order), reflux_fine[24 cap] (per correction item and face
 *     2 d + side, the slots of the 2^(d-1) finer patches across it in (z, y, x)
 *     order; -1 elsewhere), new_list[cap].
 * Entries past the counts are unspecified. *n_ints receives the size;
 * tables may be NULL (size only). Returns AMR_ERR_ARG or AMR_ERR_MESH as
 * amr_mesh_close does. */
int amr_mesh_tables(int dim, const int base_patches[3], const int periodic[3], int max_level,
                    int n, const int* keys, int* tables, long long* n_ints);

/* Weights of the learned indicator of dimension dim (flat float32, order
 * W1 (64 x K), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1), K = 5^d (d+2)). */
int amr_set_mlp(amr_ctx* ctx, const float* weights, long n_weights);

/* Cell-level agreement of the learned indicator with the plain sensor on the
 * band [-1, N]^d of every leaf patch (in-domain cells): counts[0..3] =
 * true positives, false positives, false negatives, true negatives. */
int amr_flag_stats(amr_ctx* ctx, long long counts[4]);

/* Training samples of a 1D context: for every in-domain band cell [-1, N]
 * of every leaf patch, the 5-point stencil of (rho, u, p) (n x 5 x 3
 * doubles) and the plain flag of its centre (n bytes). Two-call protocol. */
int amr_harvest(amr_ctx* ctx, long* n, double* samples, uint8_t* labels);

/* Per-class device timing of the batched step, for profiling: enable (1) or
 * disable (0) CUDA events around each kernel class. The step is still issued
 * through its captured CUDA graph (the events are event-record nodes of it),
 * or launch by launch when the context was created without graphs.
 * amr_get_timing synchronises and returns AMR_TIMING_SLOTS milliseconds.
 * Of the last step (CUDA events): ms[0] ghost fill, [1] fused RHS + stage
 * (with the finest level's restriction), [2] reflux, [3] restriction of the
 * coarser levels, [4] CFL reduction (0 if the step had a given
 * dt). Of the last regrid: [5] the flag kernel (plain or learned; CUDA
 * events), [6] host closure (wall), [7] table upload + new-patch fill (wall),
 * [8] the ghost fill that precedes flagging (CUDA events), [9] the whole
 * flagging phase: ghost fill, flag kernel, request compaction and read-back
 * (wall). launches (may be NULL) receives the kernel launches behind each
 * slot (0 for the wall-clock slots). */
#define AMR_TIMING_SLOTS 10
int amr_set_timing(amr_ctx* ctx, int enable);

/* Autotuner of the batched step's launch parameters (the kernels' grids, the
 * ghost-fill work-item size and the fused RHS's tile shape, "tile shapes and
 * schedules chosen by an autotuner"): on the current hierarchy, every
 * candidate of each kernel class is timed with CUDA events (best of 3 after a
 * warm-up) on scratch copies of the state (the stage arrays), and the fastest
 * is kept; the captured step graphs are dropped so that the next step uses
 * the choice. The state, time, dt and error word are left as they were (the
 * results of later steps do not depend on the choice). Synchronises. Not in
 * the paper (its tasks are scheduled by the Legion runtime). */
int amr_autotune(amr_ctx* ctx);
/* The launch parameters in use (AMR_TUNE_N ints, AMR_TUNE_* order) and, if
 * ms is not NULL, the best time in milliseconds the last autotune measured
 * for each (0: not measured; the two ghost-fill entries share one time). */
int amr_get_tuning(amr_ctx* ctx, int params[AMR_TUNE_N], float ms[AMR_TUNE_N]);
/* Set the launch parameters (AMR_TUNE_N ints in AMR_TUNE_* order, as
 * amr_get_tuning returns them), for instance to reuse an earlier autotune's
 * choice. CTAs per SM in [1, 64], ghost cells per work item in [32, 4096],
 * the RHS tile shape below the number of compiled candidates; otherwise
 * AMR_ERR_ARG and nothing changes. Results do not depend on the choice. */
int amr_set_tuning(amr_ctx* ctx, const int params[AMR_TUNE_N]);
int amr_get_timing(amr_ctx* ctx, double ms[AMR_TIMING_SLOTS], int launches[AMR_TIMING_SLOTS]);

/* Counters since amr_init: host-to-device and device-to-host bytes copied,
 * kernels launched (graph launches count their kernels). */
int amr_get_counters(amr_ctx* ctx, long long* h2d_bytes, long long* d2h_bytes, long long* kernels);

void amr_destroy(amr_ctx* ctx);
const char* amr_last_error(const amr_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Learned indicator network (K -> 64 -> 64 -> 1, ReLU), standalone calls.
 * Inputs are host buffers; the device work uses opt->dev_alloc / opt->stream
 * (opt may be NULL: cudaMalloc, legacy stream).
 * ------------------------------------------------------------------------- */

/* Input width K = 5^dim (dim + 2). */
int amr_mlp_k(int dim);

/* Features of 1D 5-point samples (n x 5 x 3 of rho, u, p) embedded in dim
 * dimensions along every axis and sign (2 dim rows per sample, axis-major,
 * sign -1 then +1), normalised by the centre cell. Output n*2*dim x K floats. */
int amr_mlp_features(int dim, double gamma, const double* samples, long n, float* X,
                     const amr_options_t* opt);

/* Logits of n feature rows (n x K floats) with BF16 tensor-core GEMMs and
 * FP32 accumulation. */
int amr_mlp_infer(int dim, const float* X, long n, const float* weights, float* logits,
                  const amr_options_t* opt);

/* Weighted binary cross entropy mean(pw y softplus(-z) + (1-y) softplus(z))
 * of n rows and its gradient w.r.t. the weights (FP32). */
int amr_mlp_grad(int dim, const float* X, const float* y, long n, float pos_weight,
                 const float* weights, float* grad, float* loss, const amr_options_t* opt);

/* Adam training on the device: epochs over the n rows in minibatches of
 * `batch` (order shuffled by shuffle_seed each epoch), learning rate lr.
 * weights is read as the initial point and overwritten with the result;
 * loss_hist (may be NULL) receives the mean loss of each epoch. */
int amr_mlp_train(int dim, const float* X, const float* y, long n, float pos_weight,
                  int epochs, int batch, float lr, uint64_t shuffle_seed,
                  float* weights, float* loss_hist, const amr_options_t* opt);

/* ---------------------------------------------------------------------------
 * Allocation-free variant of amr_mlp_grad (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory: code running inside a
 * task-based runtime that owns all device memory and only maps buffers for
 * its tasks, and real-time loops where an allocation could synchronise the
 * device.
 * X (n x K floats), y (n floats), weights (flat layout of amr_set_mlp), grad
 * (same layout, output) and loss (one float, output) are DEVICE pointers owned
 * by the caller; work is issued on `stream` (a cudaStream_t, NULL = legacy
 * stream) and not synchronised. The hidden activations use a fixed scratch
 * array compiled into the library (about 2.1 MB on every GPU that loads it,
 * held until the process exits), so n is limited to
 * AMR_MLP_NOALLOC_MAX_ROWS; larger n returns AMR_ERR_ARG. The call allocates
 * nothing. Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture. The cached address belongs to the device's primary
 * context: after cudaDeviceReset it is stale, so do not call this function
 * in a process that has reset the device. Every call shares the one array: calls that overlap on the
 * GPU (other streams, other host threads) race and give wrong results.
 * Returns AMR_OK, AMR_ERR_ARG or AMR_ERR_CUDA. */
#define AMR_MLP_NOALLOC_MAX_ROWS 2048
int amr_mlp_grad_noalloc(int dim, const float* X, const float* y, long n, float pos_weight,
                         const float* weights, float* grad, float* loss, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AMR_H */
