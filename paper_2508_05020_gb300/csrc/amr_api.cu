// C ABI of libamr (include/amr.h): context, patch pool, metadata tables,
// step sequence (batched persistent kernels in a CUDA graph, or one launch per
// patch per operation) and regrid.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "amr.h"
#include "amr_internal.h"
#include "amr_mesh.h"

using namespace amr;

// NVTX range over a scope: the host side of an entry point or a regrid phase,
// shown on the timeline of a profiler that records NVTX (no effect otherwise)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct amr_ctx {
    // configuration
    int dim = 1, N = 16, L = 1, nv = 3, precision = 64, ic = 0, mode = 0, use_graph = 1, flagger = 0;
    double gamma = 1.4;
    amr_options_t opt{};
    int base_cells[3] = {1, 1, 1};
    int cap = 0;
    int nsm = 1;
    // launch parameters of the batched step (CTAs per SM; ghost cells per work
    // item), the defaults or the autotuner's choice (AMR_TUNE_* order)
    int tune[AMR_TUNE_N] = {16, 128, 2, 4, 8, 8, 4, 0};
    float tune_ms[AMR_TUNE_N] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // hierarchy
    Mesh mesh;
    std::unordered_map<uint64_t, int> slot_of;   // key -> slot (when the mesh has no dense index)
    std::vector<int> slot_at;                      // position -> slot, -1 if none (dense index)
    int slot_hi = 0;                               // one past the highest slot handed out
    std::vector<uint64_t> key_of;        // slot -> packed key (valid if used)
    std::vector<char> used;
    std::set<int> free_slots;
    std::vector<Key> canon;              // canonical patch list
    std::vector<int> canon_slot;
    int level_off_h[MAXL + 1] = {0};
    int n_leaf = 0, n_reflux = 0;
    std::vector<int> leaf_slots, reflux_slots;
    // device memory
    std::vector<void*> allocs;
    void* U[3] = {nullptr, nullptr, nullptr};   // U0, Ua, Ub
    // tensor maps of the three state arrays (FP32 3D 16^3 patches) for the RHS
    // tile shapes that copy halo planes with TMA; tma_ok: encoded
    CUtensorMap tmap[3] = {};
    bool tma_ok = false;
    void* faces = nullptr;
    int* meta_d = nullptr;                     // all int tables, one block
    int* meta_h = nullptr;                     // pinned mirror
    size_t meta_ints = 0;
    int* anyflag = nullptr;
    int* req_d = nullptr;                      // [3 + 3 cap]: counts, refine, coarsen, rejected candidates
    int* rej_d = nullptr;                      // req_d + 2 + 2 cap: [count or -1, slots] the host could not coarsen
    int* req_h = nullptr;
    double* cons_partial = nullptr;
    double* cons_d = nullptr;
    double* dense_d = nullptr;                 // staging for get_level / set_state
    size_t dense_cap = 0;
    int* slots_d = nullptr;
    DevTime* time_d = nullptr;
    DevTime* time_h = nullptr;
    float* mlp_w = nullptr;
    long mlp_n = 0;
    int* ghost_tab = nullptr;
    int n_ghost = 0, n_ghost_face = 0;
    Grid grid{};
    // graph
    // captured step graphs by [CFL step][stage-1 ghost fill skipped]
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long long graph_kernels[2][2] = {{0, 0}, {0, 0}};
    // the ghosts of U0 hold the values the first stage's ghost fill would
    // write (a regrid filled them at the current time and left the mesh as it was)
    bool ghosts_valid = false;
    // steps amr_advance has taken since the last regrid (amr_regrid or its own)
    int since_regrid = 0;
    cudaEvent_t ev_req = nullptr;         // end of a regrid's request read-back
    std::chrono::steady_clock::time_point rg_t0{};
    // per-class CUDA-event timing of the last step (ghost, rhs, reflux, restrict, cfl);
    // inside a graph capture the events become external event-record nodes
    bool timing = false;
    bool capturing = false;
    cudaEvent_t ev[3][5] = {};
    cudaEvent_t ev_cfl[2] = {};
    cudaEvent_t ev_rg[3] = {};            // regrid: before the ghost fill, before / after the flag kernel
    double regrid_ms[3] = {0, 0, 0};      // flagging phase (wall), host closure, upload + new-patch fill
    int regrid_fill_launches = 0;
    bool regrid_timed = false;            // ev_rg hold a regrid issued while timing was on
    bool cfl_timed = false;
    // counters
    long long h2d = 0, d2h = 0, kernels = 0;
    bool broken = false;
    bool initialising = false;
    std::string err;
};

namespace {

int fail(amr_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(amr_ctx* c, cudaError_t e, const char* where) {
    if (c) c->broken = true;
    return fail(c, AMR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

void* dalloc(amr_ctx* c, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    void* p = nullptr;
    if (c->opt.dev_alloc) {
        p = c->opt.dev_alloc(bytes, c->opt.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) c->allocs.push_back(p);
    return p;
}

void dfree_all(amr_ctx* c) {
    for (void* p : c->allocs) {
        if (c->opt.dev_free) c->opt.dev_free(p, c->opt.user);
        else if (!c->opt.dev_alloc) cudaFree(p);
    }
    c->allocs.clear();
}

// DMR states from the Rankine-Hugoniot relations (Mach 10 into (1.4, 0, 0, 1)),
// post-shock velocity along (cos 30, -sin 30)
void dmr_states(double gamma, double* pre, double* post) {
    const double M = 10.0, r1 = 1.4, p1 = 1.0;
    const double c1 = std::sqrt(gamma * p1 / r1);
    const double W = M * c1;
    const double r2 = r1 * (gamma + 1.0) * M * M / ((gamma - 1.0) * M * M + 2.0);
    const double p2 = p1 * (2.0 * gamma * M * M - (gamma - 1.0)) / (gamma + 1.0);
    const double un = W * (1.0 - r1 / r2);
    const double s3 = std::sqrt(3.0);
    pre[0] = r1; pre[1] = 0.0; pre[2] = 0.0; pre[3] = p1;
    post[0] = r2; post[1] = un * (s3 * 0.5); post[2] = -(un * 0.5); post[3] = p2;
}

// offsets of the int tables inside meta_d / meta_h
struct MetaLayout {
    size_t level, coord, nbr, parent, child, pflag, all_list, level_off, leaf_list, counts, reflux_list, reflux_fine,
        new_list, total;
    explicit MetaLayout(size_t cap) {
        size_t o = 0;
        level = o; o += cap;
        coord = o; o += 3 * cap;
        nbr = o; o += (size_t)NBR * cap;
        parent = o; o += cap;
        child = o; o += 8 * cap;
        pflag = o; o += cap;
        all_list = o; o += cap;
        level_off = o; o += MAXL + 1;
        leaf_list = o; o += cap;
        counts = o; o += 4;
        reflux_list = o; o += cap;
        reflux_fine = o; o += 24 * cap;
        new_list = o; o += cap;
        total = o;
    }
};

int slot_lookup(const amr_ctx* c, const Key& k) {
    if (c->mesh.dense()) {
        const long long p = c->mesh.pos(k);
        return p < 0 ? -1 : c->slot_at[(size_t)p];
    }
    auto it = c->slot_of.find(pack(k));
    return it == c->slot_of.end() ? -1 : it->second;
}

void slot_map_clear(amr_ctx* c) {
    c->slot_of.clear();
    if (c->mesh.dense()) c->slot_at.assign((size_t)c->mesh.positions(), -1);
    else c->slot_at.clear();
}

void slot_map_set(amr_ctx* c, const Key& k, int s) {
    if (c->mesh.dense()) c->slot_at[(size_t)c->mesh.pos(k)] = s;
    else c->slot_of[pack(k)] = s;
}

// Every metadata table and work list of the host mirror (meta_h and the host
// lists) from the host mesh and slot map; host work only.
void fill_tables(amr_ctx* c, const std::vector<Key>& created) {
    const MetaLayout ml(c->cap);
    int* h = c->meta_h;
    const Mesh& m = c->mesh;
    c->canon = m.canonical();
    c->canon_slot.resize(c->canon.size());
    // only the entries of the slots in use are written (every per-slot entry
    // of each of them, below); the kernels read no other slot's entries
    for (int l = 0; l <= MAXL; ++l) c->level_off_h[l] = 0;
    c->leaf_slots.clear();
    c->reflux_slots.clear();
    int n_ref = 0;
    for (size_t i = 0; i < c->canon.size(); ++i) {
        const Key& k = c->canon[i];
        const int s = slot_lookup(c, k);
        c->canon_slot[i] = s;
        h[ml.all_list + i] = s;
        h[ml.level + s] = k.l;
        h[ml.coord + 3 * s + 0] = k.x;
        h[ml.coord + 3 * s + 1] = k.y;
        h[ml.coord + 3 * s + 2] = k.z;
        h[ml.parent + s] = k.l > 0 ? slot_lookup(c, Mesh::parent(k)) : -1;
        const bool has_ch = m.has_children(k);
        int pf = has_ch ? 1 : 0;
        {
            int* chs = h + ml.child + 8 * (size_t)s;
            for (int j = 0; j < 8; ++j) chs[j] = -1;
            if (has_ch) {                                  // (z, y, x)-lexicographic, x fastest
                const int nz = c->dim == 3 ? 2 : 1, ny = c->dim >= 2 ? 2 : 1;
                int j = 0;
                for (int sz = 0; sz < nz; ++sz)
                    for (int sy = 0; sy < ny; ++sy)
                        for (int sx = 0; sx < 2; ++sx)
                            chs[j++] = slot_lookup(c, Key{k.l + 1, 2 * k.x + sx, c->dim >= 2 ? 2 * k.y + sy : 0,
                                                          c->dim == 3 ? 2 * k.z + sz : 0});
            }
        }
        int* nb = h + ml.nbr + (size_t)NBR * s;
        for (int e = 0; e < NBR; ++e) nb[e] = -2;                // offsets in unused dimensions
        const int rz = c->dim == 3 ? 1 : 0, ry = c->dim >= 2 ? 1 : 0;
        for (int oz = -rz; oz <= rz; ++oz)
            for (int oy = -ry; oy <= ry; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    Key q{k.l, k.x + ox, k.y + oy, k.z + oz};
                    int v;
                    if (!m.wrap(q)) v = -2;
                    else v = slot_lookup(c, q);
                    nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] = v;
                }
        // coarse-fine faces: a leaf whose neighbour has children keeps its face
        // flux and takes the fine mean; a fine patch without a same-level
        // neighbour keeps its face flux for the coarse side
        bool any_ref = false;
        int fine[6][4];
        for (int f = 0; f < 6; ++f)
            for (int j = 0; j < 4; ++j) fine[f][j] = -1;       // faces of unused dimensions stay -1 too
        for (int d = 0; d < c->dim; ++d)
            for (int side = 0; side < 2; ++side) {
                Key q = k;
                int* qc[3] = {&q.x, &q.y, &q.z};
                *qc[d] += side ? 1 : -1;
                if (!m.wrap(q)) continue;
                const bool q_exists = m.exists(q);
                if (!has_ch && q_exists && m.has_children(q)) {
                    pf |= 1 << (8 + 2 * d + side);
                    any_ref = true;
                    // children of q adjacent to the face, transverse sub-positions (hi, lo)
                    std::vector<int> tdims;
                    for (int e = c->dim - 1; e >= 0; --e)
                        if (e != d) tdims.push_back(e);
                    const int nsub = 1 << (int)tdims.size();
                    for (int sidx = 0; sidx < nsub; ++sidx) {
                        Key f{q.l + 1, 2 * q.x, 2 * q.y, 2 * q.z};
                        int* fc[3] = {&f.x, &f.y, &f.z};
                        if (c->dim < 2) f.y = 0;
                        if (c->dim < 3) f.z = 0;
                        *fc[d] = 2 * (*qc[d]) + (side ? 0 : 1);
                        for (size_t t = 0; t < tdims.size(); ++t) {
                            const int bit = (sidx >> (tdims.size() - 1 - t)) & 1;   // first tdim = hi
                            *fc[tdims[t]] += bit;
                        }
                        fine[2 * d + side][sidx] = slot_lookup(c, f);
                    }
                }
                if (k.l > 0 && !q_exists) pf |= 1 << (8 + 2 * d + side);
            }
        h[ml.pflag + s] = pf;
        c->level_off_h[k.l + 1] = (int)i + 1;
        if (!has_ch) c->leaf_slots.push_back(s);
        if (any_ref) {
            h[ml.reflux_list + n_ref] = s;
            for (int f = 0; f < 6; ++f)
                for (int j = 0; j < 4; ++j) h[ml.reflux_fine + ((size_t)n_ref * 6 + f) * 4 + j] = fine[f][j];
            c->reflux_slots.push_back(s);
            ++n_ref;
        }
    }
    for (int l = 1; l <= c->L; ++l)
        if (c->level_off_h[l] < c->level_off_h[l - 1]) c->level_off_h[l] = c->level_off_h[l - 1];
    for (int l = 0; l <= MAXL; ++l) h[ml.level_off + l] = c->level_off_h[std::min(l, c->L)];
    for (size_t i = 0; i < c->leaf_slots.size(); ++i) h[ml.leaf_list + i] = c->leaf_slots[i];
    std::vector<Key> cr = created;
    std::sort(cr.begin(), cr.end(), canon_less);
    for (size_t i = 0; i < cr.size(); ++i) h[ml.new_list + i] = slot_lookup(c, cr[i]);
    c->n_leaf = (int)c->leaf_slots.size();
    c->n_reflux = n_ref;
    h[ml.counts + 0] = (int)c->canon.size();
    h[ml.counts + 1] = c->n_leaf;
    h[ml.counts + 2] = n_ref;
    h[ml.counts + 3] = (int)cr.size();
}

// Rebuild every metadata table and work list from the host mesh and upload them.
int rebuild_tables(amr_ctx* c, const std::vector<Key>& created) {
    fill_tables(c, created);
    const MetaLayout ml(c->cap);
    // the written parts only: per-slot tables up to the highest slot handed
    // out, the lists up to their lengths
    const size_t hi = (size_t)c->slot_hi, n_all = c->canon.size();
    const size_t n_new = (size_t)c->meta_h[ml.counts + 3];
    const size_t parts[][2] = {{ml.level, hi}, {ml.coord, 3 * hi}, {ml.nbr, NBR * hi}, {ml.parent, hi},
                               {ml.child, 8 * hi}, {ml.pflag, hi}, {ml.all_list, n_all},
                               {ml.level_off, MAXL + 1}, {ml.leaf_list, (size_t)c->n_leaf}, {ml.counts, 4},
                               {ml.reflux_list, (size_t)c->n_reflux}, {ml.reflux_fine, 24 * (size_t)c->n_reflux},
                               {ml.new_list, n_new}};
    size_t bytes = 0;
    for (const auto& pt : parts) {
        if (!pt[1]) continue;
        CK(cudaMemcpyAsync(c->meta_d + pt[0], c->meta_h + pt[0], pt[1] * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream),
           "upload tables");
        bytes += pt[1] * sizeof(int);
    }
    c->h2d += (long long)bytes;
    // the pinned mirror is rewritten by the next rebuild: wait for the copy
    CK(cudaStreamSynchronize(c->stream), "upload tables");
    return AMR_OK;
}

// give slots to new keys (lowest free first, canonical order), free deleted ones
void assign_slots(amr_ctx* c, const std::vector<Key>& created, const std::vector<Key>& deleted) {
    for (const auto& k : deleted) {
        const int s = slot_lookup(c, k);
        if (s < 0) continue;
        c->used[s] = 0;
        c->free_slots.insert(s);
        if (c->mesh.dense()) c->slot_at[(size_t)c->mesh.pos(k)] = -1;
        else c->slot_of.erase(pack(k));
    }
    std::vector<Key> cr = created;
    std::sort(cr.begin(), cr.end(), canon_less);
    for (const auto& k : cr) {
        const int s = *c->free_slots.begin();
        c->free_slots.erase(c->free_slots.begin());
        slot_map_set(c, k, s);
        c->key_of[s] = pack(k);
        c->used[s] = 1;
        c->slot_hi = std::max(c->slot_hi, s + 1);
    }
}

int grid_size(const amr_ctx* c, int per_sm) { return c->nsm * per_sm; }

// request-list entries read back with the counts (longer lists take a second read-back)
constexpr int REQ_READ = 2048;

void drop_graphs(amr_ctx* c) {
    for (auto& row : c->graph)
        for (auto& ex : row) {
            if (ex) cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
}

template <typename T>
T* St(amr_ctx* c, int i) { return reinterpret_cast<T*>(c->U[i]); }

// tensor map of the state array U for the RHS's halo copies (nullptr if none)
const void* tmap_of(const amr_ctx* c, const void* U) {
    if (!c->tma_ok) return nullptr;
    for (int i = 0; i < 3; ++i)
        if (c->U[i] == U) return &c->tmap[i];
    return nullptr;
}
// the RHS tile shapes 3 and 4 (FP32 3D 16^3 patches) copy halo planes with TMA
bool shape_needs_tma(const amr_ctx* c, int shape) { return c->precision == 32 && shape >= 3; }

// Tensor maps of the three FP32 state arrays, viewed as 4D tensors
// (x: SX, y: SY, z: SZ, slot x variable), boxes of N x N x G cells: the halo
// planes of a chunk of one variable. cuTensorMapEncodeTiled is taken from the
// driver through the runtime's entry-point query (no link to libcuda).
bool encode_tmaps(amr_ctx* c) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !fn || q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return false;
    }
    const Grid& g = c->grid;
    const cuuint64_t dims[4] = {(cuuint64_t)g.SX, (cuuint64_t)g.SY, (cuuint64_t)g.SZ, (cuuint64_t)c->cap * c->nv};
    const cuuint64_t strides[3] = {(cuuint64_t)g.SX * 4, (cuuint64_t)g.SX * g.SY * 4, (cuuint64_t)g.slot_elems * 4};
    const cuuint32_t box[4] = {(cuuint32_t)g.N, (cuuint32_t)g.N, (cuuint32_t)G, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int i = 0; i < 3; ++i)
        if (reinterpret_cast<Encode>(fn)(&c->tmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->U[i], dims, strides, box,
                                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    return true;
}

template <typename T>
int fill_all_levels(amr_ctx* c, T* U, double tfrac) {
    for (int l = 0; l < c->L; ++l) {
        CK(Kernels<T>::ghost_fill(c->grid, U, l, tfrac, grid_size(c, c->tune[AMR_TUNE_GHOST_GRID]), c->stream, -1,
                                  c->tune[AMR_TUNE_GHOST_CHUNK]),
           "ghost fill");
        ++c->kernels;
    }
    return AMR_OK;
}

// Enqueue one SSP-RK3 step of the batched mode (optionally with the CFL step).
template <typename T>
int enqueue_step(amr_ctx* c, bool with_cfl, bool skip_fill0, long long* nk) {
    const Grid& g = c->grid;
    long long k = 0;
    auto mark = [&](cudaEvent_t e) {
        if (!c->timing) return cudaSuccess;
        return c->capturing ? cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal)
                            : cudaEventRecord(e, c->stream);
    };
    if (with_cfl) {
        CK(mark(c->ev_cfl[0]), "event");
        CK(Kernels<T>::cfl(g, St<T>(c, 0), grid_size(c, c->tune[AMR_TUNE_CFL_GRID]), c->stream, -1), "cfl");
        CK(launch_finalize_dt(g, c->stream), "finalize dt");
        CK(mark(c->ev_cfl[1]), "event");
        k += 2;
    }
    const double tfrac[3] = {0.0, 1.0, 0.5};
    for (int s = 0; s < 3; ++s) {
        T* src = St<T>(c, s == 0 ? 0 : s);
        T* dst = St<T>(c, s == 0 ? 1 : (s == 1 ? 2 : 0));
        CK(mark(c->ev[s][0]), "event");
        for (int l = 0; l < c->L && !(s == 0 && skip_fill0); ++l) {
            CK(Kernels<T>::ghost_fill(g, src, l, tfrac[s], grid_size(c, c->tune[AMR_TUNE_GHOST_GRID]), c->stream, -1,
                                      c->tune[AMR_TUNE_GHOST_CHUNK], true),
               "ghost fill");
            ++k;
        }
        CK(mark(c->ev[s][1]), "event");
        CK(Kernels<T>::rhs_stage(g, src, St<T>(c, 0), dst, reinterpret_cast<T*>(c->faces), s,
                                 grid_size(c, c->tune[AMR_TUNE_RHS_GRID]),
                                 c->stream, -1, 1, tmap_of(c, src)),
           "rhs stage");
        CK(mark(c->ev[s][2]), "event");
        CK(Kernels<T>::reflux(g, dst, reinterpret_cast<T*>(c->faces), s, grid_size(c, c->tune[AMR_TUNE_REFLUX_GRID]),
                              c->stream, -1),
           "reflux");
        CK(mark(c->ev[s][3]), "event");
        k += 2;
        for (int l = c->L - 2; l >= 1; --l) {             // level L - 1: fused into the RHS
            CK(Kernels<T>::restrict_level(g, dst, l, grid_size(c, c->tune[AMR_TUNE_RESTRICT_GRID]), c->stream, -1),
               "restrict");
            ++k;
        }
        CK(mark(c->ev[s][4]), "event");
    }
    CK(launch_advance_time(g.time, c->stream), "advance time");
    ++k;
    if (nk) *nk = k;
    return AMR_OK;
}

// One launch per patch per operation (the task-per-patch baseline).
template <typename T>
int per_patch_step(amr_ctx* c, bool with_cfl) {
    const Grid& g = c->grid;
    if (with_cfl) {
        for (int s : c->leaf_slots) {
            CK(Kernels<T>::cfl(g, St<T>(c, 0), 4, c->stream, s), "cfl");
            ++c->kernels;
        }
        CK(launch_finalize_dt(g, c->stream), "finalize dt");
        ++c->kernels;
    }
    const double tfrac[3] = {0.0, 1.0, 0.5};
    for (int s = 0; s < 3; ++s) {
        T* src = St<T>(c, s == 0 ? 0 : s);
        T* dst = St<T>(c, s == 0 ? 1 : (s == 1 ? 2 : 0));
        for (int l = 0; l < c->L; ++l)
            for (int i = c->level_off_h[l]; i < c->level_off_h[l + 1]; ++i) {
                CK(Kernels<T>::ghost_fill(g, src, l, tfrac[s], 8, c->stream, c->canon_slot[i], 512, true),
                   "ghost fill");
                ++c->kernels;
            }
        for (size_t i = 0; i < c->canon_slot.size(); ++i) {
            CK(Kernels<T>::rhs_stage(g, src, St<T>(c, 0), dst, reinterpret_cast<T*>(c->faces), s, 8, c->stream,
                                     c->canon_slot[i], 0, tmap_of(c, src)),
               "rhs stage");
            ++c->kernels;
        }
        for (int e = 0; e < c->n_reflux; ++e) {
            CK(Kernels<T>::reflux(g, dst, reinterpret_cast<T*>(c->faces), s, 1, c->stream, e), "reflux");
            ++c->kernels;
        }
        for (int l = c->L - 1; l >= 1; --l)
            for (int i = c->level_off_h[l]; i < c->level_off_h[l + 1]; ++i) {
                CK(Kernels<T>::restrict_level(g, dst, l, 4, c->stream, c->canon_slot[i]), "restrict");
                ++c->kernels;
            }
    }
    CK(launch_advance_time(g.time, c->stream), "advance time");
    ++c->kernels;
    return AMR_OK;
}

// error bits of the time record already copied to time_h
int check_time(amr_ctx* c) {
    if (c->time_h->err & ERR_NONFINITE) {
        c->broken = true;
        return fail(c, AMR_ERR_NONFINITE, "non-positive density or pressure, or non-finite wave speed");
    }
    if (c->time_h->err & ERR_MESH) {
        c->broken = true;
        return fail(c, AMR_ERR_MESH, "prolongation source missing (R2 violated)");
    }
    if (c->time_h->err & ERR_TIMEOUT) {
        c->broken = true;
        return fail(c, AMR_ERR_TIMEOUT, "a bounded wait on the tensor cores gave up");
    }
    return AMR_OK;
}

int read_time(amr_ctx* c) {
    CK(cudaMemcpyAsync(c->time_h, c->time_d, sizeof(DevTime), cudaMemcpyDeviceToHost, c->stream), "read time");
    CK(cudaStreamSynchronize(c->stream), "read time");
    c->d2h += sizeof(DevTime);
    return check_time(c);
}

template <typename T>
int step_impl(amr_ctx* c, double dt, double* dt_used) {
    const bool with_cfl = !(dt > 0.0);
    if (!with_cfl) {
        CK(launch_set_dt(c->time_d, dt, c->stream), "set dt");
        ++c->kernels;
        c->h2d += sizeof(double);
    }
    c->cfl_timed = with_cfl;
    if (c->mode == AMR_MODE_PER_PATCH) {
        int r = per_patch_step<T>(c, with_cfl);
        if (r) return r;
    } else if (c->use_graph) {
        const bool skip = c->ghosts_valid;
        cudaGraphExec_t& ex = c->graph[with_cfl][skip];
        long long& nk = c->graph_kernels[with_cfl][skip];
        if (!ex) {
            cudaGraph_t gr;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            c->capturing = true;
            int r = enqueue_step<T>(c, with_cfl, skip, &nk);
            c->capturing = false;
            cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
            if (r) return r;
            if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
            e = cudaGraphInstantiate(&ex, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return cuda_fail(c, e, "instantiate graph");
        }
        CK(cudaGraphLaunch(ex, c->stream), "graph launch");
        c->kernels += nk;
    } else {
        long long nk = 0;
        int r = enqueue_step<T>(c, with_cfl, c->ghosts_valid, &nk);
        if (r) return r;
        c->kernels += nk;
    }
    c->ghosts_valid = false;                               // U0 has advanced
    if (dt_used) {
        int r = read_time(c);
        if (r) return r;
        *dt_used = c->time_h->dt;
    }
    return AMR_OK;
}

// The flagging half of a regrid, enqueued: ghost fill, flags, request
// compaction (which sets DevTime::cancel when there are requests), and the
// read-back of the request lists and of the time record; ev_req marks its end.
template <typename T>
int regrid_enqueue(amr_ctx* c) {
    c->rg_t0 = std::chrono::steady_clock::now();
    auto mark = [&](cudaEvent_t e) { return c->timing ? cudaEventRecord(e, c->stream) : cudaSuccess; };
    CK(mark(c->ev_rg[0]), "event");
    const long long k0 = c->kernels;
    int r = fill_all_levels<T>(c, St<T>(c, 0), 0.0);
    if (r) return r;
    c->regrid_fill_launches = (int)(c->kernels - k0);
    CK(mark(c->ev_rg[1]), "event");
    if (c->flagger == AMR_FLAG_MLP && (c->mlp_w || !c->initialising)) {
        if (!c->mlp_w) return fail(c, AMR_ERR_STATE, "learned indicator selected but no weights set");
        CK(Kernels<T>::flag_mlp(c->grid, St<T>(c, 0), c->mlp_w, c->anyflag, grid_size(c, 1), c->stream),
           "flag (learned)");
    } else {
        CK(Kernels<T>::flag_plain(c->grid, St<T>(c, 0), c->anyflag, grid_size(c, c->tune[AMR_TUNE_FLAG_GRID]),
                                  c->stream),
           "flag");
    }
    CK(mark(c->ev_rg[2]), "event");
    CK(launch_requests(c->grid, c->anyflag, c->rej_d, c->req_d + 2, c->req_d + 2 + c->cap, c->req_d, c->stream),
       "requests");
    c->kernels += 2;
    // counts and the first REQ_READ entries of both lists, and the time record, in one read-back
    const int head = std::min(c->cap, REQ_READ);
    CK(cudaMemcpyAsync(c->req_h, c->req_d, (2 + (size_t)head) * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "read requests");
    CK(cudaMemcpyAsync(c->req_h + 2 + c->cap, c->req_d + 2 + c->cap, (size_t)head * sizeof(int),
                       cudaMemcpyDeviceToHost, c->stream),
       "read requests");
    CK(cudaMemcpyAsync(c->time_h, c->time_d, sizeof(DevTime), cudaMemcpyDeviceToHost, c->stream), "read time");
    CK(cudaEventRecord(c->ev_req, c->stream), "read requests");
    c->ghosts_valid = true;                                // filled at the current time for the flags
    return AMR_OK;
}

// Wait for the requests of regrid_enqueue and turn them into keys; clears
// DevTime::cancel when there were any. void_step (may be NULL): the
// compaction set DevTime::cancel, so a step issued after regrid_enqueue is void.
int read_requests(amr_ctx* c, std::vector<Key>& req, std::vector<Key>& cand, bool* void_step = nullptr) {
    CK(cudaEventSynchronize(c->ev_req), "read requests");
    if (void_step) *void_step = c->time_h->cancel != 0;
    const int nr = c->req_h[0], nc = c->req_h[1];
    const int head = std::min(c->cap, REQ_READ);
    c->d2h += (long long)(2 + 2 * head) * sizeof(int) + sizeof(DevTime);
    if (nr | nc) {
        CK(cudaMemsetAsync(&c->time_d->cancel, 0, sizeof(int), c->stream), "clear cancel");
        if (nr > head || nc > head) {                      // long lists: the rest in a second read-back
            if (nr > head)
                CK(cudaMemcpyAsync(c->req_h + 2 + head, c->req_d + 2 + head, (size_t)(nr - head) * sizeof(int),
                                   cudaMemcpyDeviceToHost, c->stream),
                   "read requests");
            if (nc > head)
                CK(cudaMemcpyAsync(c->req_h + 2 + c->cap + head, c->req_d + 2 + c->cap + head,
                                   (size_t)(nc - head) * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "read requests");
            CK(cudaStreamSynchronize(c->stream), "read requests");
            c->d2h += (long long)(std::max(nr - head, 0) + std::max(nc - head, 0)) * sizeof(int);
        }
    }
    int r = check_time(c);
    if (r) return r;
    req.clear();
    cand.clear();
    for (int i = 0; i < nr; ++i) req.push_back(unpack(c->key_of[c->req_h[2 + i]]));
    for (int i = 0; i < nc; ++i) cand.push_back(unpack(c->key_of[c->req_h[2 + c->cap + i]]));
    c->regrid_ms[0] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c->rg_t0).count();
    c->regrid_timed = c->timing;
    return AMR_OK;
}

// flags of the current state (ghosts filled first) -> request keys on the host
template <typename T>
int compute_requests(amr_ctx* c, std::vector<Key>& req, std::vector<Key>& cand) {
    int r = regrid_enqueue<T>(c);
    if (r) return r;
    return read_requests(c, req, cand);
}

// The device copy of the coarsening candidates the host found it could not
// coarsen (n >= 0), or none (n = -1), for the request compaction's test.
int set_rejected(amr_ctx* c, int n) {
    int* stage = c->req_h + 2 + 2 * (size_t)c->cap;      // pinned staging word
    *stage = n;
    if (n > 0)
        CK(cudaMemcpyAsync(c->rej_d + 1, c->req_d + 2 + c->cap, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice,
                           c->stream),
           "rejected");
    CK(cudaMemcpyAsync(c->rej_d, stage, sizeof(int), cudaMemcpyHostToDevice, c->stream), "rejected");
    return AMR_OK;
}

// The host half of a regrid: the requests, closed under R2 (Algorithm 1),
// coarsening, and the new hierarchy applied. void_step (may be NULL): a step
// issued after regrid_enqueue is void; changed (may be NULL): the hierarchy
// changed.
template <typename T>
int regrid_finish(amr_ctx* c, bool resample_ic, bool* void_step, bool* changed) {
    if (changed) *changed = false;
    std::vector<Key> req, cand;
    int r = read_requests(c, req, cand, void_step);
    if (r) return r;
    const auto t1 = std::chrono::steady_clock::now();
    c->regrid_ms[1] = c->regrid_ms[2] = 0.0;
    if (req.empty() && cand.empty()) return AMR_OK;
    Mesh m2 = c->mesh;
    std::vector<Key> created, deleted;
    {
        Range closure("regrid: closure and coarsening");
        created = m2.refine(req);
        std::unordered_set<uint64_t> just;
        for (const auto& k : created) just.insert(pack(k));
        deleted = m2.coarsen(cand, just);
    }
    if (created.empty() && deleted.empty())                // the same candidates give the same answer
        return set_rejected(c, req.empty() ? (int)cand.size() : -1);
    if ((long long)m2.patches.size() > c->cap)
        return fail(c, AMR_ERR_POOL, "patch pool capacity exceeded; hierarchy left unchanged");
    c->ghosts_valid = false;                               // new and removed patches: neighbours' ghosts stale
    if (changed) *changed = true;
    r = set_rejected(c, -1);
    if (r) return r;
    Range tables("regrid: tables and new patches");
    c->mesh.swap_patches(m2);
    assign_slots(c, created, deleted);
    const auto t2 = std::chrono::steady_clock::now();
    r = rebuild_tables(c, created);
    if (r) return r;
    const MetaLayout ml(c->cap);
    const int* new_list = c->meta_d + ml.new_list;
    if (resample_ic) CK(Kernels<T>::init_ic(c->grid, St<T>(c, 0), new_list, (int)created.size(), c->stream), "ic");
    else CK(Kernels<T>::prolong_new(c->grid, St<T>(c, 0), new_list, (int)created.size(), c->stream), "prolong");
    ++c->kernels;
    if (c->timing) CK(cudaStreamSynchronize(c->stream), "regrid");
    const auto t3 = std::chrono::steady_clock::now();
    c->regrid_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    c->regrid_ms[2] = std::chrono::duration<double, std::milli>(t3 - t2).count();
    return AMR_OK;
}

template <typename T>
int regrid_impl(amr_ctx* c, bool resample_ic) {
    int r = regrid_enqueue<T>(c);
    if (r) return r;
    return regrid_finish<T>(c, resample_ic, nullptr, nullptr);
}

// n steps, a regrid after every K-th step since the last regrid. Before a
// regrid's requests are read on the host the next step is already issued; if
// there were requests, that step's kernels found DevTime::cancel set and did
// nothing, and it is issued again once the hierarchy has been updated. Steps
// between regrids are issued back to back without any host synchronisation.
template <typename T>
int advance_impl(amr_ctx* c, int n, int K) {
    if (n == 0) return AMR_OK;
    int r = step_impl<T>(c, 0.0, nullptr);
    if (r) return r;
    for (int i = 0; i < n; ++i) {
        const bool more = i + 1 < n;
        if (++c->since_regrid < K) {
            if (more && (r = step_impl<T>(c, 0.0, nullptr))) return r;
            continue;
        }
        c->since_regrid = 0;
        if ((r = regrid_enqueue<T>(c))) return r;
        if (more && (r = step_impl<T>(c, 0.0, nullptr))) return r;
        bool had = false, changed = false;                 // had: the step issued ahead is void
        if ((r = regrid_finish<T>(c, false, &had, &changed))) return r;
        if (more && had) {
            if (!changed) c->ghosts_valid = true;          // the void step left the filled ghosts as they were
            if ((r = step_impl<T>(c, 0.0, nullptr))) return r;
        }
    }
    return AMR_OK;
}

// device address of a caller's host buffer that the GPU can access directly
// (page-locked host memory, e.g. from cudaHostAlloc or PyTorch's pinned
// memory), else nullptr: such buffers are read or written by the pack and
// unpack kernels in one launch, other buffers go through the staging buffer
void* mapped_host(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();                                // not a CUDA-known pointer: clear the error
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <typename T>
int get_level_impl(amr_ctx* c, int level, int* n_out, int* coords, double* data) {
    std::vector<int> slots;
    std::vector<Key> keys;
    for (size_t i = 0; i < c->canon.size(); ++i)
        if (c->canon[i].l == level) {
            keys.push_back(c->canon[i]);
            slots.push_back(c->canon_slot[i]);
        }
    *n_out = (int)keys.size();
    if (coords)
        for (size_t i = 0; i < keys.size(); ++i) {
            const int cc[3] = {keys[i].x, keys[i].y, keys[i].z};
            for (int d = 0; d < c->dim; ++d) coords[i * c->dim + d] = cc[d];
        }
    if (data && !slots.empty()) {
        long long ncell = 1;
        for (int d = 0; d < c->dim; ++d) ncell *= c->N;
        const size_t per = (size_t)c->nv * ncell;
        if (double* dev = static_cast<double*>(mapped_host(data))) {   // straight into the caller's buffer
            const int n = (int)slots.size();
            CK(cudaMemcpyAsync(c->slots_d, slots.data(), n * sizeof(int), cudaMemcpyHostToDevice, c->stream),
               "get level");
            CK(Kernels<T>::unpack_interiors(c->grid, St<T>(c, 0), c->slots_d, n, dev, c->stream), "unpack");
            CK(cudaStreamSynchronize(c->stream), "get level");
            c->h2d += n * sizeof(int);
            c->d2h += (long long)(n * per * sizeof(double));
            ++c->kernels;
            return AMR_OK;
        }
        const size_t chunk = std::max<size_t>(1, c->dense_cap / per);
        for (size_t b = 0; b < slots.size(); b += chunk) {
            const int n = (int)std::min(chunk, slots.size() - b);
            CK(cudaMemcpyAsync(c->slots_d, slots.data() + b, n * sizeof(int), cudaMemcpyHostToDevice, c->stream),
               "get level");
            CK(Kernels<T>::unpack_interiors(c->grid, St<T>(c, 0), c->slots_d, n, c->dense_d, c->stream), "unpack");
            CK(cudaMemcpyAsync(data + b * per, c->dense_d, n * per * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream),
               "get level");
            CK(cudaStreamSynchronize(c->stream), "get level");
            c->h2d += n * sizeof(int);
            c->d2h += (long long)(n * per * sizeof(double));
            ++c->kernels;
        }
    }
    return AMR_OK;
}

template <typename T>
int set_state_impl(amr_ctx* c, int n, const int* levels, const int* coords, const double* data, double t) {
    Mesh m2(c->dim, c->mesh.base, c->mesh.periodic, c->L - 1);
    m2.clear();
    std::vector<Key> keys;
    for (int i = 0; i < n; ++i) {
        Key k{levels[i], coords[i * c->dim], c->dim >= 2 ? coords[i * c->dim + 1] : 0,
              c->dim == 3 ? coords[i * c->dim + 2] : 0};
        if (k.l < 0 || k.l >= c->L) return fail(c, AMR_ERR_MESH, "level out of range");
        for (int d = 0; d < c->dim; ++d) {                  // before packing: keys hold 20-bit coordinates
            const int x = coords[i * c->dim + d];
            if (x < 0 || x >= m2.extent(k.l, d)) return fail(c, AMR_ERR_MESH, "patch outside the domain");
        }
        if (!m2.insert(k)) return fail(c, AMR_ERR_MESH, "duplicate patch");
        keys.push_back(k);
    }
    const std::string why = m2.check();
    if (!why.empty()) return fail(c, AMR_ERR_MESH, why);
    if ((int)keys.size() > c->cap) return fail(c, AMR_ERR_POOL, "patch pool capacity exceeded");
    c->mesh.swap_patches(m2);
    slot_map_clear(c);
    c->slot_hi = 0;
    c->free_slots.clear();
    for (int s = 0; s < c->cap; ++s) {
        c->free_slots.insert(s);
        c->used[s] = 0;
    }
    std::vector<Key> all = c->mesh.canonical();
    assign_slots(c, all, {});
    c->ghosts_valid = false;
    if (int r0 = set_rejected(c, -1)) return r0;                 // a new hierarchy
    int r = rebuild_tables(c, {});
    if (r) return r;
    long long ncell = 1;
    for (int d = 0; d < c->dim; ++d) ncell *= c->N;
    const size_t per = (size_t)c->nv * ncell;
    const size_t chunk = std::max<size_t>(1, c->dense_cap / per);
    std::vector<int> slots(n);
    for (int i = 0; i < n; ++i) slots[i] = slot_lookup(c, keys[i]);
    const double* dev = static_cast<const double*>(mapped_host(data));   // read in place if possible
    if (dev) {
        CK(cudaMemcpyAsync(c->slots_d, slots.data(), n * sizeof(int), cudaMemcpyHostToDevice, c->stream), "set");
        CK(Kernels<T>::pack_interiors(c->grid, St<T>(c, 0), c->slots_d, n, dev, c->stream), "pack");
        CK(cudaStreamSynchronize(c->stream), "set");
        c->h2d += (long long)(n * sizeof(int) + n * per * sizeof(double));
        ++c->kernels;
    }
    for (int b = 0; dev == nullptr && b < n; b += (int)chunk) {
        const int m = (int)std::min<size_t>(chunk, n - b);
        CK(cudaMemcpyAsync(c->slots_d, slots.data() + b, m * sizeof(int), cudaMemcpyHostToDevice, c->stream), "set");
        CK(cudaMemcpyAsync(c->dense_d, data + (size_t)b * per, m * per * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream),
           "set");
        CK(Kernels<T>::pack_interiors(c->grid, St<T>(c, 0), c->slots_d, m, c->dense_d, c->stream), "pack");
        CK(cudaStreamSynchronize(c->stream), "set");
        c->h2d += (long long)(m * sizeof(int) + m * per * sizeof(double));
        ++c->kernels;
    }
    c->time_h->t = t;
    c->time_h->dt = 0.0;
    c->time_h->lam = 0ull;
    c->time_h->err = 0;
    c->time_h->cancel = 0;
    CK(cudaMemcpyAsync(c->time_d, c->time_h, sizeof(DevTime), cudaMemcpyHostToDevice, c->stream), "set time");
    CK(cudaStreamSynchronize(c->stream), "set time");
    return AMR_OK;
}

template <typename T>
int cons_impl(amr_ctx* c, double* out) {
    CK(Kernels<T>::cons_sums(c->grid, St<T>(c, 0), c->cons_partial, c->cons_d, c->stream), "cons sums");
    c->kernels += 2;
    CK(cudaMemcpyAsync(out, c->cons_d, c->nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cons sums");
    CK(cudaStreamSynchronize(c->stream), "cons sums");
    c->d2h += c->nv * sizeof(double);
    return AMR_OK;
}

bool valid_bc(int b) { return b >= AMR_BC_OUTFLOW && b <= AMR_BC_DMR_TOP; }

}  // namespace

// ---------------------------------------------------------------------------
// Autotuner of the batched step's launch parameters: each candidate timed
// with CUDA events (best of 3 after a warm-up) on the stage arrays, which hold
// a copy of the state; the device time record is saved and put back.
template <typename T>
int autotune_impl(amr_ctx* c) {
    const Grid& g = c->grid;
    const size_t state_bytes = (size_t)c->cap * g.patch_elems * sizeof(T);
    T* A = St<T>(c, 1);
    T* B = St<T>(c, 2);
    T* faces = reinterpret_cast<T*>(c->faces);
    CK(cudaMemcpyAsync(A, St<T>(c, 0), state_bytes, cudaMemcpyDeviceToDevice, c->stream), "autotune copy");
    DevTime saved;
    CK(cudaMemcpyAsync(&saved, c->time_d, sizeof(DevTime), cudaMemcpyDeviceToHost, c->stream), "autotune");
    CK(cudaStreamSynchronize(c->stream), "autotune");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "autotune");
    cudaError_t err = cudaEventCreate(&e1);
    long long nk = 0;
    // best-of-3 device time of launch() after one warm-up call
    auto timed = [&](auto&& launch, float& best) -> cudaError_t {
        cudaError_t e = launch();
        if (e != cudaSuccess) return e;
        best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) return e;
            if ((e = launch()) != cudaSuccess) return e;
            if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess) return e;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
            best = ms < best ? ms : best;
        }
        return cudaSuccess;
    };
    // pick the fastest of `cands` for parameter `slot`: launch(candidate)
    auto tune_one = [&](int slot, const int* cands, int n, auto&& launch) -> cudaError_t {
        float bestv = 1e30f;
        int pick = c->tune[slot];
        for (int i = 0; i < n; ++i) {
            float t = 0.f;
            const cudaError_t e = timed([&]() { return launch(cands[i]); }, t);
            if (e != cudaSuccess) return e;
            if (t < bestv) {
                bestv = t;
                pick = cands[i];
            }
        }
        c->tune[slot] = pick;
        c->tune_ms[slot] = bestv;
        return cudaSuccess;
    };
    if (err == cudaSuccess) {                            // ghost fill of every level: grid x work-item size
        const int grids[] = {4, 8, 16, 32}, chunks[] = {64, 128, 256, 512, 1024};
        float bestv = 1e30f;
        for (int gr : grids)
            for (int ch : chunks) {
                float t = 0.f;
                err = timed([&]() {
                    for (int l = 0; l < c->L; ++l) {
                        const cudaError_t e = Kernels<T>::ghost_fill(g, A, l, 0.0, grid_size(c, gr), c->stream, -1, ch,
                                                                     true);
                        ++nk;
                        if (e != cudaSuccess) return e;
                    }
                    return cudaSuccess;
                }, t);
                if (err != cudaSuccess) break;
                if (t < bestv) {
                    bestv = t;
                    c->tune[AMR_TUNE_GHOST_GRID] = gr;
                    c->tune[AMR_TUNE_GHOST_CHUNK] = ch;
                }
            }
        c->tune_ms[AMR_TUNE_GHOST_GRID] = c->tune_ms[AMR_TUNE_GHOST_CHUNK] = bestv;
    }
    if (err == cudaSuccess) {                            // fused RHS: tile shape x grid, timed on a stage
        // that reads only its input (A -> B) and one that also reads U0 and
        // writes in place (B, U0 = A -> A, as the step's last stage does)
        const int shapes = Kernels<T>::rhs_shapes(g);
        float bestv = 1e30f;
        int best_shape = 0, best_grid = c->tune[AMR_TUNE_RHS_GRID];
        for (int sh = 0; sh < shapes && err == cudaSuccess; ++sh) {
            if (shape_needs_tma(c, sh) && !c->tma_ok) continue;
            c->grid.rhs_shape = sh;
            // CTAs per SM of grid: beyond the resident count, a finer share of
            // the work items per CTA evens out the tail of a launch
            const int rgrid[] = {1, 2, 3, 4, 6, 8, 12, 16};
            for (int gi = 0; gi < 8 && err == cudaSuccess; ++gi) {
                const int gr = rgrid[gi];
                float t = 0.f;
                err = timed([&]() {
                    nk += 2;
                    const cudaError_t e =
                        Kernels<T>::rhs_stage(g, A, St<T>(c, 0), B, faces, 0, grid_size(c, gr), c->stream, -1, 1,
                                              tmap_of(c, A));
                    if (e != cudaSuccess) return e;
                    return Kernels<T>::rhs_stage(g, B, A, A, faces, 2, grid_size(c, gr), c->stream, -1, 1,
                                                 tmap_of(c, B));
                }, t);
                if (t < bestv) {
                    bestv = t;
                    best_shape = sh;
                    best_grid = gr;
                }
            }
        }
        c->tune[AMR_TUNE_RHS_SHAPE] = best_shape;
        c->tune[AMR_TUNE_RHS_GRID] = best_grid;
        c->grid.rhs_shape = best_shape;
        c->tune_ms[AMR_TUNE_RHS_SHAPE] = c->tune_ms[AMR_TUNE_RHS_GRID] = bestv;
    }
    if (err == cudaSuccess) {                            // reflux of stage 1 into B
        const int cands[] = {1, 2, 4, 8, 16};
        err = tune_one(AMR_TUNE_REFLUX_GRID, cands, 5, [&](int gr) {
            ++nk;
            return Kernels<T>::reflux(g, B, faces, 0, grid_size(c, gr), c->stream, -1);
        });
    }
    if (err == cudaSuccess) {                            // restriction of the levels a step restricts
        const int cands[] = {2, 4, 8, 16, 32};           // (the finest is fused into the RHS)
        err = tune_one(AMR_TUNE_RESTRICT_GRID, cands, 5, [&](int gr) {
            for (int l = c->L - 2; l >= 1; --l) {
                ++nk;
                const cudaError_t e = Kernels<T>::restrict_level(g, A, l, grid_size(c, gr), c->stream, -1);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        });
    }
    if (err == cudaSuccess) {                            // CFL reduction over the leaves of A
        const int cands[] = {2, 4, 8, 16, 32};
        err = tune_one(AMR_TUNE_CFL_GRID, cands, 5, [&](int gr) {
            ++nk;
            return Kernels<T>::cfl(g, A, grid_size(c, gr), c->stream, -1);
        });
    }
    if (err == cudaSuccess) {                            // plain flagging of A (scratch flags)
        const int cands[] = {1, 2, 4, 8, 16};
        err = tune_one(AMR_TUNE_FLAG_GRID, cands, 5, [&](int gr) {
            ++nk;
            return Kernels<T>::flag_plain(g, A, c->anyflag, grid_size(c, gr), c->stream);
        });
    }
    c->kernels += nk;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(c, err, "autotune");
    CK(cudaMemcpyAsync(c->time_d, &saved, sizeof(DevTime), cudaMemcpyHostToDevice, c->stream), "autotune");
    CK(cudaStreamSynchronize(c->stream), "autotune");
    drop_graphs(c);
    return AMR_OK;
}

extern "C" {

void amr_default_options(amr_options_t* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = 64;
    opt->cfl = 0.5;
    opt->t_end = 0.0;
    opt->flagger = AMR_FLAG_PLAIN;
    opt->theta_rho = 0.05;
    opt->theta_p = 0.05;
    opt->max_patches = 0;
    opt->seed = 0;
    opt->amp = 0.01;
    opt->mode = AMR_MODE_BATCHED;
    opt->use_graph = 1;
    opt->theta_switch = 0.05;
}

int amr_init(amr_ctx** out, const amr_domain_t* dom, double gamma, const int base_cells[3], int levels, int ratio,
             int patch_size, int ic_id, const amr_options_t* opt) {
    if (!out || !dom || !base_cells) return AMR_ERR_ARG;
    *out = nullptr;
    amr_ctx* c = new (std::nothrow) amr_ctx();
    if (!c) return AMR_ERR_ARG;
    if (opt) c->opt = *opt;
    else amr_default_options(&c->opt);
    auto bad = [&](const char* m) {
        c->err = m;
        *out = c;   // the caller can read the message, then destroy
        return AMR_ERR_ARG;
    };
    const int dim = dom->dim;
    if (dim < 1 || dim > 3) return bad("dim must be 1, 2 or 3");
    if (ratio != 2) return bad("ratio must be 2");
    if (!(patch_size == 8 || patch_size == 16 || (patch_size == 32 && dim < 3)))
        return bad("patch size must be 8, 16 or 32 (3D: 8 or 16)");
    if (levels < 1 || levels > MAXL) return bad("levels must be in [1, 8]");
    if (!(gamma > 1.0)) return bad("gamma must exceed 1");
    if (c->opt.precision != 32 && c->opt.precision != 64) return bad("precision must be 32 or 64");
    if (ic_id < AMR_IC_SOD || ic_id > AMR_IC_SHEAR_LAYER) return bad("unknown initial condition");
    if (!(c->opt.cfl > 0.0)) return bad("cfl must be positive");
    if (c->opt.flagger != AMR_FLAG_PLAIN && c->opt.flagger != AMR_FLAG_MLP) return bad("unknown flagger");
    if (c->opt.mode != AMR_MODE_BATCHED && c->opt.mode != AMR_MODE_PER_PATCH) return bad("unknown mode");
    if (c->opt.flux != AMR_FLUX_RUSANOV && c->opt.flux != AMR_FLUX_HLLC && c->opt.flux != AMR_FLUX_CENTRAL &&
        c->opt.flux != AMR_FLUX_HYBRID)
        return bad("unknown flux");
    if (c->opt.theta_switch != c->opt.theta_switch) return bad("theta_switch is NaN");
    if (!(c->opt.mlp_keep_margin >= 0.0) || !(c->opt.mlp_keep_margin < 1.0e30))
        return bad("mlp_keep_margin must be in [0, 1e30)");
    if (!(c->opt.mlp_refine_margin >= 0.0) || !(c->opt.mlp_refine_margin <= c->opt.mlp_keep_margin))
        return bad("mlp_refine_margin must be in [0, mlp_keep_margin]");
    int bp[3] = {1, 1, 1};
    bool periodic[3] = {false, false, false};
    for (int d = 0; d < dim; ++d) {
        if (base_cells[d] < patch_size || base_cells[d] % patch_size) return bad("base cells must be multiples of the patch size");
        if (!(dom->hi[d] > dom->lo[d])) return bad("empty domain");
        if (!valid_bc(dom->bc_lo[d]) || !valid_bc(dom->bc_hi[d])) return bad("unknown boundary kind");
        if ((dom->bc_lo[d] == AMR_BC_PERIODIC) != (dom->bc_hi[d] == AMR_BC_PERIODIC))
            return bad("periodic boundaries must be periodic on both sides");
        if (dom->bc_lo[d] >= AMR_BC_DMR_INFLOW || dom->bc_hi[d] >= AMR_BC_DMR_INFLOW)
            if (dim != 2) return bad("double-Mach boundaries are 2D only");
        bp[d] = base_cells[d] / patch_size;
        if (((long long)bp[d] << (levels - 1)) >= (1LL << 20))       // keys hold 20-bit patch coordinates
            return bad("more than 2^20 - 1 patches along a dimension of the finest level");
        periodic[d] = dom->bc_lo[d] == AMR_BC_PERIODIC;
    }
    c->dim = dim;
    c->N = patch_size;
    c->L = levels;
    c->nv = dim + 2;
    c->gamma = gamma;
    c->precision = c->opt.precision;
    c->ic = ic_id;
    c->mode = c->opt.mode;
    c->use_graph = c->opt.use_graph;
    c->flagger = c->opt.flagger;
    for (int d = 0; d < 3; ++d) c->base_cells[d] = d < dim ? base_cells[d] : 1;
    // pool capacity, checked before the level-0 layout is built
    long long full = 0;
    for (int l = 0; l < levels; ++l) {
        long long n = 1;
        for (int d = 0; d < dim; ++d) n *= (long long)bp[d] << l;
        full += n;
    }
    if (c->opt.max_patches <= 0 && full > 0x7fffffffLL)
        return bad("every level fully refined exceeds 2^31 - 1 patches: set max_patches");
    c->cap = c->opt.max_patches > 0 ? (int)std::min<long long>(c->opt.max_patches, full) : (int)full;
    if ((long long)bp[0] * bp[1] * bp[2] > c->cap) return bad("pool smaller than the base level");
    c->mesh = Mesh(dim, bp, periodic, levels - 1);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        c->err = "no CUDA device";
        *out = c;
        return AMR_ERR_CUDA;
    }
    if (c->opt.stream) {
        c->stream = reinterpret_cast<cudaStream_t>(c->opt.stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            c->err = "stream creation failed";
            *out = c;
            return AMR_ERR_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;

    // pool
    const int S = patch_size + 2 * G;
    Grid& g = c->grid;
    g.dim = dim;
    g.N = patch_size;
    g.L = levels;
    g.nv = c->nv;
    {
        const int per32 = 32 / (c->precision == 64 ? 8 : 4);       // elements per 32-byte sector
        g.XP = (per32 - G % per32) % per32;
        g.SX = (g.XP + S + 7) / 8 * 8;
    }
    g.SY = dim >= 2 ? S : 1;
    g.SZ = dim == 3 ? S : 1;
    g.slot_elems = (long long)g.SX * g.SY * g.SZ;
    g.patch_elems = g.slot_elems * c->nv;
    g.cap = c->cap;
    for (int l = 0; l < MAXL; ++l)
        for (int d = 0; d < 3; ++d) {
            g.ext[l][d] = d < dim ? (bp[d] << std::min(l, 20)) : 1;
            g.dx[l][d] = d < dim ? (dom->hi[d] - dom->lo[d]) / (double)((long long)base_cells[d] << l) : 1.0;
        }
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = d < dim ? dom->lo[d] : 0.0;
        g.periodic[d] = periodic[d] ? 1 : 0;
        g.bc[d][0] = d < dim ? dom->bc_lo[d] : AMR_BC_OUTFLOW;
        g.bc[d][1] = d < dim ? dom->bc_hi[d] : AMR_BC_OUTFLOW;
        g.base_cells[d] = c->base_cells[d];
    }
    g.gamma = gamma;
    g.cfl = c->opt.cfl;
    g.t_end = c->opt.t_end;
    g.theta_rho = c->opt.theta_rho;
    g.theta_p = c->opt.theta_p;
    g.ic = ic_id;
    g.flux = c->opt.flux;
    g.theta_sw = c->opt.theta_switch;
    g.rhs_shape = 0;
    g.mlp_keep = (float)c->opt.mlp_keep_margin;
    g.mlp_refine = (float)c->opt.mlp_refine_margin;
    g.tc_wait = TC_WAIT_CYCLES;
    g.tc_test = 0;
    g.seed = c->opt.seed;
    g.amp = c->opt.amp;
    dmr_states(gamma, g.dmr_pre, g.dmr_post);

    const size_t esz = c->precision == 64 ? 8 : 4;
    const size_t state_bytes = (size_t)c->cap * g.patch_elems * esz;
    long long trans = 1;
    for (int d = 1; d < dim; ++d) trans *= patch_size;
    const size_t face_bytes = (size_t)c->cap * 2 * dim * c->nv * trans * esz;
    for (int i = 0; i < 3; ++i) c->U[i] = dalloc(c, state_bytes);
    c->faces = dalloc(c, face_bytes);
    const MetaLayout ml(c->cap);
    c->meta_ints = ml.total;
    c->meta_d = (int*)dalloc(c, ml.total * sizeof(int));
    c->anyflag = (int*)dalloc(c, (c->cap + 32) * sizeof(int));     // flags + the learned flagger's work counter
    c->req_d = (int*)dalloc(c, (3 + 3 * (size_t)c->cap) * sizeof(int));
    c->cons_partial = (double*)dalloc(c, (size_t)c->cap * c->nv * sizeof(double));
    c->cons_d = (double*)dalloc(c, 8 * sizeof(double));
    c->dense_cap = std::max<size_t>((size_t)g.patch_elems * 64, (size_t)1 << 22);
    c->dense_d = (double*)dalloc(c, c->dense_cap * sizeof(double));
    c->slots_d = (int*)dalloc(c, c->cap * sizeof(int));
    c->time_d = (DevTime*)dalloc(c, sizeof(DevTime));
    for (int i = 0; i < 3; ++i)
        if (!c->U[i]) return fail(c, AMR_ERR_CUDA, "device allocation failed");
    if (c->precision == 32 && dim == 3 && patch_size == 16) c->tma_ok = encode_tmaps(c);
    if (!c->faces || !c->meta_d || !c->anyflag || !c->req_d || !c->cons_partial || !c->cons_d || !c->dense_d ||
        !c->slots_d || !c->time_d)
        return fail(c, AMR_ERR_CUDA, "device allocation failed");
    if (cudaMallocHost((void**)&c->meta_h, ml.total * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&c->req_h, (3 + 2 * (size_t)c->cap) * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&c->time_h, sizeof(DevTime)) != cudaSuccess)
        return fail(c, AMR_ERR_CUDA, "pinned host allocation failed");
    CK(cudaEventCreateWithFlags(&c->ev_req, cudaEventDisableTiming), "event");
    c->rej_d = c->req_d + 2 + 2 * (size_t)c->cap;
    CK(cudaMemsetAsync(c->rej_d, 0xFF, sizeof(int), c->stream), "clear rejected");   // -1: none
    for (int i = 0; i < 3; ++i) CK(cudaMemsetAsync(c->U[i], 0, state_bytes, c->stream), "clear pool");
    CK(cudaMemsetAsync(c->faces, 0, face_bytes, c->stream), "clear faces");
    CK(cudaMemsetAsync(c->anyflag, 0, c->cap * sizeof(int), c->stream), "clear flags");
    std::memset(c->time_h, 0, sizeof(DevTime));
    CK(cudaMemcpyAsync(c->time_d, c->time_h, sizeof(DevTime), cudaMemcpyHostToDevice, c->stream), "time");

    // ghost-cell tables of a slot, packed slot coordinates (x | y << 10 | z << 20):
    // every ghost cell in slot order (the regrid's fill, before the flag
    // stencils), then the face ghosts (outside the interior along one
    // dimension) box by box (x low, x high, y low, ...; G N^(d-1) cells each,
    // slot order inside a box: a stage fills or skips a box whole)
    std::vector<int> gt, gt_box;
    for (int z = 0; z < g.SZ; ++z)
        for (int y = 0; y < g.SY; ++y)
            for (int x = 0; x < S; ++x) {
                const bool gx = x < G || x >= G + patch_size;
                const bool gy = dim >= 2 && (y < G || y >= G + patch_size);
                const bool gz = dim == 3 && (z < G || z >= G + patch_size);
                if (gx || gy || gz) gt.push_back(x | ((dim >= 2 ? y : G) << 10) | ((dim == 3 ? z : G) << 20));
            }
    for (int b = 0; b < 2 * dim; ++b)
        for (int z = 0; z < g.SZ; ++z)
            for (int y = 0; y < g.SY; ++y)
                for (int x = 0; x < S; ++x) {
                    const int cc[3] = {x, y, z};
                    int nout = 0, dout = -1, sout = 0;
                    for (int d = 0; d < dim; ++d)
                        if (cc[d] < G || cc[d] >= G + patch_size) {
                            ++nout;
                            dout = d;
                            sout = cc[d] >= G + patch_size;
                        }
                    if (nout == 1 && 2 * dout + sout == b)
                        gt_box.push_back(x | ((dim >= 2 ? y : G) << 10) | ((dim == 3 ? z : G) << 20));
                }
    c->n_ghost = (int)gt.size();
    c->n_ghost_face = (int)gt_box.size();
    gt.insert(gt.end(), gt_box.begin(), gt_box.end());
    c->ghost_tab = (int*)dalloc(c, gt.size() * sizeof(int));
    if (!c->ghost_tab) return fail(c, AMR_ERR_CUDA, "device allocation failed");
    CK(cudaMemcpyAsync(c->ghost_tab, gt.data(), gt.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "ghosts");
    CK(cudaStreamSynchronize(c->stream), "init");

    g.level = c->meta_d + ml.level;
    g.coord = c->meta_d + ml.coord;
    g.nbr = c->meta_d + ml.nbr;
    g.parent = c->meta_d + ml.parent;
    g.child = c->meta_d + ml.child;
    g.pflag = c->meta_d + ml.pflag;
    g.all_list = c->meta_d + ml.all_list;
    g.level_off = c->meta_d + ml.level_off;
    g.leaf_list = c->meta_d + ml.leaf_list;
    g.counts = c->meta_d + ml.counts;
    g.reflux_list = c->meta_d + ml.reflux_list;
    g.reflux_fine = c->meta_d + ml.reflux_fine;
    g.new_list = c->meta_d + ml.new_list;
    g.ghost_tab = c->ghost_tab;
    g.n_ghost = c->n_ghost;
    g.n_ghost_face = c->n_ghost_face;
    g.time = c->time_d;
    {
        cudaError_t e = c->precision == 64 ? Kernels<double>::prepare(g) : Kernels<float>::prepare(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel attributes");
        e = c->precision == 64 ? Kernels<double>::prepare_mlp(g) : Kernels<float>::prepare_mlp(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel attributes");
    }

    if (c->opt.mlp_weights) {
        if (c->opt.mlp_n_weights != mlp_n_weights(dim)) return bad("weight count does not match the dimension");
        c->mlp_w = (float*)dalloc(c, c->opt.mlp_n_weights * sizeof(float));
        if (!c->mlp_w) return fail(c, AMR_ERR_CUDA, "device allocation failed");
        c->mlp_n = c->opt.mlp_n_weights;
        CK(cudaMemcpyAsync(c->mlp_w, c->opt.mlp_weights, c->mlp_n * sizeof(float), cudaMemcpyHostToDevice,
                           c->stream), "weights");
        c->h2d += c->mlp_n * sizeof(float);
    }
    c->opt.mlp_weights = nullptr;     // host pointer not kept
    // level 0 and the initial condition, then the initial hierarchy
    c->initialising = true;
    c->used.assign(c->cap, 0);
    c->key_of.assign(c->cap, 0);
    for (int s = 0; s < c->cap; ++s) c->free_slots.insert(s);
    slot_map_clear(c);
    c->slot_hi = 0;
    std::vector<Key> base = c->mesh.canonical();
    assign_slots(c, base, {});
    int r = rebuild_tables(c, base);
    if (r) return r;
    const int* new_list = c->meta_d + ml.new_list;
    if (c->precision == 64) {
        CK(Kernels<double>::init_ic(g, St<double>(c, 0), new_list, (int)base.size(), c->stream), "ic");
        for (int i = 1; i < levels; ++i)
            if ((r = regrid_impl<double>(c, true))) return r;
    } else {
        CK(Kernels<float>::init_ic(g, St<float>(c, 0), new_list, (int)base.size(), c->stream), "ic");
        for (int i = 1; i < levels; ++i)
            if ((r = regrid_impl<float>(c, true))) return r;
    }
    ++c->kernels;
    CK(cudaStreamSynchronize(c->stream), "init");
    c->initialising = false;
    if (c->opt.autotune) {
        r = c->precision == 64 ? autotune_impl<double>(c) : autotune_impl<float>(c);
        if (r) return r;
    }
    return AMR_OK;
}

#define GUARD(c)                                                        \
    do {                                                                \
        if (!(c)) return AMR_ERR_ARG;                                   \
        if ((c)->broken) return fail((c), AMR_ERR_STATE, "context unusable after an earlier device error"); \
        if (!(c)->U[0]) return fail((c), AMR_ERR_STATE, "context not initialised"); \
    } while (0)

int amr_step(amr_ctx* c, double dt, double* dt_used) {
    GUARD(c);
    Range range("amr_step");
    if (std::isnan(dt)) return fail(c, AMR_ERR_ARG, "dt is NaN");
    return c->precision == 64 ? step_impl<double>(c, dt, dt_used) : step_impl<float>(c, dt, dt_used);
}

int amr_regrid(amr_ctx* c) {
    GUARD(c);
    Range range("amr_regrid");
    if (c->L == 1) return AMR_OK;
    c->since_regrid = 0;
    return c->precision == 64 ? regrid_impl<double>(c, false) : regrid_impl<float>(c, false);
}

int amr_advance(amr_ctx* c, int n_steps, int regrid) {
    GUARD(c);
    Range range("amr_advance");
    if (n_steps < 0) return fail(c, AMR_ERR_ARG, "negative step count");
    if (regrid < 0) return fail(c, AMR_ERR_ARG, "negative regrid interval");
    if (regrid && c->L > 1 && c->mode == AMR_MODE_BATCHED)
        return c->precision == 64 ? advance_impl<double>(c, n_steps, regrid) : advance_impl<float>(c, n_steps, regrid);
    for (int i = 0; i < n_steps; ++i) {
        int r = c->precision == 64 ? step_impl<double>(c, 0.0, nullptr) : step_impl<float>(c, 0.0, nullptr);
        if (r) return r;
        if (regrid && c->L > 1 && ++c->since_regrid >= regrid) {
            c->since_regrid = 0;
            r = c->precision == 64 ? regrid_impl<double>(c, false) : regrid_impl<float>(c, false);
            if (r) return r;
        }
    }
    return AMR_OK;
}

int amr_get_level(amr_ctx* c, int level, int* n_patches, int* coords, double* data) {
    if (!c || !n_patches) return AMR_ERR_ARG;
    if (level < 0 || level >= c->L) return fail(c, AMR_ERR_ARG, "level out of range");
    if (!c->U[0]) return fail(c, AMR_ERR_STATE, "context not initialised");
    return c->precision == 64 ? get_level_impl<double>(c, level, n_patches, coords, data)
                              : get_level_impl<float>(c, level, n_patches, coords, data);
}

int amr_get_diag(amr_ctx* c, double* t, double cons_sums[5], int patches_per_level[8]) {
    if (!c) return AMR_ERR_ARG;
    if (!c->U[0]) return fail(c, AMR_ERR_STATE, "context not initialised");
    if (patches_per_level) {
        for (int l = 0; l < 8; ++l) patches_per_level[l] = 0;
        for (const auto& k : c->canon) patches_per_level[k.l]++;
    }
    if (t) {
        CK(cudaMemcpyAsync(c->time_h, c->time_d, sizeof(DevTime), cudaMemcpyDeviceToHost, c->stream), "diag");
        CK(cudaStreamSynchronize(c->stream), "diag");
        c->d2h += sizeof(DevTime);
        *t = c->time_h->t;
    }
    if (cons_sums) {
        int r = c->precision == 64 ? cons_impl<double>(c, cons_sums) : cons_impl<float>(c, cons_sums);
        if (r) return r;
    }
    return AMR_OK;
}

int amr_set_state(amr_ctx* c, int n, const int* levels, const int* coords, const double* data, double t) {
    GUARD(c);
    if (n <= 0 || !levels || !coords || !data) return fail(c, AMR_ERR_ARG, "empty state");
    return c->precision == 64 ? set_state_impl<double>(c, n, levels, coords, data, t)
                              : set_state_impl<float>(c, n, levels, coords, data, t);
}

static const char CKPT_TAG[8] = {'A', 'M', 'R', 'C', 'K', 'P', 'T', '1'};

int amr_checkpoint(amr_ctx* c, const char* path) {
    GUARD(c);
    if (!path) return fail(c, AMR_ERR_ARG, "no path");
    const long long per = (long long)c->nv * (c->dim == 1 ? c->N : (c->dim == 2 ? c->N * c->N : c->N * c->N * c->N));
    std::vector<int> lv, co;
    std::vector<double> da;
    for (int l = 0; l < c->L; ++l) {
        int n = 0;
        int r = amr_get_level(c, l, &n, nullptr, nullptr);
        if (r) return r;
        const size_t o = lv.size();
        lv.resize(o + n, l);
        co.resize((o + n) * c->dim);
        da.resize((o + n) * per);
        r = amr_get_level(c, l, &n, co.data() + o * c->dim, da.data() + o * per);
        if (r) return r;
    }
    double t = 0.0;
    int r = amr_get_diag(c, &t, nullptr, nullptr);
    if (r) return r;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, AMR_ERR_IO, "cannot open the checkpoint file for writing");
    const int hdr[5] = {c->dim, c->N, c->L, c->nv, (int)lv.size()};
    bool ok = std::fwrite(CKPT_TAG, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 5, f) == 5 &&
              std::fwrite(&t, sizeof(double), 1, f) == 1 &&
              std::fwrite(lv.data(), sizeof(int), lv.size(), f) == lv.size() &&
              std::fwrite(co.data(), sizeof(int), co.size(), f) == co.size() &&
              std::fwrite(da.data(), sizeof(double), da.size(), f) == da.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(c, AMR_ERR_IO, "checkpoint write failed");
    return AMR_OK;
}

int amr_restore(amr_ctx* c, const char* path) {
    GUARD(c);
    if (!path) return fail(c, AMR_ERR_ARG, "no path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, AMR_ERR_IO, "cannot open the checkpoint file");
    char tag[8];
    int hdr[5];
    double t = 0.0;
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, CKPT_TAG, 8) == 0 &&
              std::fread(hdr, sizeof(int), 5, f) == 5 && std::fread(&t, sizeof(double), 1, f) == 1;
    ok = ok && hdr[0] == c->dim && hdr[1] == c->N && hdr[2] == c->L && hdr[3] == c->nv && hdr[4] > 0 &&
         hdr[4] <= c->cap;
    const long long per = (long long)c->nv * (c->dim == 1 ? c->N : (c->dim == 2 ? c->N * c->N : c->N * c->N * c->N));
    std::vector<int> lv, co;
    std::vector<double> da;
    if (ok) {
        const size_t n = (size_t)hdr[4];
        lv.resize(n);
        co.resize(n * c->dim);
        da.resize(n * per);
        ok = std::fread(lv.data(), sizeof(int), n, f) == n && std::fread(co.data(), sizeof(int), co.size(), f) == co.size() &&
             std::fread(da.data(), sizeof(double), da.size(), f) == da.size();
    }
    std::fclose(f);
    if (!ok) return fail(c, AMR_ERR_IO, "checkpoint file is short or does not match this context");
    return amr_set_state(c, (int)lv.size(), lv.data(), co.data(), da.data(), t);
}

int amr_get_requests(amr_ctx* c, int* n_refine, int* refine_keys, int* n_coarsen, int* coarsen_keys) {
    GUARD(c);
    if (!n_refine || !n_coarsen) return fail(c, AMR_ERR_ARG, "count pointers required");
    std::vector<Key> req, cand;
    int r = c->precision == 64 ? compute_requests<double>(c, req, cand) : compute_requests<float>(c, req, cand);
    if (r) return r;
    std::sort(req.begin(), req.end(), canon_less);
    std::sort(cand.begin(), cand.end(), canon_less);
    *n_refine = (int)req.size();
    *n_coarsen = (int)cand.size();
    if (refine_keys)
        for (size_t i = 0; i < req.size(); ++i) {
            refine_keys[4 * i] = req[i].l;
            refine_keys[4 * i + 1] = req[i].x;
            refine_keys[4 * i + 2] = req[i].y;
            refine_keys[4 * i + 3] = req[i].z;
        }
    if (coarsen_keys)
        for (size_t i = 0; i < cand.size(); ++i) {
            coarsen_keys[4 * i] = cand[i].l;
            coarsen_keys[4 * i + 1] = cand[i].x;
            coarsen_keys[4 * i + 2] = cand[i].y;
            coarsen_keys[4 * i + 3] = cand[i].z;
        }
    return AMR_OK;
}

// Test hook of the timeout path of the learned-flag kernel, deliberately not
// declared in include/amr.h: `cycles` (> 0) replaces the limit of every role
// wait of its tensor-core pipeline (the tear-down's wait for in-flight MMAs
// keeps the full limit), and `withhold` != 0 makes its MMA thread withhold the
// epilogue's accumulator signal, so that one of those waits cannot complete
// and the kernel must take its abort path (AMR_ERR_TIMEOUT at the next
// regrid). A context that reported the timeout refuses further work.
extern "C" int amr_test_tc_wait(amr_ctx* c, long long cycles, int withhold) {
    GUARD(c);
    if (cycles <= 0) return fail(c, AMR_ERR_ARG, "wait limit must be positive");
    c->grid.tc_wait = cycles;
    c->grid.tc_test = withhold ? 1 : 0;
    return AMR_OK;
}

int amr_plain_requests(amr_ctx* c, int* n_refine) {
    GUARD(c);
    if (!n_refine) return fail(c, AMR_ERR_ARG, "count pointer required");
    *n_refine = 0;
    if (c->L == 1) return AMR_OK;
    std::vector<Key> req, cand;
    const int flagger = c->flagger;
    c->flagger = AMR_FLAG_PLAIN;
    const int r = c->precision == 64 ? compute_requests<double>(c, req, cand) : compute_requests<float>(c, req, cand);
    c->flagger = flagger;
    if (r) return r;
    *n_refine = (int)req.size();
    return AMR_OK;
}

int amr_set_mlp(amr_ctx* c, const float* w, long n) {
    GUARD(c);
    if (!w || n != mlp_n_weights(c->dim)) return fail(c, AMR_ERR_ARG, "weight count does not match the dimension");
    if (!c->mlp_w) {
        c->mlp_w = (float*)dalloc(c, n * sizeof(float));
        if (!c->mlp_w) return fail(c, AMR_ERR_CUDA, "device allocation failed");
    }
    c->mlp_n = n;
    CK(cudaMemcpyAsync(c->mlp_w, w, n * sizeof(float), cudaMemcpyHostToDevice, c->stream), "set mlp");
    CK(cudaStreamSynchronize(c->stream), "set mlp");
    c->h2d += n * sizeof(float);
    return AMR_OK;
}

int amr_flag_stats(amr_ctx* c, long long counts[4]) {
    GUARD(c);
    if (!counts) return AMR_ERR_ARG;
    if (!c->mlp_w) return fail(c, AMR_ERR_STATE, "no learned indicator weights set");
    unsigned long long* d = (unsigned long long*)c->dense_d;     // 4 counters + per-slot scratch flags
    if ((size_t)c->cap + 16 > c->dense_cap * 2) return fail(c, AMR_ERR_STATE, "staging buffer too small");
    CK(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), c->stream), "stats");
    int r;
    cudaError_t e;
    if (c->precision == 64) {
        if ((r = fill_all_levels<double>(c, St<double>(c, 0), 0.0))) return r;
        e = Kernels<double>::flag_stats(c->grid, St<double>(c, 0), c->mlp_w, d, grid_size(c, 1), c->stream);
    } else {
        if ((r = fill_all_levels<float>(c, St<float>(c, 0), 0.0))) return r;
        e = Kernels<float>::flag_stats(c->grid, St<float>(c, 0), c->mlp_w, d, grid_size(c, 1), c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "flag stats");
    unsigned long long hc[4];
    CK(cudaMemcpyAsync(hc, d, sizeof(hc), cudaMemcpyDeviceToHost, c->stream), "stats");
    CK(cudaStreamSynchronize(c->stream), "stats");
    for (int i = 0; i < 4; ++i) counts[i] = (long long)hc[i];
    return AMR_OK;
}

int amr_harvest(amr_ctx* c, long* n, double* samples, uint8_t* labels) {
    GUARD(c);
    if (!n) return AMR_ERR_ARG;
    if (c->dim != 1) return fail(c, AMR_ERR_ARG, "harvest needs a 1D hierarchy");
    const long slots = (long)c->n_leaf * (c->N + 2);
    // samples and labels share the dense staging buffer; valid ones are
    // compacted on the host side of the two-call protocol
    std::vector<double> smp((size_t)slots * 15);
    std::vector<unsigned char> lab((size_t)slots);
    if ((size_t)slots * 16 > c->dense_cap) return fail(c, AMR_ERR_ARG, "too many samples for the staging buffer");
    double* dsm = c->dense_d;
    unsigned char* dlb = reinterpret_cast<unsigned char*>(c->dense_d + (size_t)slots * 15);
    int r;
    cudaError_t e;
    if (c->precision == 64) {
        if ((r = fill_all_levels<double>(c, St<double>(c, 0), 0.0))) return r;
        e = Kernels<double>::harvest(c->grid, St<double>(c, 0), nullptr, dsm, dlb, (int)slots, c->stream);
    } else {
        if ((r = fill_all_levels<float>(c, St<float>(c, 0), 0.0))) return r;
        e = Kernels<float>::harvest(c->grid, St<float>(c, 0), nullptr, dsm, dlb, (int)slots, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "harvest");
    CK(cudaMemcpyAsync(smp.data(), dsm, smp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "harvest");
    CK(cudaMemcpyAsync(lab.data(), dlb, lab.size(), cudaMemcpyDeviceToHost, c->stream), "harvest");
    CK(cudaStreamSynchronize(c->stream), "harvest");
    c->d2h += (long long)(smp.size() * sizeof(double) + lab.size());
    long k = 0;
    for (long i = 0; i < slots; ++i) {
        if (lab[i] == 255) continue;
        if (samples) std::memcpy(samples + 15 * k, smp.data() + 15 * i, 15 * sizeof(double));
        if (labels) labels[k] = lab[i];
        ++k;
    }
    *n = k;
    return AMR_OK;
}

int amr_autotune(amr_ctx* c) {
    GUARD(c);
    return c->precision == 64 ? autotune_impl<double>(c) : autotune_impl<float>(c);
}

int amr_set_tuning(amr_ctx* c, const int params[AMR_TUNE_N]) {
    GUARD(c);
    if (!params) return fail(c, AMR_ERR_ARG, "no parameters");
    for (int i = 0; i < AMR_TUNE_N; ++i) {
        const int v = params[i];
        bool ok;
        if (i == AMR_TUNE_GHOST_CHUNK) ok = v >= 32 && v <= 4096;
        else if (i == AMR_TUNE_RHS_SHAPE)
            ok = v >= 0 && v < (c->precision == 64 ? Kernels<double>::rhs_shapes(c->grid)
                                                   : Kernels<float>::rhs_shapes(c->grid)) &&
                 !(shape_needs_tma(c, v) && !c->tma_ok);
        else ok = v >= 1 && v <= 64;
        if (!ok) return fail(c, AMR_ERR_ARG, "launch parameter out of range");
    }
    for (int i = 0; i < AMR_TUNE_N; ++i) c->tune[i] = params[i];
    c->grid.rhs_shape = c->tune[AMR_TUNE_RHS_SHAPE];
    drop_graphs(c);
    return AMR_OK;
}

int amr_get_tuning(amr_ctx* c, int params[AMR_TUNE_N], float ms[AMR_TUNE_N]) {
    if (!c || !params) return AMR_ERR_ARG;
    for (int i = 0; i < AMR_TUNE_N; ++i) {
        params[i] = c->tune[i];
        if (ms) ms[i] = c->tune_ms[i];
    }
    return AMR_OK;
}

int amr_set_timing(amr_ctx* c, int enable) {
    GUARD(c);
    const bool en = enable != 0;
    if (en == c->timing) return AMR_OK;
    if (en && !c->ev[0][0]) {
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < 5; ++i) CK(cudaEventCreate(&c->ev[s][i]), "event");
        CK(cudaEventCreate(&c->ev_cfl[0]), "event");
        CK(cudaEventCreate(&c->ev_cfl[1]), "event");
        for (int i = 0; i < 3; ++i) CK(cudaEventCreate(&c->ev_rg[i]), "event");
        c->regrid_timed = false;
    }
    // the captured step graphs carry the event-record nodes or not: capture again
    drop_graphs(c);
    c->timing = en;
    return AMR_OK;
}

int amr_get_timing(amr_ctx* c, double ms[AMR_TIMING_SLOTS], int launches[AMR_TIMING_SLOTS]) {
    GUARD(c);
    if (!ms) return AMR_ERR_ARG;
    if (!c->timing) return fail(c, AMR_ERR_STATE, "timing is not enabled");
    if (c->mode != AMR_MODE_BATCHED) return fail(c, AMR_ERR_STATE, "timing covers the batched mode");
    CK(cudaStreamSynchronize(c->stream), "timing");
    for (int i = 0; i < AMR_TIMING_SLOTS; ++i) ms[i] = 0.0;
    for (int s = 0; s < 3; ++s)
        for (int i = 0; i < 4; ++i) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, c->ev[s][i], c->ev[s][i + 1]), "timing");
            ms[i] += t;
        }
    if (c->cfl_timed) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev_cfl[0], c->ev_cfl[1]), "timing");
        ms[4] = t;
    }
    if (c->regrid_timed) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev_rg[1], c->ev_rg[2]), "timing");
        ms[5] = t;
        CK(cudaEventElapsedTime(&t, c->ev_rg[0], c->ev_rg[1]), "timing");
        ms[8] = t;
    }
    ms[6] = c->regrid_ms[1];
    ms[7] = c->regrid_ms[2];
    ms[9] = c->regrid_ms[0];
    if (launches) {
        const int rt = c->regrid_timed ? 1 : 0;
        // restriction: levels L-2..1 per stage (level L-1 is restricted inside the RHS launch)
        const int l[AMR_TIMING_SLOTS] = {3 * c->L, 3, 3, 3 * std::max(c->L - 2, 0), c->cfl_timed ? 2 : 0, rt, 0, 0,
                                         rt * c->regrid_fill_launches, 0};
        for (int i = 0; i < AMR_TIMING_SLOTS; ++i) launches[i] = l[i];
    }
    return AMR_OK;
}

int amr_get_counters(amr_ctx* c, long long* h2d, long long* d2h, long long* kernels) {
    if (!c) return AMR_ERR_ARG;
    if (h2d) *h2d = c->h2d;
    if (d2h) *d2h = c->d2h;
    if (kernels) *kernels = c->kernels;
    return AMR_OK;
}

void amr_destroy(amr_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->ev[0][0]) {
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < 5; ++i) cudaEventDestroy(c->ev[s][i]);
        cudaEventDestroy(c->ev_cfl[0]);
        cudaEventDestroy(c->ev_cfl[1]);
        for (int i = 0; i < 3; ++i) cudaEventDestroy(c->ev_rg[i]);
    }
    if (c->ev_req) cudaEventDestroy(c->ev_req);
    dfree_all(c);
    if (c->meta_h) cudaFreeHost(c->meta_h);
    if (c->req_h) cudaFreeHost(c->req_h);
    if (c->time_h) cudaFreeHost(c->time_h);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* amr_last_error(const amr_ctx* c) { return c ? c->err.c_str() : "null context"; }

int amr_mesh_tables(int dim, const int base_patches[3], const int periodic[3], int max_level, int n,
                    const int* keys, int* tables, long long* n_ints) {
    if (dim < 1 || dim > 3 || !base_patches || !periodic || max_level < 0 || max_level >= MAXL || n < 1 ||
        !keys || !n_ints)
        return AMR_ERR_ARG;
    int bp[3] = {1, 1, 1};
    bool per[3] = {false, false, false};
    for (int d = 0; d < dim; ++d) {
        if (base_patches[d] < 1 || ((long long)base_patches[d] << max_level) >= (1LL << 20)) return AMR_ERR_ARG;
        bp[d] = base_patches[d];
        per[d] = periodic[d] != 0;
    }
    amr_ctx t;                                  // host fields only: no device memory, no stream
    t.dim = dim;
    t.L = max_level + 1;
    t.cap = n;
    t.mesh = Mesh(dim, bp, per, max_level);
    t.mesh.clear();
    for (int i = 0; i < n; ++i) {
        const int* r = keys + 4 * (size_t)i;
        const Key k{r[0], r[1], r[2], r[3]};
        if (k.l < 0 || k.l > max_level) return AMR_ERR_ARG;
        const int cc[3] = {k.x, k.y, k.z};
        for (int d = 0; d < 3; ++d)
            if (cc[d] < 0 || cc[d] >= t.mesh.extent(k.l, d)) return AMR_ERR_ARG;
        if (!t.mesh.insert(k)) return AMR_ERR_MESH;
    }
    if (!t.mesh.check().empty()) return AMR_ERR_MESH;
    const MetaLayout ml(n);
    *n_ints = (long long)ml.total;
    if (!tables) return AMR_OK;
    const std::vector<Key> all = t.mesh.canonical();
    slot_map_clear(&t);
    for (int i = 0; i < n; ++i) slot_map_set(&t, all[i], i);    // slot = canonical index
    t.slot_hi = n;
    std::vector<int> h(ml.total, 0);
    t.meta_h = h.data();
    fill_tables(&t, {});
    t.meta_h = nullptr;
    std::copy(h.begin(), h.end(), tables);
    return AMR_OK;
}

}  // extern "C"
