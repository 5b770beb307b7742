// Host-side patch hierarchy: Algorithm 1 and the coarsening rule of Sec. 4.3.
#include "amr_mesh.h"

#include "amr.h"

#include <algorithm>
#include <sstream>

namespace amr {

Mesh::Mesh(int dim_, const int base_[3], const bool periodic_[3], int max_level_) : dim(dim_), max_level(max_level_) {
    for (int d = 0; d < 3; ++d) {
        base[d] = d < dim ? base_[d] : 1;
        periodic[d] = d < dim ? periodic_[d] : false;
    }
    long long o = 0;
    for (int l = 0; l <= max_level; ++l) {
        lvl_off[l] = o;
        o += (long long)extent(l, 0) * extent(l, 1) * extent(l, 2);
    }
    for (int l = max_level + 1; l < 9; ++l) lvl_off[l] = o;
    if (o <= kDenseMax) present.assign((size_t)o, 0);
    // R1: the level-0 Cartesian layout is the permanent scaffold
    for (int z = 0; z < base[2]; ++z)
        for (int y = 0; y < base[1]; ++y)
            for (int x = 0; x < base[0]; ++x) insert(Key{0, x, y, z});
}

bool Mesh::wrap(Key& k) const {
    int* c[3] = {&k.x, &k.y, &k.z};
    for (int d = 0; d < 3; ++d) {
        if (d >= dim) {
            if (*c[d] != 0) return false;
            continue;
        }
        const int n = extent(k.l, d);
        if (*c[d] < 0 || *c[d] >= n) {
            if (!periodic[d]) return false;
            *c[d] = ((*c[d] % n) + n) % n;
        }
    }
    return true;
}

std::vector<Key> Mesh::moore(const Key& k) const {
    std::vector<Key> out;
    const int rz = dim == 3 ? 1 : 0, ry = dim >= 2 ? 1 : 0;
    for (int oz = -rz; oz <= rz; ++oz)
        for (int oy = -ry; oy <= ry; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                if (!ox && !oy && !oz) continue;
                Key q{k.l, k.x + ox, k.y + oy, k.z + oz};
                if (!wrap(q)) continue;
                if (q == k) continue;
                if (std::find(out.begin(), out.end(), q) == out.end()) out.push_back(q);
            }
    return out;
}

std::vector<Key> Mesh::children(const Key& k) const {
    std::vector<Key> out;
    const int nz = dim == 3 ? 2 : 1, ny = dim >= 2 ? 2 : 1;
    for (int sz = 0; sz < nz; ++sz)
        for (int sy = 0; sy < ny; ++sy)
            for (int sx = 0; sx < 2; ++sx)
                out.push_back(Key{k.l + 1, 2 * k.x + sx, dim >= 2 ? 2 * k.y + sy : 0, dim == 3 ? 2 * k.z + sz : 0});
    return out;
}

std::vector<Key> Mesh::canonical() const {
    std::vector<Key> out;
    out.reserve(patches.size());
    if (dense() && (long long)patches.size() * 16 >= positions()) {
        // the position order is the canonical order
        for (int l = 0; l <= max_level; ++l) {
            const int ex = extent(l, 0), ey = extent(l, 1), ez = extent(l, 2);
            long long p = lvl_off[l];
            for (int z = 0; z < ez; ++z)
                for (int y = 0; y < ey; ++y)
                    for (int x = 0; x < ex; ++x, ++p)
                        if (present[(size_t)p]) out.push_back(Key{l, x, y, z});
        }
        return out;
    }
    for (uint64_t v : patches) out.push_back(unpack(v));
    std::sort(out.begin(), out.end(), canon_less);
    return out;
}

std::string Mesh::check() const {
    std::ostringstream why;
    for (int z = 0; z < base[2]; ++z)
        for (int y = 0; y < base[1]; ++y)
            for (int x = 0; x < base[0]; ++x)
                if (!exists(Key{0, x, y, z})) {
                    why << "level-0 patch (" << x << "," << y << "," << z << ") missing (R1)";
                    return why.str();
                }
    for (uint64_t v : patches) {
        const Key k = unpack(v);
        if (k.l < 0 || k.l > max_level) {
            why << "patch beyond the finest level";
            return why.str();
        }
        Key w = k;
        if (!wrap(w) || !(w == k)) {
            why << "patch outside the domain";
            return why.str();
        }
        if (k.l > 0 && !exists(parent(k))) {
            why << "patch without parent";
            return why.str();
        }
        const auto ch = children(k);
        int present = 0;
        for (const auto& c : ch) present += exists(c);
        if (present != 0 && present != (int)ch.size()) {
            why << "incomplete sibling group";
            return why.str();
        }
        if (present) {
            for (const auto& q : moore(k))
                if (!exists(q)) {
                    why << "R2 violated: a refined patch lacks a Moore neighbour";
                    return why.str();
                }
        }
    }
    return std::string();
}

// Algorithm 1 (RefinePatch): before a leaf gets its children, every missing
// position of its Moore neighbourhood is created by refining the parent's
// corresponding neighbour, recursively (R2).
void Mesh::refine_patch(const Key& k, std::vector<Key>& created) {
    if (!is_leaf(k)) return;
    for (const auto& q : moore(k)) {
        if (!exists(q)) refine_patch(parent(q), created);
    }
    for (const auto& c : children(k)) {
        if (insert(c)) created.push_back(c);
    }
}

std::vector<Key> Mesh::refine(std::vector<Key> requests) {
    std::sort(requests.begin(), requests.end(), canon_less);
    std::vector<Key> created;
    for (const auto& k : requests) {
        if (exists(k) && is_leaf(k) && k.l < max_level) refine_patch(k, created);
    }
    return created;
}

// Sec. 4.3: the children of P are deleted iff P has children, they are all
// leaves (and were not created by this regrid), and none of them lies in the
// Moore neighbourhood of another level-(l+1) patch that has children.
bool Mesh::coarsen_allowed(const Key& k, const std::unordered_set<uint64_t>& just_created) const {
    if (!exists(k) || !has_children(k)) return false;
    const auto ch = children(k);
    for (const auto& c : ch) {
        if (!is_leaf(c)) return false;
        if (just_created.count(pack(c))) return false;
    }
    for (const auto& c : ch) {
        for (const auto& D : moore(c)) {
            if (std::find(ch.begin(), ch.end(), D) != ch.end()) continue;
            if (exists(D) && has_children(D)) return false;
        }
    }
    return true;
}

// Passes of the rule over the pending candidates on the current mesh, each
// pass deleting its accepted children together, until a pass accepts none:
// deletions only remove "has children" facts, so the outcome does not depend
// on the order of the candidates.
std::vector<Key> Mesh::coarsen(const std::vector<Key>& candidates, const std::unordered_set<uint64_t>& just_created) {
    std::vector<Key> pending = candidates;
    std::sort(pending.begin(), pending.end(), canon_less);
    pending.erase(std::unique(pending.begin(), pending.end()), pending.end());
    std::vector<Key> deleted;
    while (true) {
        std::vector<Key> accept, rest;
        for (const auto& k : pending) (coarsen_allowed(k, just_created) ? accept : rest).push_back(k);
        if (accept.empty()) break;
        for (const auto& k : accept)
            for (const auto& c : children(k)) {
                erase(c);
                deleted.push_back(c);
            }
        pending.swap(rest);
    }
    return deleted;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// amr_mesh_close: the host half of a regrid on a caller's hierarchy.
// ---------------------------------------------------------------------------
namespace {

// a (level, cx, cy, cz) row inside the level range and the domain (not wrapped)
bool key_of_row(const amr::Mesh& m, const int* r, amr::Key& k) {
    k = amr::Key{r[0], r[1], r[2], r[3]};
    if (k.l < 0 || k.l > m.max_level) return false;
    const int c[3] = {k.x, k.y, k.z};
    for (int d = 0; d < 3; ++d)
        if (c[d] < 0 || c[d] >= m.extent(k.l, d)) return false;
    return true;
}

}  // namespace

extern "C" int amr_mesh_close(int dim, const int base_patches[3], const int periodic[3], int max_level, int n,
                              const int* keys, int n_refine, const int* refine_keys, int n_candidates,
                              const int* candidate_keys, int cap_out, int* n_out, int* out_keys, int* n_created,
                              int* n_deleted) {
    using amr::Key;
    if (dim < 1 || dim > 3 || !base_patches || !periodic || max_level < 0 || max_level > 7 || n < 0 ||
        n_refine < 0 || n_candidates < 0 || cap_out < 0 || !n_out)
        return AMR_ERR_ARG;
    if ((n > 0 && !keys) || (n_refine > 0 && !refine_keys) || (n_candidates > 0 && !candidate_keys) ||
        (cap_out > 0 && !out_keys))
        return AMR_ERR_ARG;
    int base[3] = {1, 1, 1};
    bool per[3] = {false, false, false};
    for (int d = 0; d < dim; ++d) {
        if (base_patches[d] < 1 || ((long long)base_patches[d] << max_level) >= (1LL << 20)) return AMR_ERR_ARG;
        base[d] = base_patches[d];
        per[d] = periodic[d] != 0;
    }
    amr::Mesh m(dim, base, per, max_level);
    m.clear();
    for (int i = 0; i < n; ++i) {
        Key k;
        if (!key_of_row(m, keys + 4 * (size_t)i, k)) return AMR_ERR_ARG;
        if (!m.insert(k)) return AMR_ERR_MESH;
    }
    if (!m.check().empty()) return AMR_ERR_MESH;
    std::vector<Key> req(n_refine), cand(n_candidates);
    for (int i = 0; i < n_refine; ++i)
        if (!key_of_row(m, refine_keys + 4 * (size_t)i, req[i])) return AMR_ERR_ARG;
    for (int i = 0; i < n_candidates; ++i)
        if (!key_of_row(m, candidate_keys + 4 * (size_t)i, cand[i])) return AMR_ERR_ARG;
    const std::vector<Key> created = m.refine(req);
    std::unordered_set<uint64_t> just;
    for (const auto& k : created) just.insert(amr::pack(k));
    const std::vector<Key> deleted = m.coarsen(cand, just);
    *n_out = (int)m.patches.size();
    if (n_created) *n_created = (int)created.size();
    if (n_deleted) *n_deleted = (int)deleted.size();
    if ((long long)m.patches.size() > cap_out) return AMR_ERR_POOL;
    const std::vector<Key> all = m.canonical();
    for (size_t i = 0; i < all.size(); ++i) {
        out_keys[4 * i + 0] = all[i].l;
        out_keys[4 * i + 1] = all[i].x;
        out_keys[4 * i + 2] = all[i].y;
        out_keys[4 * i + 3] = all[i].z;
    }
    return AMR_OK;
}
