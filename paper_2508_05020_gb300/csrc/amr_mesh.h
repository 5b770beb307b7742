// Host-side patch hierarchy (Sec. 4.2-4.3): the active patch set keyed by
// (level, integer patch coordinates), rules R1/R2, Algorithm 1 (recursive
// refinement) and the coarsening rule of Sec. 4.3.
#pragma once
#include <cstdint>
#include <algorithm>
#include <string>
#include <unordered_set>
#include <vector>

namespace amr {

struct Key {
    int l, x, y, z;
    bool operator==(const Key& o) const { return l == o.l && x == o.x && y == o.y && z == o.z; }
};

// canonical order: level, then lexicographic (z, y, x)
inline bool canon_less(const Key& a, const Key& b) {
    if (a.l != b.l) return a.l < b.l;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
}

inline uint64_t pack(const Key& k) {
    return ((uint64_t)(uint32_t)k.l << 60) | ((uint64_t)(uint32_t)k.z << 40) | ((uint64_t)(uint32_t)k.y << 20) |
           (uint64_t)(uint32_t)k.x;
}
inline Key unpack(uint64_t v) {
    Key k;
    k.l = (int)(v >> 60);
    k.z = (int)((v >> 40) & 0xFFFFF);
    k.y = (int)((v >> 20) & 0xFFFFF);
    k.x = (int)(v & 0xFFFFF);
    return k;
}

class Mesh {
public:
    Mesh() = default;
    Mesh(int dim, const int base[3], const bool periodic[3], int max_level);

    int dim = 1, max_level = 0;
    int base[3] = {1, 1, 1};
    bool periodic[3] = {false, false, false};
    // the patch set; read freely, change only through insert / erase / clear /
    // swap_patches, which keep the position index below in step
    std::unordered_set<uint64_t> patches;
    // Dense position index of every patch position a level can hold: level
    // by level, then lexicographic (z, y, x), i.e. the canonical order. Used
    // (present non-empty) when all positions fit in kDenseMax; a membership
    // test is then one array read.
    static constexpr long long kDenseMax = 1ll << 26;
    long long lvl_off[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<uint8_t> present;

    int extent(int level, int d) const { return d < dim ? base[d] << level : 1; }
    // position of k in the dense index, -1 outside the levels or the domain
    long long pos(const Key& k) const {
        if (k.l < 0 || k.l > max_level) return -1;
        const int ex = extent(k.l, 0), ey = extent(k.l, 1), ez = extent(k.l, 2);
        if (k.x < 0 || k.x >= ex || k.y < 0 || k.y >= ey || k.z < 0 || k.z >= ez) return -1;
        return lvl_off[k.l] + ((long long)k.z * ey + k.y) * ex + k.x;
    }
    long long positions() const { return lvl_off[max_level + 1]; }
    bool dense() const { return !present.empty(); }
    bool exists(const Key& k) const {
        if (dense()) {
            const long long p = pos(k);
            return p >= 0 && present[(size_t)p];
        }
        return patches.count(pack(k)) != 0;
    }
    // false if k is present already (or, with the dense index, outside it)
    bool insert(const Key& k) {
        const long long p = dense() ? pos(k) : 0;
        if (p < 0 || !patches.insert(pack(k)).second) return false;
        if (dense()) present[(size_t)p] = 1;
        return true;
    }
    bool erase(const Key& k) {
        if (!patches.erase(pack(k))) return false;
        if (dense()) present[(size_t)pos(k)] = 0;
        return true;
    }
    void clear() {
        patches.clear();
        std::fill(present.begin(), present.end(), 0);
    }
    void swap_patches(Mesh& o) {
        patches.swap(o.patches);
        present.swap(o.present);
    }
    // wrap coordinates across periodic dimensions; false if outside the domain
    bool wrap(Key& k) const;
    // in-domain Moore-neighbour positions (wrapped), excluding the patch itself
    std::vector<Key> moore(const Key& k) const;
    std::vector<Key> children(const Key& k) const;   // (z, y, x)-lexicographic, x fastest
    static Key parent(const Key& k) { return Key{k.l - 1, k.x >> 1, k.y >> 1, k.z >> 1}; }
    bool has_children(const Key& k) const {     // the first child (all or none exist)
        return exists(Key{k.l + 1, 2 * k.x, dim >= 2 ? 2 * k.y : 0, dim == 3 ? 2 * k.z : 0});
    }
    bool is_leaf(const Key& k) const { return !has_children(k); }
    std::vector<Key> canonical() const;

    // tree structure, R1 (all level-0 patches present) and R2; empty string if valid
    std::string check() const;

    // Algorithm 1 on each request (canonical order); returns the created patches
    std::vector<Key> refine(std::vector<Key> requests);
    // Sec. 4.3 coarsening rule iterated to its fixed point; returns deleted patches
    std::vector<Key> coarsen(const std::vector<Key>& candidates, const std::unordered_set<uint64_t>& just_created);
    bool coarsen_allowed(const Key& k, const std::unordered_set<uint64_t>& just_created) const;

private:
    void refine_patch(const Key& k, std::vector<Key>& created);
};

}  // namespace amr
