// Host-side patch hierarchy (Sec. 4.2-4.3): the active patch set keyed by
// (level, integer patch coordinates), rules R1/R2, Algorithm 1 (recursive
// refinement) and the coarsening rule of Sec. 4.3.
#pragma once
#include <cstdint>
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
    std::unordered_set<uint64_t> patches;

    int extent(int level, int d) const { return d < dim ? base[d] << level : 1; }
    bool exists(const Key& k) const { return patches.count(pack(k)) != 0; }
    // wrap coordinates across periodic dimensions; false if outside the domain
    bool wrap(Key& k) const;
    // in-domain Moore-neighbour positions (wrapped), excluding the patch itself
    std::vector<Key> moore(const Key& k) const;
    std::vector<Key> children(const Key& k) const;   // (z, y, x)-lexicographic, x fastest
    static Key parent(const Key& k) { return Key{k.l - 1, k.x >> 1, k.y >> 1, k.z >> 1}; }
    bool has_children(const Key& k) const { return exists(children(k)[0]); }
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
