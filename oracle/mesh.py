"""Patch hierarchy of the oracle: R1/R2, Algorithm 1 and the coarsening rule.

Test infrastructure (see ``oracle/__init__``). Pure Python on integers.

A patch is the key (level, (cx, cy, cz)) of its integer patch coordinates at
its level (unused dimensions are 0). Level-0 patches form a Cartesian layout
and are the roots of binary trees / quadtrees / octrees (Sec. 4.3); a patch at
level l+1 with coordinates c has the parent (l, c // 2), and a refined patch
owns all 2^d children at once (``child[4]`` in the metadata of Sec. 4.2).
"""
import itertools


class Mesh:
    def __init__(self, dim, base_patches, periodic, max_level):
        self.dim = dim
        self.base = tuple(base_patches) + (1,) * (3 - len(base_patches))
        self.periodic = tuple(periodic)
        self.max_level = max_level          # finest admissible level (L - 1)
        self.patches = set()
        for c in itertools.product(*[range(self.base[d]) if d < dim else [0] for d in (2, 1, 0)]):
            self.patches.add((0, (c[2], c[1], c[0])))

    # ---- geometry -------------------------------------------------------
    def extent(self, level):
        """Patches per dimension at a level."""
        return tuple(self.base[d] * 2 ** level if d < self.dim else 1 for d in range(3))

    def wrap(self, level, c):
        """Wrap patch coordinates across periodic dimensions; None if outside."""
        ext = self.extent(level)
        out = []
        for d in range(3):
            x = c[d]
            if d >= self.dim:
                out.append(0)
                continue
            if x < 0 or x >= ext[d]:
                if not self.periodic[d]:
                    return None
                x %= ext[d]
            out.append(x)
        return tuple(out)

    def offsets(self):
        """Moore-neighbourhood offsets {-1,0,1}^d without 0 (Sec. 4.3)."""
        rng = [(-1, 0, 1) if d < self.dim else (0,) for d in range(3)]
        return [o for o in itertools.product(*rng) if any(o)]

    def moore(self, key):
        """In-domain Moore-neighbour positions of a patch at its own level.

        Positions beyond a non-periodic boundary belong to ghost patches, which
        always satisfy the rules (Sec. 4.3); periodic ones wrap around.
        """
        l, c = key
        out = []
        for o in self.offsets():
            w = self.wrap(l, tuple(c[d] + o[d] for d in range(3)))
            if w is not None and (l, w) != key:
                out.append((l, w))
        return sorted(set(out), key=canon)

    # ---- tree -----------------------------------------------------------
    def children(self, key):
        l, c = key
        rng = [(0, 1) if d < self.dim else (0,) for d in range(3)]
        return [(l + 1, tuple(2 * c[d] + s[d] for d in range(3)))
                for s in (tuple(reversed(t)) for t in itertools.product(*reversed(rng)))]

    @staticmethod
    def parent(key):
        l, c = key
        return (l - 1, tuple(x // 2 for x in c))

    def has_children(self, key):
        return self.children(key)[0] in self.patches

    def is_leaf(self, key):
        return not self.has_children(key)

    def level_list(self, level):
        return sorted((k for k in self.patches if k[0] == level), key=canon)

    def canonical(self):
        return sorted(self.patches, key=canon)

    # ---- rules ----------------------------------------------------------
    def violations(self):
        """List of broken rules: tree structure (all-or-none children, parents
        present) and R2 (a patch with children has its whole Moore neighbourhood
        active, Sec. 4.3). R1 is structural: level-0 patches are never removed."""
        bad = []
        for k in self.patches:
            l, c = k
            if l > 0 and self.parent(k) not in self.patches:
                bad.append(('orphan', k))
            ch = self.children(k)
            present = [x in self.patches for x in ch]
            if any(present) and not all(present):
                bad.append(('partial-children', k))
            if all(present) and l >= self.max_level:
                bad.append(('too-deep', k))
            if all(present):
                for q in self.moore(k):
                    if q not in self.patches:
                        bad.append(('R2', k, q))
        return bad

    # ---- Algorithm 1 ------------------------------------------------------
    def refine_patch(self, key, created):
        """Algorithm 1 (RefinePatch): refine a leaf after making sure its whole
        Moore neighbourhood exists, refining the parent's corresponding
        neighbour recursively where a position is missing (R2)."""
        if not self.is_leaf(key):
            return
        for q in self.moore(key):
            if q not in self.patches:
                # the missing position lies in a child of the parent's neighbour
                r = self.parent(q)
                self.refine_patch(r, created)
        for ch in self.children(key):
            self.patches.add(ch)
            created.add(ch)

    def refine(self, requests):
        """Process refinement requests in canonical order (level, z, y, x).
        Returns the set of patches created."""
        created = set()
        for k in sorted(requests, key=canon):
            if k in self.patches and self.is_leaf(k) and k[0] < self.max_level:
                self.refine_patch(k, created)
        return created

    # ---- coarsening (Sec. 4.3 text rule) ----------------------------------
    def coarsen_allowed(self, key, just_created):
        """Coarsening rule of Sec. 4.3: the children of P can be deleted iff P
        has children, they are all leaves, none was just created, and no
        level-(l+1) patch D outside children(P) that itself has children has a
        child of P in its Moore neighbourhood (that child supports D's R2)."""
        if key not in self.patches or not self.has_children(key):
            return False
        ch = self.children(key)
        if any(not self.is_leaf(x) for x in ch):
            return False
        if any(x in just_created for x in ch):
            return False
        chs = set(ch)
        l = key[0] + 1
        for x in ch:
            # every D whose Moore neighbourhood contains x is a Moore neighbour of x
            for D in self.moore(x):
                if D in chs or D not in self.patches:
                    continue
                if self.has_children(D):
                    return False
        return True

    def coarsen(self, candidates, just_created):
        """Apply the coarsening rule to the requested patches until nothing
        changes: each pass evaluates the rule for every pending candidate on
        the current mesh and deletes the accepted children together. Deleting
        children only removes 'has children' facts, which can only unblock
        other candidates, so the result is the unique greatest fixed point and
        does not depend on the order of the requests. Returns deleted keys."""
        pending = sorted(set(candidates), key=canon)
        deleted = set()
        while True:
            accept = [k for k in pending if self.coarsen_allowed(k, just_created)]
            if not accept:
                return deleted
            for k in accept:
                for x in self.children(k):
                    self.patches.discard(x)
                    deleted.add(x)
            pending = [k for k in pending if k not in accept]


def canon(key):
    """Canonical order: level, then lexicographic (z, y, x) coordinates."""
    l, c = key
    return (l, c[2], c[1], c[0])
