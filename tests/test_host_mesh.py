"""The host half of the library's regrid (amr_mesh_close: Algorithm 1 and the
coarsening rule of Sec. 4.3, in C++) against the oracle's hierarchy rules on
random hierarchies, requests and candidates, and its argument checks. Host
code only: runs without a GPU."""
import ctypes as C
import random

import numpy as np
import pytest

from oracle.mesh import Mesh, canon


@pytest.fixture(scope='module')
def lib():
    from paper_2508_05020_gb300 import build
    build.build()
    from paper_2508_05020_gb300 import amr
    return amr


def rows(keys):
    return [[l, c[0], c[1], c[2]] for l, c in sorted(keys, key=canon)]


def random_mesh(rng, dim, base, periodic, max_level, n_refine):
    m = Mesh(dim, base, periodic, max_level)
    for _ in range(n_refine):
        leaves = [k for k in m.canonical() if m.is_leaf(k) and k[0] < max_level]
        if leaves:
            m.refine([rng.choice(leaves)])
    return m


CASES = [
    (1, (4,), (False,), 3),
    (1, (3,), (True,), 3),
    (2, (3, 3), (False, False), 2),
    (2, (2, 3), (True, False), 2),
    (2, (2, 2), (True, True), 3),
    (3, (2, 2, 2), (False, False, False), 2),
    (3, (2, 1, 2), (True, True, False), 2),
]


@pytest.mark.parametrize('dim,base,periodic,max_level', CASES)
def test_matches_the_oracle_on_random_regrids(lib, dim, base, periodic, max_level):
    # the library's closure and coarsening against the oracle's on the same
    # hierarchy, requests and candidates (given in shuffled order): the same
    # resulting patch list, and counts that add up
    rng = random.Random(17 * dim + max_level)
    changed = 0
    for trial in range(40 if dim < 3 else 12):
        m = random_mesh(rng, dim, base, periodic, max_level, rng.randint(0, 8))
        assert m.violations() == []
        keys = rows(m.patches)
        leaves = sorted((k for k in m.patches if m.is_leaf(k)), key=canon)
        parents = sorted((k for k in m.patches if m.has_children(k)), key=canon)
        req = rng.sample(leaves, rng.randint(0, min(4, len(leaves))))
        cand = rng.sample(parents, rng.randint(0, len(parents)))
        # requests the rule skips (a patch with children, an absent child of a
        # leaf) and candidates it rejects (leaves)
        if parents and rng.random() < 0.3:
            req.append(rng.choice(parents))
        absent = [c for k in leaves if k[0] < max_level for c in m.children(k)]
        if absent and rng.random() < 0.3:
            req.append(rng.choice(absent))
        cand += rng.sample(leaves, min(2, len(leaves)))
        rng.shuffle(req)
        rng.shuffle(cand)
        rng.shuffle(keys)
        got, n_created, n_deleted = lib.mesh_close(dim, base, periodic, max_level, keys, rows(req), rows(cand))
        n0 = len(m.patches)
        created = m.refine(req)
        deleted = m.coarsen(cand, created)
        assert m.violations() == []
        assert got.tolist() == rows(m.patches)
        assert (n_created, n_deleted) == (len(created), len(deleted))
        assert len(got) == n0 + n_created - n_deleted
        changed += bool(created or deleted)
    assert changed >= 5


def keys_1d(*pairs):
    return [[l, x, 0, 0] for l, x in pairs]


def test_invalid_hierarchies_are_refused(lib):
    base = [(0, 0), (0, 1), (0, 2), (0, 3)]
    cases = [
        base[1:],                                                  # a level-0 patch missing (R1)
        base + [(1, 0)],                                           # an incomplete sibling group
        base + [(1, 2), (1, 3), (2, 6), (2, 7)],                   # R2: (1, 3) refined, (1, 4) absent
        base + [(0, 1)],                                           # a key given twice
    ]
    for keys in cases:
        with pytest.raises(lib.AMRError) as e:
            lib.mesh_close(1, (4,), (False,), 2, keys_1d(*keys))
        assert e.value.code == -7, keys


def test_invalid_arguments_are_refused(lib):
    ok = keys_1d((0, 0), (0, 1), (0, 2), (0, 3))
    bad = [
        dict(dim=0),
        dict(dim=4),
        dict(max_level=-1),
        dict(max_level=8),
        dict(base=(1 << 19,)),                                     # extent 2^20 at level 1
        dict(base=(0,)),
        dict(keys=ok + [[3, 0, 0, 0]]),                            # beyond the finest level
        dict(keys=ok + [[1, 8, 0, 0]]),                            # outside the domain
        dict(keys=ok + [[1, 0, 1, 0]]),                            # an unused dimension
        dict(refine=[[0, -1, 0, 0]]),
        dict(candidates=[[0, 4, 0, 0]]),
    ]
    for b in bad:
        a = dict(dim=1, base=(4,), max_level=1 if 'base' in b and b['base'][0] > 4 else 2, keys=ok,
                 refine=(), candidates=())
        a.update(b)
        with pytest.raises(lib.AMRError) as e:
            lib.mesh_close(a['dim'], a['base'], (False,), a['max_level'], a['keys'], a['refine'], a['candidates'])
        assert e.value.code == -1, b


def test_output_capacity_and_counts(lib):
    # the two-call protocol: too small an output reports the size and writes nothing
    L = lib.load()
    bp = np.array([4, 1, 1], dtype=np.int32)
    per = np.zeros(3, dtype=np.int32)
    keys = np.array(keys_1d((0, 0), (0, 1), (0, 2), (0, 3)), dtype=np.int32)
    req = np.array(keys_1d((0, 1)), dtype=np.int32)
    out = np.full((5, 4), -9, dtype=np.int32)
    n_out, n_cr, n_del = C.c_int(-1), C.c_int(-1), C.c_int(-1)
    rc = L.amr_mesh_close(1, lib._ptr(bp), lib._ptr(per), 2, 4, lib._ptr(keys), 1, lib._ptr(req), 0, None, 5,
                          C.byref(n_out), lib._ptr(out), C.byref(n_cr), C.byref(n_del))
    assert rc == -2 and n_out.value == 6 and n_cr.value == 2 and n_del.value == 0
    assert np.all(out == -9)
    out = np.zeros((6, 4), dtype=np.int32)
    rc = L.amr_mesh_close(1, lib._ptr(bp), lib._ptr(per), 2, 4, lib._ptr(keys), 1, lib._ptr(req), 0, None, 6,
                          C.byref(n_out), lib._ptr(out), None, None)
    assert rc == 0
    assert out.tolist() == keys_1d((0, 0), (0, 1), (0, 2), (0, 3), (1, 2), (1, 3))


def expected_tables(m):
    """The tables of include/amr.h for the oracle mesh m, slot = canonical
    index, written from the definitions: neighbours by offset (wrapped
    across periodic sides, -2 outside), parent, children, face flags and the
    finer patches across each face of a leaf next to a refined patch."""
    keys = sorted(m.patches, key=canon)
    slot = {k: i for i, k in enumerate(keys)}
    n, dim = len(keys), m.dim
    nbr = np.full((n, 27), -9)
    child = np.full((n, 8), -1)
    parent = np.full(n, -1)
    pflag = np.zeros(n, dtype=np.int64)
    rl, rf = [], []
    for s, k in enumerate(keys):
        l, c = k
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    o = (ox, oy, oz)
                    e = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)
                    if any(o[d] != 0 for d in range(dim, 3)):
                        nbr[s, e] = -2                                     # unused dimensions
                        continue
                    q = m.wrap(l, tuple(c[d] + o[d] for d in range(3)))
                    nbr[s, e] = -2 if q is None else slot.get((l, q), -1)
        if l > 0:
            parent[s] = slot[Mesh.parent(k)]
        if m.has_children(k):
            pflag[s] |= 1
            for j, x in enumerate(m.children(k)):
                child[s, j] = slot[x]
        faces = np.full((6, 4), -1)
        item = False
        for d in range(dim):
            for side in (0, 1):
                q = m.wrap(l, tuple(c[e] + ((1 if side else -1) if e == d else 0) for e in range(3)))
                if q is None:
                    continue
                if m.is_leaf(k) and (l, q) in m.patches and m.has_children((l, q)):
                    pflag[s] |= 1 << (8 + 2 * d + side)
                    item = True
                    # the children of q touching the shared face, in canonical order
                    touch = [x for x in m.children((l, q)) if x[1][d] == 2 * q[d] + (0 if side else 1)]
                    for j, x in enumerate(sorted(touch, key=canon)):
                        faces[2 * d + side, j] = slot[x]
                if l > 0 and (l, q) not in m.patches:
                    pflag[s] |= 1 << (8 + 2 * d + side)
        if item:
            rl.append(s)
            rf.append(faces)
    leaves = [slot[k] for k in keys if m.is_leaf(k)]
    off = [sum(1 for k in keys if k[0] < l) for l in range(9)]
    return dict(level=[k[0] for k in keys], coord=[x for k in keys for x in k[1]], nbr=nbr, parent=parent,
                child=child, pflag=pflag, all_list=list(range(n)), level_off=off, leaf_list=leaves,
                counts=[n, len(leaves), len(rl), 0], reflux_list=rl, reflux_fine=rf)


@pytest.mark.parametrize('dim,base,periodic,max_level', CASES)
def test_metadata_tables_match_their_definitions(lib, dim, base, periodic, max_level):
    rng = random.Random(29 * dim + max_level)
    items = 0
    for trial in range(15 if dim < 3 else 6):
        m = random_mesh(rng, dim, base, periodic, max_level, rng.randint(0, 8))
        keys = rows(m.patches)
        rng.shuffle(keys)
        t = lib.mesh_tables(dim, base, periodic, max_level, keys)
        e = expected_tables(m)
        n = len(m.patches)
        for name in ('level', 'coord', 'parent', 'pflag', 'all_list', 'level_off', 'counts'):
            assert t[name].tolist() == list(np.asarray(e[name]).tolist()), name
        assert np.array_equal(t['nbr'].reshape(n, 27), e['nbr'])
        assert np.array_equal(t['child'].reshape(n, 8), e['child'])
        nl, nr = e['counts'][1], e['counts'][2]
        assert t['leaf_list'][:nl].tolist() == e['leaf_list']
        assert t['reflux_list'][:nr].tolist() == e['reflux_list']
        fine = t['reflux_fine'].reshape(n, 6, 4)[:nr]
        for i in range(nr):
            assert np.array_equal(fine[i], e['reflux_fine'][i]), i
        items += nr
    if max_level > 0:
        assert items > 0
