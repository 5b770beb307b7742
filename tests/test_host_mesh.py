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
