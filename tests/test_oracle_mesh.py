"""Pins of the oracle's hierarchy rules (Sec. 4.3: R1, R2, Algorithm 1 and the
coarsening rule) against the paper's figures and brute force (no GPU)."""
import itertools
import json
import os
import random

import pytest

from oracle.mesh import Mesh, canon

GOLD = os.path.join(os.path.dirname(__file__), 'golden')


def mesh_from_refined(dim, base, periodic, max_level, refined):
    """Mesh whose refined (non-leaf) patches are exactly `refined` (which must be
    closed under taking parents)."""
    m = Mesh(dim, base, periodic, max_level)
    for k in sorted(refined, key=canon):
        assert k in m.patches, k
        for ch in m.children(k):
            m.patches.add(ch)
    return m


def refined_of(m):
    return {k for k in m.patches if m.has_children(k)}


def least_valid_refined(m0, requests):
    """Least set of refined patches containing m0's and the requests such that
    every refined patch has its whole Moore neighbourhood (R2): plain Kleene
    iteration, independent of Algorithm 1's recursion."""
    S = refined_of(m0) | set(requests)
    while True:
        m = mesh_from_refined(m0.dim, m0.base, m0.periodic, m0.max_level, S)
        add = set()
        for P in S:
            for q in m.moore(P):
                if q not in m.patches:
                    add.add(Mesh.parent(q))
        if not add - S:
            return S
        S |= add


def test_paper_refinement_figure():
    g = json.load(open(os.path.join(GOLD, 'refine_figure.json')))
    before = {(l, (c[0], c[1], 0)) for l, c in g['before']['refined']}
    m = mesh_from_refined(2, g['base'], (False, False), g['levels'] - 1, before)
    assert m.violations() == []
    l, c = g['request']
    created = m.refine([(l, (c[0], c[1], 0))])
    after = {(l, (c[0], c[1], 0)) for l, c in g['after']['refined']}
    assert refined_of(m) == after
    assert [len(m.level_list(l)) for l in range(3)] == g['after']['n_patches']
    assert m.violations() == []
    assert len(created) == 4 * 4


def test_paper_valid_figure():
    g = json.load(open(os.path.join(GOLD, 'valid_figure.json')))
    ref = {(l, (c[0], c[1], 0)) for l, c in g['refined']}
    m = mesh_from_refined(2, g['base'], (False, False), g['levels'] - 1, ref)
    assert m.violations() == []
    # one level deeper at a corner child without its neighbours breaks R2
    m2 = mesh_from_refined(2, g['base'], (False, False), 2, ref | {(1, (2, 2, 0))})
    assert any(v[0] == 'R2' for v in m2.violations())


def all_valid_meshes_1d(nbase, max_level, periodic):
    """Every valid 1D mesh: enumerate refined sets level by level."""
    base = Mesh(1, (nbase,), (periodic,), max_level)
    out = [set()]
    for lev in range(max_level):
        nxt = []
        for S in out:
            m = mesh_from_refined(1, (nbase,), (periodic,), max_level, S)
            leaves = [k for k in m.level_list(lev)]
            for bits in itertools.product((0, 1), repeat=len(leaves)):
                T = S | {k for k, b in zip(leaves, bits) if b}
                nxt.append(T)
        out = nxt
    valid = []
    for S in out:
        m = mesh_from_refined(1, (nbase,), (periodic,), max_level, S)
        if not m.violations():
            valid.append(S)
    assert base.violations() == []
    return valid


@pytest.mark.parametrize('periodic', [False, True])
def test_algorithm1_is_least_fixed_point_1d_exhaustive(periodic):
    nb, ml = 4, 2
    meshes = all_valid_meshes_1d(nb, ml, periodic)
    assert len(meshes) > 10
    n_cases = 0
    for S in meshes:
        m0 = mesh_from_refined(1, (nb,), (periodic,), ml, S)
        leaves = [k for k in m0.canonical() if m0.is_leaf(k) and k[0] < ml]
        for bits in itertools.product((0, 1), repeat=len(leaves)):
            req = [k for k, b in zip(leaves, bits) if b]
            m = mesh_from_refined(1, (nb,), (periodic,), ml, S)
            created = m.refine(req)
            assert m.violations() == []
            want = least_valid_refined(m0, req)
            assert refined_of(m) == want
            assert created == set(m.patches) - set(m0.patches)
            n_cases += 1
    assert n_cases > 100


def random_valid_mesh(rng, dim, base, periodic, max_level, n_req):
    m = Mesh(dim, base, periodic, max_level)
    for _ in range(n_req):
        leaves = [k for k in m.canonical() if m.is_leaf(k) and k[0] < max_level]
        m.refine([rng.choice(leaves)])
    return m


@pytest.mark.parametrize('dim,base,periodic', [
    (2, (3, 3), (False, False)), (2, (2, 2), (True, True)), (2, (4, 2), (True, False)),
    (3, (2, 2, 2), (False, False, False))])
def test_algorithm1_random_2d_3d(dim, base, periodic):
    rng = random.Random(7)
    for trial in range(30 if dim == 2 else 8):
        m0 = random_valid_mesh(rng, dim, base, periodic, 2, rng.randint(0, 4))
        assert m0.violations() == []
        leaves = [k for k in m0.canonical() if m0.is_leaf(k) and k[0] < 2]
        req = rng.sample(leaves, min(len(leaves), rng.randint(1, 4)))
        want = least_valid_refined(m0, req)
        results = []
        for shuffle in range(3):
            m = mesh_from_refined(dim, m0.base, periodic, 2, refined_of(m0))
            r = list(req)
            rng.shuffle(r)
            # process in a shuffled order, one request at a time: confluence
            for k in r:
                m.refine([k])
            assert m.violations() == []
            results.append(refined_of(m))
        assert all(x == want for x in results)


@pytest.mark.parametrize('dim,base,periodic', [
    (1, (4,), (False,)), (2, (3, 3), (False, False)), (2, (2, 2), (True, True)),
    (3, (2, 2, 2), (True, False, False))])
def test_coarsening_rule_valid_and_maximal(dim, base, periodic):
    rng = random.Random(11)
    for trial in range(25):
        m = random_valid_mesh(rng, dim, base, periodic, 2, rng.randint(1, 6))
        cands = [k for k in m.canonical() if m.has_children(k)
                 and all(m.is_leaf(x) for x in m.children(k))]
        cands = rng.sample(cands, rng.randint(0, len(cands)))
        base0 = set(m.level_list(0))
        m.coarsen(cands, set())
        assert m.violations() == []
        assert set(m.level_list(0)) == base0                           # R1
        for P in cands:
            if m.has_children(P) and all(m.is_leaf(x) for x in m.children(P)):
                # rejected: deleting its children now would break R2
                trial_mesh = mesh_from_refined(dim, m.base, periodic, 2, refined_of(m) - {P})
                assert trial_mesh.violations() != [], P


@pytest.mark.parametrize('dim,base,periodic', [
    (1, (4,), (False,)), (2, (3, 3), (False, False)), (2, (2, 2), (True, True))])
def test_coarsening_order_independent(dim, base, periodic):
    # one candidate at a time, in random order, repeated until nothing changes,
    # reaches the same mesh as the pass-wise evaluation
    rng = random.Random(5)
    for trial in range(25):
        m = random_valid_mesh(rng, dim, base, periodic, 2, rng.randint(1, 6))
        cands = [k for k in m.canonical() if m.has_children(k)
                 and all(m.is_leaf(x) for x in m.children(k))]
        S = refined_of(m)
        m1 = mesh_from_refined(dim, m.base, periodic, 2, S)
        m1.coarsen(cands, set())
        m2 = mesh_from_refined(dim, m.base, periodic, 2, S)
        changed = True
        while changed:
            changed = False
            order = list(cands)
            rng.shuffle(order)
            for k in order:
                if m2.coarsen_allowed(k, set()):
                    for x in m2.children(k):
                        m2.patches.discard(x)
                    changed = True
        assert m1.patches == m2.patches


def test_coarsening_keeps_just_created():
    m = Mesh(2, (2, 2), (False, False), 2)
    created = m.refine([(0, (0, 0, 0))])
    assert created
    m.coarsen([(0, (0, 0, 0))], created)
    assert m.has_children((0, (0, 0, 0)))
    m.coarsen([(0, (0, 0, 0))], set())
    assert not m.has_children((0, (0, 0, 0)))


def test_printed_algorithm2_would_block_2x2_block():
    # the printed Algorithm 2 rejects P if any Moore neighbour has children;
    # the text rule lets a 2x2 block of refined level-0 patches coarsen
    m = Mesh(2, (2, 2), (False, False), 1)
    m.refine(m.level_list(0))
    assert len(m.level_list(1)) == 16
    m.coarsen(m.level_list(0), set())
    assert len(m.level_list(1)) == 0
