"""Parity at the full sizes of the 3D blast benchmark (128^3 base, 3 levels,
16^3 patches), the double Mach reflection (512 x 128 base, 4 levels) and the
four-quadrant problem (256^2 base, 3 levels), in the launch configuration
bench.py times (batched step in a CUDA graph, autotuned launch parameters,
amr_advance; FP32 fields with the learned flags and keep margin 12, the
blast also with the bench's lookahead network regridding every 4 steps). The
oracle cannot run these sizes, so it checks sampled outputs it computes one
by one (per-patch flags and requests from the GPU's own state) and
properties that hold at any size (conservation, mesh validity, FP32 against
the bit-exact FP64 path)."""
import os

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEEP = 12.0                     # keep margin of the learned flags in bench.py
BF16_MARGIN = 0.02              # logits this close to a threshold may round either way


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


FULL = ['blast3d', 'dmr', 'riemann2d']


def bf16(x):
    """Round to the nearest BF16 (ties to even), as __float2bfloat16_rn does."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def oracle_from_gpu(w, g):
    """An oracle hierarchy holding the GPU's patches and interiors (FP64
    images of its values), ghosts filled by the oracle."""
    from oracle.amr import Oracle
    r = Oracle(w, init=False)
    r.mesh.patches = set()
    r.U = {}
    t, _, _ = g.diag()
    for l in range(w['levels']):
        c, x = g.get_level(l)
        for i in range(len(c)):
            key = (l, tuple(int(c[i][d]) if d < r.dim else 0 for d in range(3)))
            r.mesh.patches.add(key)
            A = np.zeros(r.slot_shape())
            A[r.inner()] = x[i].reshape(A[r.inner()].shape)
            r.U[key] = A
    r.t = t
    r.fill_ghosts(r.U, r.t)
    return r


def keys_of(rows):
    return {(int(x[0]), (int(x[1]), int(x[2]), int(x[3]))) for x in rows}


def sample(rng, items, n):
    items = sorted(items)
    idx = rng.choice(len(items), size=min(n, len(items)), replace=False)
    return [items[i] for i in sorted(idx)]


@pytest.mark.parametrize('name', ['blast3d', 'riemann2d'])
def test_fullsize_fp64_conserves_and_keeps_a_valid_mesh(name):
    # the same hierarchy and kernels in a periodic box (an outflow side lets
    # the Rusanov dissipation of the seeded density perturbation carry mass
    # out): every total is kept to round-off, and the mesh stays valid
    from paper_2508_05020_gb300.amr import AMR
    w0 = workload(name)
    w = workload(name, bc=tuple(('periodic', 'periodic') if d < w0['dim'] else w0['bc'][d] for d in range(3)))
    g = AMR(w, precision=64)
    _, c0, _ = g.diag()
    g.advance(3)
    t, c1, ppl = g.diag()
    nv = w['dim'] + 2
    assert t > 0.0
    assert abs(c1[0] - c0[0]) <= 1e-12 * c0[0]
    assert abs(c1[nv - 1] - c0[nv - 1]) <= 1e-12 * c0[nv - 1]
    assert np.all(np.abs(c1[1:nv - 1] - c0[1:nv - 1]) <= 1e-12 * c0[0])
    r = oracle_from_gpu(w, g)
    assert r.mesh.violations() == []
    assert list(ppl[:w['levels']]) == [len(r.mesh.level_list(l)) for l in range(w['levels'])]
    g.close()


@pytest.mark.parametrize('name', FULL)
def test_fullsize_plain_requests_match_oracle_on_sampled_patches(name):
    # FP64 state of the full hierarchy: the oracle's flag of each sampled leaf
    # and the candidate status of each sampled parent equal the GPU's
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name)
    g = AMR(w, precision=64)
    g.advance(2)
    r = oracle_from_gpu(w, g)
    rg, cg = g.requests()
    refine, cand = keys_of(rg), keys_of(cg)
    rng = np.random.default_rng(11)
    leaves = [k for k in r.mesh.patches if r.mesh.is_leaf(k) and k[0] < r.L - 1]
    for k in sample(rng, leaves, 48):
        assert r.anyflag(k)[0] == (k in refine), k
    parents = [k for k in r.mesh.patches if not r.mesh.is_leaf(k)
               and all(r.mesh.is_leaf(x) for x in r.mesh.children(k))]
    assert parents
    for k in sample(rng, parents, 24):
        expect = not any(r.anyflag(x)[1] for x in r.mesh.children(k))
        assert expect == (k in cand), k
    g.close()


def max_logit_bf16(r, q, key):
    """Largest logit over the in-domain band cells of a patch, by the oracle
    network evaluated with the BF16 roundings of the tensor-core kernel."""
    from oracle import mlp
    R, Us, P, cells = mlp.cell_stencils(r, key)
    X = mlp.features(R, Us, P, r.gamma)
    h1 = bf16(np.maximum(bf16(X) @ bf16(q['W1']).T + q['b1'], 0.0))
    z = np.maximum(h1 @ bf16(q['W2']).T + q['b2'], 0.0) @ q['W3'][0] + q['b3'][0]
    ok = np.ones(len(z), dtype=bool)
    for d in range(r.dim):
        gi = key[1][d] * r.N + cells[:, d]
        ok &= (gi >= 0) & (gi < r.mesh.extent(key[0])[d] * r.N)
    return float(np.max(z[ok]))


@pytest.mark.parametrize('name,wname,K', [('blast3d', 'indicator_d{d}_diag_k4.npy', 4),
                                           ('blast3d', 'indicator_d{d}.npy', 1),
                                           ('dmr', 'indicator_d{d}.npy', 1),
                                           ('riemann2d', 'indicator_d{d}.npy', 1)])
def test_fullsize_learned_requests_match_oracle_on_sampled_patches(name, wname, K):
    # FP32, learned flags, keep margin, autotuned, after timed-style steps of
    # amr_advance (the first case is the bench's configuration: the lookahead
    # network regridding every 4 steps); refine bits of sampled leaves below
    # the finest level and candidate status of sampled parents, except where
    # a logit lies within the BF16 margin of its threshold
    from oracle import mlp
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name)
    wf = np.load(os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights',
                              wname.format(d=w['dim']))).astype(np.float32)
    g = AMR(w, precision=32, flagger='mlp', mlp_weights=wf, autotune=True, mlp_keep_margin=KEEP)
    g.advance(3 if K == 1 else 2 * K + 1, regrid=K)
    r = oracle_from_gpu(w, g)
    q = mlp.unflatten(wf.astype(np.float64), mlp.k_in(w['dim']))
    rg, cg = g.requests()
    refine, cand = keys_of(rg), keys_of(cg)
    rng = np.random.default_rng(12)
    leaves = [k for k in r.mesh.patches if r.mesh.is_leaf(k) and k[0] < r.L - 1]
    checked = 0
    for k in sample(rng, leaves, 24):
        z = max_logit_bf16(r, q, k)
        if abs(z) > BF16_MARGIN:
            assert (z > 0.0) == (k in refine), (k, z)
            checked += 1
    assert checked >= 12
    for k in sample(rng, sorted(refine & set(leaves)), 6):      # flagged leaves, whatever the sample held
        z = max_logit_bf16(r, q, k)
        assert z > -BF16_MARGIN, (k, z)
    parents = [k for k in r.mesh.patches if not r.mesh.is_leaf(k)
               and all(r.mesh.is_leaf(x) for x in r.mesh.children(k))]
    checked = 0
    for k in sample(rng, parents, 8):
        zs = [max_logit_bf16(r, q, x) for x in r.mesh.children(k)]
        if all(abs(z + KEEP) > BF16_MARGIN for z in zs):
            assert (not any(z > -KEEP for z in zs)) == (k in cand), (k, zs)
            checked += 1
    assert checked >= 4
    g.close()


@pytest.mark.parametrize('name', FULL)
def test_fullsize_fp32_against_fp64(name):
    # the batched FP32 path against the batched FP64 path (bit-exact with the
    # oracle at the sizes it runs) with the same dt sequence: relative L1(rho)
    # of level 0 (the conservative average of the whole hierarchy) within 1e-5
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name)
    a = AMR(w, precision=64)
    dts = []
    for _ in range(3):
        dts.append(a.step())
        a.regrid()
    _, x64 = a.get_level(0)
    a.close()
    b = AMR(w, precision=32, autotune=True)
    for dt in dts:
        b.step(dt=dt)
        b.regrid()
    _, x32 = b.get_level(0)
    b.close()
    err = np.sum(np.abs(x32[:, 0] - x64[:, 0])) / np.sum(np.abs(x64[:, 0]))
    assert err <= 1e-5, err
