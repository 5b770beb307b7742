"""The learned refinement indicator on the GPU (through the C ABI) against the
FP64 oracle network: features, BF16 tensor-core logits, FP32 gradients,
training, and the fused per-patch flagging inside the AMR hierarchy."""
import numpy as np
import pytest

from synth import mlp_init, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def samples(seed, n):
    rng = np.random.default_rng(seed)
    s = np.empty((n, 5, 3))
    s[:] = rng.uniform(0.5, 2.0, size=(n, 1, 3))
    s[:, :, 1] = rng.normal(0, 0.5, size=(n, 5))
    jump = rng.uniform(size=n) < 0.5
    pos = rng.integers(1, 5, size=n)
    for i in np.nonzero(jump)[0]:
        s[i, pos[i]:, 0] *= rng.uniform(0.3, 3.0)
        s[i, pos[i]:, 2] *= rng.uniform(0.3, 3.0)
    s[:, :, 0] *= 1.0 + 0.01 * rng.normal(size=(n, 5))
    return s


def bf16(x):
    """Round to the nearest BF16 (ties to even), as __float2bfloat16_rn does."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(p):
    from oracle import mlp
    return mlp.flatten(p).astype(np.float32)


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_features_match_oracle(dim):
    from oracle import mlp
    from paper_2508_05020_gb300 import amr
    s = samples(0, 64)
    Xg = amr.mlp_features(dim, 1.4, s)
    Xr = mlp.embedded_features(s, dim, 1.4)
    assert Xg.shape == Xr.shape
    assert np.allclose(Xg, Xr, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_bf16_logits(dim):
    # the oracle network evaluated in FP64 on the BF16-rounded weights,
    # features and hidden activations the tensor-core kernel uses
    from oracle import mlp
    from paper_2508_05020_gb300 import amr
    s = samples(1, 200)
    X = mlp.embedded_features(s, dim, 1.4).astype(np.float32)
    p = mlp_init(0, mlp.k_in(dim))
    w = flat(p)
    z = amr.mlp_infer(dim, X, w)
    q = mlp.unflatten(w.astype(np.float64), mlp.k_in(dim))
    a1 = bf16(X) @ bf16(q['W1']).T + q['b1']
    h1 = bf16(np.maximum(a1, 0.0))
    a2 = h1 @ bf16(q['W2']).T + q['b2']
    zr = np.maximum(a2, 0.0) @ q['W3'][0] + q['b3'][0]
    scale = max(1.0, float(np.sqrt(np.mean(zr ** 2))))
    assert np.max(np.abs(z - zr)) <= 2e-2 * scale
    # and against plain FP64 (no BF16 rounding) within the BF16 error budget
    zf, _ = mlp.forward(q, X.astype(np.float64))
    assert np.max(np.abs(z - zf)) <= 0.1 * scale


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_fp32_gradient_matches_oracle(dim):
    from oracle import mlp
    from paper_2508_05020_gb300 import amr
    s = samples(2, 96)
    X = mlp.embedded_features(s, dim, 1.4)
    y = np.repeat(mlp.plain_flag_1d(s, 0.05, 0.05), 2 * dim).astype(np.float64)
    p = mlp_init(0, mlp.k_in(dim))
    pw = mlp.bce_pos_weight(y)
    lr, gr = mlp.loss_and_grad(p, X, y, pw)
    lg, gg = amr.mlp_grad(dim, X.astype(np.float32), y.astype(np.float32), pw, flat(p))
    gref = mlp.flatten(gr)
    assert abs(lg - lr) <= 1e-5 * max(1.0, abs(lr))
    assert np.linalg.norm(gg - gref) <= 1e-4 * np.linalg.norm(gref)


def test_training_learns_the_plain_flag():
    from oracle import mlp
    from paper_2508_05020_gb300 import amr
    s = samples(3, 4000)
    t = samples(4, 1000)
    dim = 2
    X = amr.mlp_features(dim, 1.4, s)
    y = np.repeat(mlp.plain_flag_1d(s, 0.05, 0.05), 2 * dim).astype(np.float32)
    pw = mlp.bce_pos_weight(y)
    w0 = flat(mlp_init(0, mlp.k_in(dim)))
    w, hist = amr.mlp_train(dim, X, y, pw, w0, epochs=30, batch=256, lr=2e-3, seed=1)
    assert hist[-1] < 0.5 * hist[0]
    Xt = amr.mlp_features(dim, 1.4, t)
    yt = np.repeat(mlp.plain_flag_1d(t, 0.05, 0.05), 2 * dim)
    pred = amr.mlp_infer(dim, Xt, w) > 0
    tp = np.sum(pred & yt)
    recall = tp / max(1, np.sum(yt))
    precision = tp / max(1, np.sum(pred))
    assert recall > 0.9 and precision > 0.8, (recall, precision)


@pytest.mark.parametrize('keep,b3', [(0.0, -0.5), (1.5, -2.5)])
def test_fused_flags_agree_with_oracle_flagger(keep, b3):
    # identical state on both sides; per-patch decisions may differ only where
    # the oracle's largest band logit is within the BF16 margin of zero (the
    # refine bit) or of -keep (the keep bit, which blocks coarsening)
    from oracle import mlp
    from oracle.amr import Oracle
    from paper_2508_05020_gb300.amr import AMR
    w = workload('riemann2d', base_cells=(32, 32, 1), patch=8)
    r = Oracle(w)
    for _ in range(2):
        r.step()
        r.regrid()
    p = mlp_init(5, mlp.k_in(2))
    p['b3'][:] = b3
    wf = flat(p)
    q = mlp.unflatten(wf.astype(np.float64), mlp.k_in(2))
    r.flag_override = mlp.make_flagger(q, 1.4, keep_margin=keep)
    g = AMR(w, flagger='mlp', mlp_keep_margin=keep)
    g.set_mlp(wf)
    keys = r.mesh.canonical()
    g.set_state(np.array([k[0] for k in keys]), np.array([[k[1][0], k[1][1]] for k in keys]),
                np.stack([r.U[k][r.inner()].reshape((4, 8, 8)) for k in keys]), t=r.t)
    rg, cg = g.requests()
    rr, cr, af = r.requests()
    # margin per leaf patch: max logit over its in-domain band cells
    margin = {}
    for k in af:
        R, Us, P, cells = mlp.cell_stencils(r, k)
        z, _ = mlp.forward(q, mlp.features(R, Us, P, 1.4))
        ok = np.ones(len(z), dtype=bool)
        for d in range(2):
            gidx = k[1][d] * r.N + cells[:, d]
            ok &= (gidx >= 0) & (gidx < r.mesh.extent(k[0])[d] * r.N)
        margin[k] = float(np.max(z[ok]))
    sg = {(int(x[0]), (int(x[1]), int(x[2]), int(x[3]))) for x in rg}
    sr = set(rr)
    for k in sg ^ sr:
        assert abs(margin[k]) < 0.05, (k, margin[k])
    assert len(sg ^ sr) <= max(1, len(sr) // 20)
    cgs = {(int(x[0]), (int(x[1]), int(x[2]), int(x[3]))) for x in cg}
    crs = set(cr)
    assert crs, 'no coarsening candidates: the case does not test the keep bit'
    for k in cgs ^ crs:
        assert min(abs(margin[c] + keep) for c in r.mesh.children(k)) < 0.05, k
    assert len(cgs ^ crs) <= max(1, len(crs) // 20)
    counts = g.flag_stats()
    assert counts.sum() > 0
    g.close()


def oracle_cell_counts(r, wf, margin):
    """Per-cell agreement of the network with the plain sensor over the
    in-domain band cells [-1, N]^d of every leaf: (TP, FP, FN, TN), and the
    number of cells whose logit lies within `margin` of zero. The network is
    the oracle's, evaluated in FP64 on the BF16-rounded weights, features and
    hidden activations the tensor-core kernel uses."""
    from oracle import mlp
    dim = r.dim
    q = mlp.unflatten(wf.astype(np.float64), mlp.k_in(dim))
    r.fill_ghosts(r.U, r.t)
    offs = mlp.stencil_offsets(dim)
    c0 = offs.index((0, 0, 0))
    cnt = np.zeros(4, dtype=np.int64)
    near = 0
    for k in r.mesh.canonical():
        if not r.mesh.is_leaf(k):
            continue
        R, Us, P, cells = mlp.cell_stencils(r, k)
        X = mlp.features(R, Us, P, r.gamma)
        h1 = bf16(np.maximum(bf16(X) @ bf16(q['W1']).T + q['b1'], 0.0))
        z = np.maximum(h1 @ bf16(q['W2']).T + q['b2'], 0.0) @ q['W3'][0] + q['b3'][0]
        plain = np.zeros(len(z), dtype=bool)
        for phi, th in ((R, r.w['theta_rho']), (P, r.w['theta_p'])):
            for d in range(dim):
                e = [0, 0, 0]
                e[d] = 1
                ip, im = offs.index(tuple(e)), offs.index(tuple(-x for x in e))
                plain |= np.abs(phi[:, ip] - phi[:, im]) > th * (phi[:, ip] + 2.0 * phi[:, c0] + phi[:, im])
        ok = np.ones(len(z), dtype=bool)
        for d in range(dim):
            if r.periodic[d]:
                continue
            gi = k[1][d] * r.N + cells[:, d]
            ok &= (gi >= 0) & (gi < r.mesh.extent(k[0])[d] * r.N)
        m = z > 0.0
        cnt += [np.sum(ok & plain & m), np.sum(ok & ~plain & m), np.sum(ok & plain & ~m), np.sum(ok & ~plain & ~m)]
        near += int(np.sum(ok & (np.abs(z) < margin)))
    return cnt, near


@pytest.mark.parametrize('name,base,patch', [('sod', (64, 1, 1), 16), ('shu_osher', (64, 1, 1), 8),
                                             ('riemann2d', (32, 32, 1), 8), ('riemann2d', (32, 32, 1), 16),
                                             ('blast3d', (16, 16, 16), 8), ('blast3d', (16, 16, 16), 16)])
def test_fused_cell_counts_match_oracle(name, base, patch):
    # every band cell's learned decision (fused kernel: features in shared
    # memory, BF16 operands in tensor memory, row <-> cell maps of the
    # producer and epilogue roles) against the FP64 oracle network, cell by
    # cell through the agreement counts with the plain sensor; FP64 state so
    # that the plain flags coincide bit for bit
    import os
    from oracle.amr import Oracle
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name, base_cells=base, patch=patch, levels=2)
    dim = w['dim']
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    wf = np.load(os.path.join(here, 'paper_2508_05020_gb300', 'weights', 'indicator_d%d.npy' % dim)).astype(np.float32)
    r = Oracle(w)
    ref, near = oracle_cell_counts(r, wf, margin=0.02)
    assert ref[0] + ref[1] > 0 and ref[2] + ref[3] > 0
    g = AMR(w, precision=64, flagger='mlp', mlp_weights=wf)
    keys = r.mesh.canonical()
    shape = (w['dim'] + 2,) + (patch,) * dim
    g.set_state(np.array([k[0] for k in keys]), np.array([list(k[1][:dim]) for k in keys]),
                np.stack([r.U[k][r.inner()].reshape(shape) for k in keys]), t=r.t)
    got = g.flag_stats()
    g.close()
    # plain positives and negatives are the same cells on both sides
    assert got[0] + got[2] == ref[0] + ref[2] and got[1] + got[3] == ref[1] + ref[3], (got, ref)
    # learned decisions may differ only where the logit is within the rounding margin
    assert np.all(np.abs(got - ref) <= near), (got, ref, near)


def test_adam_steps_match_oracle():
    # full-batch training for two epochs = two Adam steps; against the
    # oracle's Adam on the oracle's FP64 gradients from the same start
    from oracle import mlp
    from paper_2508_05020_gb300 import amr
    s = samples(6, 128)
    dim = 1
    X = amr.mlp_features(dim, 1.4, s)
    y = np.repeat(mlp.plain_flag_1d(s, 0.05, 0.05), 2 * dim).astype(np.float32)
    pw = mlp.bce_pos_weight(y)
    w0 = flat(mlp_init(0, mlp.k_in(dim)))
    n, lr = X.shape[0], 1e-3
    p = mlp.unflatten(w0.astype(np.float64), mlp.k_in(dim))
    st = {}
    ref = []
    for _ in range(2):
        _, g = mlp.loss_and_grad(p, X.astype(np.float64), y.astype(np.float64), pw)
        if not ref:
            g1 = mlp.flatten(g)
        mlp.adam(p, g, st, lr)
        ref.append(mlp.flatten(p))
    w1, _ = amr.mlp_train(dim, X, y, pw, w0, epochs=1, batch=n, lr=lr, seed=1)
    step = w1.astype(np.float64) - w0.astype(np.float64)
    big = np.abs(g1) > 1e-3 * np.max(np.abs(g1))          # away from a sign change of the gradient
    assert np.all(np.abs(step) <= lr * (1.0 + 1e-3) + 1e-7)
    assert np.allclose(step[big], (ref[0] - w0)[big], rtol=0, atol=1e-3 * lr + 1e-7)
    w2, _ = amr.mlp_train(dim, X, y, pw, w0, epochs=2, batch=n, lr=lr, seed=1)
    assert np.allclose((w2 - w0)[big], (ref[1] - w0)[big], rtol=0, atol=0.1 * lr + 1e-7)
