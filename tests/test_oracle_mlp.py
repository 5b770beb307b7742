"""Pins of the oracle's refinement-indicator network (no GPU)."""
import numpy as np
import pytest

from oracle import mlp
from synth import mlp_init


def random_samples(rng, n):
    """1D 5-point samples (rho, u, p) with a mix of smooth data and jumps."""
    s = np.empty((n, 5, 3))
    base = rng.uniform(0.5, 2.0, size=(n, 1, 3))
    s[:] = base
    s[:, :, 1] = rng.normal(0, 0.5, size=(n, 5))
    jump = rng.uniform(size=n) < 0.5
    pos = rng.integers(1, 5, size=n)
    for i in np.nonzero(jump)[0]:
        s[i, pos[i]:, 0] *= rng.uniform(0.2, 3.0)
        s[i, pos[i]:, 2] *= rng.uniform(0.2, 3.0)
    s[:, :, 0] *= 1.0 + 0.01 * rng.normal(size=(n, 5))
    return s


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_gradient_matches_finite_differences(dim):
    rng = np.random.default_rng(0)
    smp = random_samples(rng, 16)
    X = mlp.embedded_features(smp, dim, 1.4)
    y = np.repeat(mlp.plain_flag_1d(smp, 0.05, 0.05), 2 * dim).astype(np.float64)
    params = mlp_init(0, mlp.k_in(dim))
    pw = mlp.bce_pos_weight(y)
    _, g = mlp.loss_and_grad(params, X, y, pw)
    gvec = mlp.flatten(g)
    idx, fd = mlp.gradient_fd(params, X, y, pw, h=1e-6, n_probe=40, seed=1)
    assert np.allclose(gvec[idx], fd, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_embedding_keeps_the_plain_flag(dim):
    # the plain sensor evaluated on the d-dimensional embedded stencil (centre
    # and its +-1 neighbours along every axis) equals the 1D flag: transverse
    # differences vanish
    rng = np.random.default_rng(1)
    smp = random_samples(rng, 200)
    f1 = mlp.plain_flag_1d(smp, 0.05, 0.05)
    offs = mlp.stencil_offsets(dim)
    centre = offs.index((0, 0, 0))
    for a in range(dim):
        for s in (-1, 1):
            rho, u, p = mlp.embed_1d(smp, dim, a, s)
            flag = np.zeros(len(smp), dtype=bool)
            for phi, th in ((rho, 0.05), (p, 0.05)):
                for d in range(dim):
                    e = [0, 0, 0]
                    e[d] = 1
                    ip = offs.index(tuple(e))
                    im = offs.index(tuple(-x for x in e))
                    fm, f0, fp = phi[:, im], phi[:, centre], phi[:, ip]
                    flag |= np.abs(fp - fm) > th * (fp + 2.0 * f0 + fm)
            assert np.array_equal(flag, f1)


def test_features_centre_normalisation():
    rng = np.random.default_rng(2)
    smp = random_samples(rng, 10)
    X = mlp.embedded_features(smp, 2, 1.4).reshape(10, 4, 25, 4)
    c0 = np.sqrt(1.4 * smp[:, 2, 2] / smp[:, 2, 0])
    # centre point (index 12): rho~ = 0, p~ = 0, u~ along the axis = +-u0 / c0
    assert np.allclose(X[:, :, 12, 0], 0.0, atol=1e-15)
    assert np.allclose(X[:, :, 12, 3], 0.0, atol=1e-15)
    assert np.allclose(X[:, 1, 12, 1], smp[:, 2, 1] / c0)
    assert np.allclose(X[:, 0, 12, 1], -smp[:, 2, 1] / c0)
    assert np.allclose(X[:, 3, 12, 2], smp[:, 2, 1] / c0)


def test_adam_training_reduces_loss():
    rng = np.random.default_rng(3)
    smp = random_samples(rng, 400)
    X = mlp.embedded_features(smp, 1, 1.4)
    y = np.repeat(mlp.plain_flag_1d(smp, 0.05, 0.05), 2).astype(np.float64)
    params = mlp_init(0, mlp.k_in(1))
    pw = mlp.bce_pos_weight(y)
    st = {}
    l0, _ = mlp.loss_and_grad(params, X, y, pw)
    for _ in range(200):
        _, g = mlp.loss_and_grad(params, X, y, pw)
        mlp.adam(params, g, st, 3e-3)
    l1, _ = mlp.loss_and_grad(params, X, y, pw)
    assert l1 < 0.5 * l0


def test_keep_margin_hysteresis():
    # refinement requests do not depend on the keep margin; coarsening
    # candidates shrink as it grows (a child keeps its parent refined while
    # any band logit is above -H), margin 0 is the single-threshold flagger,
    # and a margin above every logit leaves no candidate at all
    from oracle.amr import Oracle
    from synth import workload
    w = workload('riemann2d', base_cells=(16, 16, 1), patch=8, levels=2)
    r = Oracle(w)
    r.step()
    r.regrid()
    p = mlp_init(5, mlp.k_in(2))
    p['b3'][:] = -3.0
    q = mlp.unflatten(mlp.flatten(p), mlp.k_in(2))
    out = {}
    for H in (None, 0.0, 0.5, 2.0, 1e9):
        r.flag_override = mlp.make_flagger(q, 1.4) if H is None else mlp.make_flagger(q, 1.4, keep_margin=H)
        rr, cr, _ = r.requests()
        out[H] = (rr, set(cr))
    assert out[None][1], 'no coarsening candidates: the case does not test the keep bit'
    for H in (0.0, 0.5, 2.0, 1e9):
        assert out[H][0] == out[None][0]
    assert out[0.0][1] == out[None][1]
    assert out[2.0][1] <= out[0.5][1] <= out[0.0][1]
    assert out[2.0][1] < out[None][1]
    assert not out[1e9][1]


def test_refine_margin_widens_refinement():
    # refinement requests grow with the refine margin R (a leaf refines when
    # a band logit is above -R): nested sets, R = 0 the default flagger,
    # strictly more leaves refined at a wider margin, every leaf below the
    # finest level once R exceeds every logit's distance below 0; and a
    # network whose every logit is exactly -3 (zero weights, output bias -3)
    # refines nothing at R = 2.9 and every such leaf at R = 3.1
    from oracle.amr import Oracle
    from synth import workload
    w = workload('riemann2d', base_cells=(48, 48, 1), patch=8, levels=2)
    r = Oracle(w)
    r.step()
    r.regrid()
    below = {k for k in r.mesh.canonical() if r.mesh.is_leaf(k) and k[0] < r.L - 1}
    assert below, 'no leaf below the finest level: the case does not test refinement'
    p = mlp_init(5, mlp.k_in(2))
    p['b3'][:] = -3.0
    q = mlp.unflatten(mlp.flatten(p), mlp.k_in(2))

    def refined(flagger):
        r.flag_override = flagger
        rr, _, _ = r.requests()
        return set(rr)
    out = {R: refined(mlp.make_flagger(q, 1.4, keep_margin=1e9, refine_margin=R)) for R in (0.0, 2.0, 3.0, 1e9)}
    assert out[0.0] == refined(mlp.make_flagger(q, 1.4))
    assert out[0.0] <= out[2.0] <= out[3.0] <= out[1e9]
    assert out[3.0] > out[0.0]
    assert len(out[1e9]) == len(below)
    zero = {k: np.zeros_like(v) for k, v in q.items()}
    zero['b3'][:] = -3.0
    assert not refined(mlp.make_flagger(zero, 1.4, keep_margin=6.0, refine_margin=2.9))
    assert len(refined(mlp.make_flagger(zero, 1.4, keep_margin=6.0, refine_margin=3.1))) == len(below)


def test_adam_steps_from_the_definition():
    # with a constant gradient the bias-corrected moments are g and g^2 at
    # every step, so each update is -lr g / (|g| + eps); a zero gradient
    # leaves the parameter where it is
    rng = np.random.default_rng(4)
    p = mlp_init(0, mlp.k_in(1))
    g = {k: rng.normal(size=np.shape(v)) for k, v in p.items()}
    g['b3'][:] = 0.0
    st = {}
    lr = 1e-3
    for _ in range(3):
        before = {k: np.array(v, copy=True) for k, v in p.items()}
        mlp.adam(p, g, st, lr)
        for k in p:
            step = p[k] - before[k]
            assert np.allclose(step, -lr * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-9, atol=1e-15), k
    assert st['t'] == 3


def test_weighted_bce_closed_form():
    # all weights zero and output bias z: every logit is z, the loss is
    # mean(pw y log(1 + e^-z) + (1 - y) log(1 + e^z)), its b3 gradient is
    # mean(pw y (sigma(z) - 1) + (1 - y) sigma(z)), the other gradients vanish
    p = {k: np.zeros_like(v) for k, v in mlp_init(0, mlp.k_in(2)).items()}
    y = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0])
    pw = mlp.bce_pos_weight(y)
    assert pw == 2.0                                       # 4 negatives / 2 positives
    X = np.random.default_rng(5).normal(size=(6, mlp.k_in(2)))
    for z in (-3.0, 0.0, 0.7, 12.0):
        p['b3'][:] = z
        loss, g = mlp.loss_and_grad(p, X, y, pw)
        s = 1.0 / (1.0 + np.exp(-z))
        ref = np.mean(pw * y * np.log1p(np.exp(-z)) + (1.0 - y) * np.log1p(np.exp(z)))
        assert loss == pytest.approx(ref, rel=1e-12)
        assert g['b3'][0] == pytest.approx(np.mean(pw * y * (s - 1.0) + (1.0 - y) * s), rel=1e-12, abs=1e-15)
        for k in ('W1', 'b1', 'W2', 'b2', 'W3'):
            assert not np.any(g[k]), k
