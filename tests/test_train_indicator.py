"""Host-side data preparation of the indicator training
(paper_2508_05020_gb300/train_indicator.py) against the oracle: the planar
wave embedding of 1D windows gives the features of the sampled d-dimensional
wave, and the plain sensor flags such a wave exactly where the 1D sensor
flags the profile, so the windows' 1D labels hold in every direction (no GPU)."""
import numpy as np
import pytest

from oracle import mlp
from oracle.amr import G, Oracle
from synth import workload


@pytest.fixture(scope='module')
def ti():
    from paper_2508_05020_gb300 import train_indicator
    return train_indicator


def windows(rng, m, n):
    rho = rng.uniform(0.5, 2.0, (m, n))
    u = rng.uniform(-1.0, 1.0, (m, n))
    p = rng.uniform(0.2, 3.0, (m, n))
    return np.stack([rho, u, p], axis=2)


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_planar_embedding_gives_the_features_of_the_sampled_wave(ti, dim):
    # stencil point o of a wave along the integer direction n reads the window
    # at o . n and carries the velocity u n / |n|; the features are then the
    # oracle's centre-normalised features of that stencil
    rng = np.random.default_rng(4 + dim)
    m = 12
    prof = windows(rng, m, ti.PROFILE)
    h = ti.PROFILE // 2
    offs = mlp.stencil_offsets(dim)
    dirs = ti.directions(dim)
    assert len(dirs) == 3 ** dim - 1
    for n in dirs:
        X = ti.embedded_features(prof, dim, np.repeat(n[None, :], m, axis=0), 1.4)
        idx = np.array([h + sum(o[d] * n[d] for d in range(dim)) for o in offs])
        rho, un, p = prof[:, idx, 0], prof[:, idx, 1], prof[:, idx, 2]
        norm = np.sqrt(float(np.dot(n, n)))
        ref = mlp.features(rho, [un * (n[d] / norm) for d in range(dim)], p, 1.4)
        assert X.shape == (m, mlp.k_in(dim))
        assert np.allclose(X, ref, rtol=1e-13, atol=1e-13), n


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_axis_embedding_matches_the_five_point_embedding(ti, dim):
    # along an axis the wave embedding of a window is the embedding of its
    # centre 5 points that the fused kernel's training rows use
    rng = np.random.default_rng(9)
    m = 10
    prof = windows(rng, m, ti.PROFILE)
    h = ti.PROFILE // 2
    for a in range(dim):
        for s in (-1, 1):
            n = np.zeros(dim, dtype=int)
            n[a] = s
            X = ti.embedded_features(prof, dim, np.repeat(n[None, :], m, axis=0), 1.4)
            ref = mlp.features(*mlp.embed_1d(prof[:, h - 2:h + 3, :], dim, a, s), 1.4)
            assert np.allclose(X, ref, rtol=1e-13, atol=1e-13), (a, s)


@pytest.mark.parametrize('dim', [2, 3])
def test_plain_sensor_flags_a_planar_wave_like_its_profile(ti, dim):
    # a periodic 1D profile with a few jumps laid along every direction of the
    # training set on a periodic box: the oracle's sensor flags cell c exactly
    # when the 1D sensor flags the profile at c . n
    n_cells = 16 if dim == 2 else 8
    rng = np.random.default_rng(21)
    P = n_cells
    x = np.arange(P)
    rho = 1.0 + 0.02 * np.sin(2 * np.pi * x / P) + np.where((x >= 3) & (x < 9), 0.8, 0.0)
    p = 1.0 + 0.01 * rng.uniform(size=P) + np.where(x >= 11, 1.5, 0.0)
    u = 0.1 * np.cos(2 * np.pi * x / P)
    th = 0.05
    flag1 = np.zeros(P, dtype=bool)
    for f in (rho, p):
        fm, fp = np.roll(f, 1), np.roll(f, -1)
        flag1 |= np.abs(fp - fm) > th * (fp + 2.0 * f + fm)
    assert 0 < flag1.sum() < P
    base = tuple(n_cells if d < dim else 1 for d in range(3))
    w = workload('constant', dim=dim, base_cells=base, patch=8, levels=1,
                 bc=(('periodic', 'periodic'),) * 3, theta_rho=th, theta_p=th)
    for n in ti.directions(dim):
        o = Oracle(w)
        norm = np.sqrt(float(np.dot(n, n)))
        grids = np.meshgrid(*[np.arange(base[d]) for d in (2, 1, 0)][3 - dim:], indexing='ij')
        gi = {d: grids[dim - 1 - d] for d in range(dim)}                 # global index along dimension d
        k = sum(gi[d] * n[d] for d in range(dim)) % P
        E = p[k] / 0.4 + 0.5 * rho[k] * u[k] ** 2
        for key in o.mesh.canonical():
            sl = tuple(slice(key[1][d] * 8, key[1][d] * 8 + 8) for d in reversed(range(dim)))
            A = o.U[key]
            inner = A[o.inner()]
            inner[0] = rho[k][sl].reshape(inner[0].shape)
            for d in range(dim):
                inner[1 + d] = (rho[k] * u[k] * (n[d] / norm))[sl].reshape(inner[0].shape)
            inner[dim + 1] = E[sl].reshape(inner[0].shape)
            A[o.inner()] = inner
        o.fill_ghosts(o.U, 0.0)
        for key in o.mesh.canonical():
            f = o.patch_flags(key)
            core = tuple([slice(None)] * (3 - dim) + [slice(2, 10)] * dim)
            sl = tuple(slice(key[1][d] * 8, key[1][d] * 8 + 8) for d in reversed(range(dim)))
            assert np.array_equal(f[core].reshape(k[sl].shape), flag1[k[sl]]), (n, key)


def test_evaluation_weight_specs():
    from paper_2508_05020_gb300 import eval_indicator as ev
    specs = ev.parse_weights(['net=paper_2508_05020_gb300/weights/indicator_d{d}.npy',
                              'lookahead=paper_2508_05020_gb300/weights/indicator_d{d}_k4.npy'])
    assert [s[0] for s in specs] == ['net', 'lookahead']
    for dim in (1, 2, 3):
        for _, p in specs:
            w = ev.load_weights(p, dim)
            assert w is not None and w.dtype == np.float32 and w.size == 64 * mlp.k_in(dim) + 64 * 64 + 3 * 64 + 1
    assert ev.load_weights('paper_2508_05020_gb300/weights/none_d{d}.npy', 1) is None
    for bad in ('net', '=x_d{d}.npy', 'net=indicator.npy'):
        with pytest.raises(ValueError):
            ev.parse_weights([bad])
