"""amr_plain_requests: the plain sensor's refinement requests on the current
hierarchy of a context that regrids with the learned indicator or every K
steps (the unmet requests of that choice)."""
import os

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def _weights(d):
    return np.load(os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights', 'indicator_d%d_k4.npy' % d)).astype(np.float32)


def _state(a):
    lv, co, da = [], [], []
    for l in range(a.L):
        c, x = a.get_level(l)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c)
        da.append(x)
    return np.concatenate(lv), np.concatenate(co), np.concatenate(da)


@pytest.mark.parametrize('name,base,precision,flagger,K', [('riemann2d', (64, 64, 1), 64, 'plain', 4),
                                                           ('riemann2d', (64, 64, 1), 64, 'mlp', 3),
                                                           ('blast3d', (32, 32, 32), 32, 'mlp', 3)])
def test_plain_requests_equal_a_plain_context_on_the_same_state(name, base, precision, flagger, K):
    """The count equals the refinement requests of a plain-sensor context
    holding the same hierarchy and state, and calling it changes nothing: the
    run continues bit for bit as one without the calls. With the plain sensor
    regridding every 4 steps the fronts move ahead of the mesh between
    regrids, so some requests go unmet."""
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name, base_cells=base)
    kw = dict(flagger='mlp', mlp_weights=_weights(w['dim']), mlp_keep_margin=12.0) if flagger == 'mlp' else {}
    a = AMR(w, precision=precision, **kw)
    b = AMR(w, precision=precision, **kw)
    plain = AMR(w, precision=precision, flagger='plain')
    counts = []
    for i in range(8):
        a.advance(1, regrid=K)
        b.advance(1, regrid=K)
        n = a.plain_requests()
        lv, co, da = _state(a)
        plain.set_state(lv, co, da, t=a.diag()[0])
        r, _ = plain.requests()
        assert n == len(r), (i, n, len(r))
        counts.append(n)
    assert a.diag()[0] == b.diag()[0]
    for l in range(a.L):
        ca, xa = a.get_level(l)
        cb, xb = b.get_level(l)
        assert np.array_equal(ca, cb) and np.array_equal(xa, xb)
    for o in (a, b, plain):
        o.close()


def test_a_network_that_never_flags_leaves_every_plain_request_unmet():
    """A learned indicator whose logit is -1 everywhere (zero weights, output
    bias -1) never refines, so the hierarchy stays at level 0 and every patch
    the plain sensor would refine is counted: the four-quadrant problem's
    discontinuities cross level-0 patches."""
    from paper_2508_05020_gb300.amr import AMR, mlp_k
    w = workload('riemann2d', base_cells=(64, 64, 1))
    K = mlp_k(2)
    wts = np.zeros(64 * K + 64 + 64 * 64 + 64 + 64 + 1, dtype=np.float32)
    wts[-1] = -1.0
    a = AMR(w, precision=64, flagger='mlp', mlp_weights=wts)
    assert list(a.diag()[2][1:]) == [0] * (a.L - 1)
    n = a.plain_requests()
    plain = AMR(w, precision=64, flagger='plain')
    lv, co, da = _state(a)
    plain.set_state(lv, co, da, t=0.0)
    r, _ = plain.requests()
    assert n == len(r) > 0
    a.close()
    plain.close()


def test_plain_requests_single_level_and_plain_context():
    from paper_2508_05020_gb300.amr import AMR
    one = AMR(workload('sod', levels=1), precision=64)
    assert one.plain_requests() == 0
    one.close()
    p = AMR(workload('sod'), precision=64)
    p.step()
    r, _ = p.requests()
    assert p.plain_requests() == len(r)
    p.close()


def test_refine_margin_refines_at_least_as_much():
    """The learned flags' refine margin R (refine where a band logit is above
    -R): the learned cells found per band cell (true and false positives
    against the plain sensor) and the patches after a regrid do not shrink as
    R grows, and R = H refines every leaf whose keep bit is set."""
    from paper_2508_05020_gb300.amr import AMR
    w = workload('blast3d', base_cells=(32, 32, 32))
    out = []
    for R in (0.0, 2.0, 12.0):
        a = AMR(w, precision=32, flagger='mlp', mlp_weights=_weights(3), mlp_keep_margin=12.0, mlp_refine_margin=R)
        c = a.flag_stats()
        n = int(sum(a.diag()[2]))
        out.append((int(c[0] + c[1]), n))
        a.close()
    assert out[0][0] <= out[1][0] <= out[2][0]
    assert out[0][1] <= out[1][1] <= out[2][1]
    assert out[2][0] > out[0][0]
