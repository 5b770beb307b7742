"""amr_advance (the production loop) against the same steps and regrids
issued one call at a time."""
import numpy as np
import pytest

from synth import workload

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


@pytest.mark.parametrize('name,base,precision', [('riemann2d', (64, 64, 1), 64), ('shu_osher', (64, 1, 1), 32)])
def test_advance_equals_step_regrid(name, base, precision):
    from paper_2508_05020_gb300.amr import AMR, AMRError
    w = workload(name, base_cells=base)
    a = AMR(w, precision=precision)
    b = AMR(w, precision=precision)
    for _ in range(4):
        a.step()
        a.regrid()
    b.advance(4)
    assert a.diag()[0] == b.diag()[0]
    for l in range(a.L):
        ca, xa = a.get_level(l)
        cb, xb = b.get_level(l)
        assert np.array_equal(ca, cb) and np.array_equal(xa, xb)
    with pytest.raises(AMRError):
        b.advance(-1)
    a.close()
    b.close()


@pytest.mark.parametrize('name,base,precision,flagger,K', [('riemann2d', (64, 64, 1), 64, 'plain', 3),
                                                           ('blast3d', (32, 32, 32), 32, 'mlp', 4)])
def test_regrid_interval_equals_step_calls(name, base, precision, flagger, K):
    """amr_advance(n, K): a regrid after every K-th step, the count carried
    across calls and restarted by amr_regrid; the same as issuing the steps
    and regrids one call at a time, bit for bit."""
    import os
    from paper_2508_05020_gb300.amr import AMR, AMRError
    w = workload(name, base_cells=base)
    kw = {}
    if flagger == 'mlp':
        kw = dict(flagger='mlp', mlp_keep_margin=12.0,
                  mlp_weights=np.load(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                   'paper_2508_05020_gb300', 'weights',
                                                   'indicator_d%d_k4.npy' % w['dim'])).astype(np.float32))
    a = AMR(w, precision=precision, **kw)
    b = AMR(w, precision=precision, **kw)
    c = AMR(w, precision=precision, **kw)
    n = 3 * K + 2
    for i in range(n):
        a.step()
        if (i + 1) % K == 0:
            a.regrid()
    b.advance(n, regrid=K)
    for _ in range(n):                              # one step per call: the interval carries over
        c.advance(1, regrid=K)
    assert a.diag()[0] == b.diag()[0] == c.diag()[0]
    for l in range(a.L):
        ca, xa = a.get_level(l)
        for o in (b, c):
            co, xo = o.get_level(l)
            assert np.array_equal(ca, co) and np.array_equal(xa, xo)
    # amr_regrid restarts the count: K - 1 more steps take no regrid, the K-th does
    a.regrid()
    b.regrid()
    for i in range(K):
        a.step()
    a.regrid()
    b.advance(K - 1, regrid=K)
    b.advance(1, regrid=K)
    assert a.diag()[0] == b.diag()[0]
    for l in range(a.L):
        ca, xa = a.get_level(l)
        cb, xb = b.get_level(l)
        assert np.array_equal(ca, cb) and np.array_equal(xa, xb)
    with pytest.raises(AMRError):
        b.advance(1, regrid=-1)
    for o in (a, b, c):
        o.close()


@pytest.mark.parametrize('levels', [2, 3])
def test_step_timing_slots(levels):
    """amr_set_timing / amr_get_timing on the batched step: every class timed,
    the launch counts of the step's classes as issued (the finest level's
    restriction runs inside the RHS launch, so the restriction slot has the
    coarser levels only), and timing leaves the results unchanged."""
    from paper_2508_05020_gb300.amr import AMR
    w = workload('blast3d', base_cells=(32, 32, 32), levels=levels)
    a = AMR(w, precision=32)
    b = AMR(w, precision=32)
    a.set_timing(True)
    for _ in range(2):
        assert a.step() == b.step()
        a.regrid()
        b.regrid()
    a.advance(1, regrid=False)
    b.advance(1, regrid=False)
    ms, n = a.timing()
    slots = dict(zip(AMR.TIMING_SLOTS, range(len(AMR.TIMING_SLOTS))))
    assert ms[slots['rhs']] > 0 and ms[slots['ghost']] > 0 and ms[slots['cfl']] > 0
    assert n[slots['rhs']] == 3 and n[slots['reflux']] == 3
    assert n[slots['restrict']] == 3 * (levels - 2)
    assert ms[slots['restrict']] >= 0 and (levels == 2 or ms[slots['restrict']] > 0)
    for l in range(a.L):
        ca, xa = a.get_level(l)
        cb, xb = b.get_level(l)
        assert np.array_equal(ca, cb) and np.array_equal(xa, xb)
    a.close()
    b.close()
