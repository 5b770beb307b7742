"""Checkpoint and restart through the C ABI (amr_checkpoint, amr_restore): a
run continued from a checkpoint repeats the original run bit for bit; files
that do not match are refused with AMR_ERR_IO and leave the context usable."""
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


def state(g, L):
    return [g.get_level(l) for l in range(L)]


def same(a, b):
    for (ca, xa), (cb, xb) in zip(a, b):
        if not (np.array_equal(ca, cb) and np.array_equal(xa, xb)):
            return False
    return True


@pytest.mark.parametrize('name,kw,precision,flagger', [
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8), 64, 'plain'),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2), 32, 'plain'),
    ('dmr', dict(base_cells=(64, 16, 1), patch=8, levels=3), 32, 'plain'),
])
def test_restart_repeats_the_run(tmp_path, name, kw, precision, flagger):
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name, **kw)
    path = str(tmp_path / 'run.ckpt')
    a = AMR(w, precision=precision, flagger=flagger)
    a.advance(3)
    a.checkpoint(path)
    t_ck = a.diag()[0]
    s_ck = state(a, w['levels'])
    a.advance(3)
    s_a = state(a, w['levels'])
    t_a = a.diag()[0]
    b = AMR(w, precision=precision, flagger=flagger)
    b.restore(path)
    assert b.diag()[0] == t_ck
    assert same(state(b, w['levels']), s_ck)
    b.advance(3)
    assert b.diag()[0] == t_a
    assert same(state(b, w['levels']), s_a)
    a.close()
    b.close()


def test_fp64_checkpoint_into_fp32_context(tmp_path):
    from paper_2508_05020_gb300.amr import AMR
    w = workload('riemann2d', base_cells=(32, 32, 1), patch=8)
    path = str(tmp_path / 'fp64.ckpt')
    a = AMR(w, precision=64)
    a.advance(2)
    a.checkpoint(path)
    b = AMR(w, precision=32)
    b.restore(path)
    for (ca, xa), (cb, xb) in zip(state(a, w['levels']), state(b, w['levels'])):
        assert np.array_equal(ca, cb)
        assert np.array_equal(xb, xa.astype(np.float32).astype(np.float64))
    b.advance(1)
    a.close()
    b.close()


def test_mismatched_or_missing_files_are_refused(tmp_path):
    from paper_2508_05020_gb300.amr import AMR, AMRError
    w2 = workload('riemann2d', base_cells=(32, 32, 1), patch=8)
    w1 = workload('sod')
    p2 = str(tmp_path / 'two.ckpt')
    a = AMR(w2, precision=64)
    a.checkpoint(p2)
    b = AMR(w1, precision=64)
    before = state(b, w1['levels'])
    for path in (p2, str(tmp_path / 'missing.ckpt')):
        with pytest.raises(AMRError) as e:
            b.restore(path)
        assert e.value.code == -8
    short = str(tmp_path / 'short.ckpt')
    with open(p2, 'rb') as f:
        blob = f.read()
    with open(short, 'wb') as f:
        f.write(blob[:len(blob) // 2])
    c = AMR(w2, precision=64)
    with pytest.raises(AMRError) as e:
        c.restore(short)
    assert e.value.code == -8
    assert same(state(b, w1['levels']), before)
    b.advance(2)                                   # still usable
    c.advance(1)
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize('name,kw,precision', [
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8), 64),
    ('blast3d', dict(base_cells=(32, 32, 32), levels=3), 32),
    ('sod', dict(), 64),
])
def test_pinned_host_buffers_are_used_in_place(name, kw, precision):
    """amr_get_level and amr_set_state with page-locked host buffers (read and
    written by the device in one kernel) give the same bits as with pageable
    buffers (copied through the staging buffer), and a context loaded from
    either continues identically."""
    import torch
    from paper_2508_05020_gb300.amr import AMR
    w = workload(name, **kw)
    a = AMR(w, precision=precision)
    for _ in range(3):
        a.step()
        a.regrid()
    t = a.diag()[0]
    lv, co, pageable, pinned = [], [], [], []
    for l in range(a.L):
        c, x = a.get_level(l)                                   # pageable numpy buffer
        buf = torch.empty(x.shape, dtype=torch.float64, pin_memory=True).numpy()
        buf[...] = -1.0
        c2, _ = a.get_level(l, out=buf)                         # page-locked: written in place
        assert np.array_equal(c, c2) and np.array_equal(x, buf)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c.astype(np.int32))
        pageable.append(x)
        pinned.append(buf)
    lv, co = np.concatenate(lv), np.concatenate(co)
    dp = np.concatenate(pageable)
    dq = torch.empty(dp.shape, dtype=torch.float64, pin_memory=True).numpy()
    dq[...] = dp
    b = AMR(w, precision=precision)
    c_ = AMR(w, precision=precision)
    b.set_state(lv, co, dp, t=t)                                # staged
    c_.set_state(lv, co, dq, t=t)                               # read in place
    assert same(state(b, b.L), state(c_, c_.L))
    for _ in range(2):
        assert b.step() == c_.step()
        b.regrid()
        c_.regrid()
    assert same(state(b, b.L), state(c_, c_.L))
    for g in (a, b, c_):
        g.close()
