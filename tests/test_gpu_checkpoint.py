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
