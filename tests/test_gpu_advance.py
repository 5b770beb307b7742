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

