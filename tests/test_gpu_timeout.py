"""The timeout path of the learned-flag kernel's tensor-core pipeline.

A test hook (not part of the public header) shortens the limit of the
pipeline's role waits to about half a millisecond and makes the MMA thread
withhold the epilogue's accumulator signal, so that a wait cannot complete:
no GPU fault, hang or trap is involved. The kernel must set its abort word,
let every role reach the tear-down, wait for its in-flight MMAs, free its
tensor memory and report the timeout, which reaches the host as
AMR_ERR_TIMEOUT; the context then refuses work, can be destroyed, and a fresh
context on the same device runs as one that never saw the timeout."""
import ctypes as C
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


def _run(precision, weights, hook=None):
    from paper_2508_05020_gb300.amr import AMR
    w = workload('blast3d', base_cells=(16, 16, 16), patch=8, levels=2)
    a = AMR(w, precision=precision, flagger='mlp', mlp_weights=weights, mlp_keep_margin=12.0)
    if hook:
        hook(a)
    return a


@pytest.mark.parametrize('precision', [32, 64])
def test_role_wait_timeout_reports_and_leaves_the_device_usable(precision):
    from paper_2508_05020_gb300.amr import AMRError
    weights = np.load(os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights', 'indicator_d3.npy')).astype(np.float32)
    ref = _run(precision, weights)
    ref.step()
    ref.regrid()
    ref_keys = ref.patch_keys()
    ref_state = [ref.get_level(l)[1] for l in range(ref.L)]
    ref.close()

    def hook(a):
        lib = a.lib
        f = lib.amr_test_tc_wait
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_longlong, C.c_int]
        assert f(a.ctx, 0, 1) == -1                            # AMR_ERR_ARG: the limit must be positive
        assert f(a.ctx, 1 << 20, 1) == 0                       # about half a millisecond

    bad = _run(precision, weights, hook)
    bad.step()
    with pytest.raises(AMRError) as e:
        bad.regrid()
    assert e.value.code == -5, e.value                         # AMR_ERR_TIMEOUT
    with pytest.raises(AMRError) as e:
        bad.step()
    assert e.value.code == -6                                  # AMR_ERR_STATE: the context refuses work
    bad.close()
    # a fresh context runs as if nothing had happened, bit for bit
    again = _run(precision, weights)
    again.step()
    again.regrid()
    assert again.patch_keys() == ref_keys
    for l in range(again.L):
        assert np.array_equal(again.get_level(l)[1], ref_state[l])
    again.close()


def test_shortened_limit_without_withholding_completes():
    """The shortened limit alone on a pipeline whose signals all arrive: the
    waits that complete are not affected by the hook's limit unless they run
    longer, so the regrid either succeeds with the flags of a normal run or
    reports the timeout; it never returns wrong flags silently."""
    from paper_2508_05020_gb300.amr import AMRError
    weights = np.load(os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights', 'indicator_d3.npy')).astype(np.float32)
    ref = _run(32, weights)
    ref.step()
    ref.regrid()
    ref_keys = ref.patch_keys()
    ref.close()

    def hook(a):
        f = a.lib.amr_test_tc_wait
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.c_longlong, C.c_int]
        assert f(a.ctx, 1 << 30, 0) == 0

    a = _run(32, weights, hook)
    a.step()
    try:
        a.regrid()
        assert a.patch_keys() == ref_keys
    except AMRError as e:
        assert e.code == -5
    a.close()
