"""The lookahead indicator (trained to predict the plain flag within the next
4 steps, train_indicator --lookahead 4) against the plain sensor when the
hierarchy is regridded only every 4 steps: on the shock tube it leaves fewer
of the plain sensor's refinement requests unmet along the run, at nearly the
same number of patches."""
import os

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def state(a):
    lv, co, da = [], [], []
    for l in range(a.L):
        c, x = a.get_level(l)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c)
        da.append(x)
    return np.concatenate(lv), np.concatenate(co), np.concatenate(da)


def unmet(w, flagger, weights, every, steps):
    """Mean number of patches per step that the plain sensor would refine on
    the run's current hierarchy (before its scheduled regrid), and the mean
    patch count."""
    from paper_2508_05020_gb300.amr import AMR
    a = AMR(w, precision=64, flagger=flagger, mlp_weights=weights)
    plain_ref = AMR(w, precision=64, flagger='plain')
    miss, patches = [], []
    for i in range(steps):
        a.step()
        lv, co, da = state(a)
        plain_ref.set_state(lv, co, da, t=a.diag()[0])
        r, _ = plain_ref.requests()
        miss.append(len(r))
        patches.append(int(sum(a.diag()[2])))
        if (i + 1) % every == 0:
            a.regrid()
    a.close()
    plain_ref.close()
    return float(np.mean(miss)), float(np.mean(patches))


def test_lookahead_indicator_keeps_refinement_ahead_of_the_shock():
    w = workload('sod')
    wk = np.load(os.path.join(HERE, 'paper_2508_05020_gb300', 'weights', 'indicator_d1_k4.npy')).astype(np.float32)
    plain_miss, plain_patches = unmet(w, 'plain', None, 4, 80)
    la_miss, la_patches = unmet(w, 'mlp', wk, 4, 80)
    assert plain_miss > 0.2
    assert la_miss < 0.5 * plain_miss, (la_miss, plain_miss)
    assert la_patches <= 1.2 * plain_patches, (la_patches, plain_patches)
