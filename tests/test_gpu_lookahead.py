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


def _level0_rho(a):
    coords, x = a.get_level(0)
    d, N = a.dim, a.N
    ext = [int(coords[:, k].max()) + 1 if k < d else 1 for k in range(3)]
    out = np.zeros(tuple(ext[k] * (N if k < d else 1) for k in (2, 1, 0)))
    for c, patch in zip(coords, x[:, 0]):
        sl = tuple(slice(int(c[k]) * N, int(c[k]) * N + N) if k < d else slice(None) for k in (2, 1, 0))
        out[sl] = patch.reshape(out[sl].shape)
    return out


def test_learned_lookahead_mesh_is_closer_to_the_fully_refined_solution():
    """What the trained network gains over the plain method on the 3D blast
    (32^3 base, 3 levels) run to t_end: every run replays the dt sequence of
    the FP32 plain run regridding every step, and the density on level 0 is
    compared with that of the same problem with every cell refined to the
    finest level (the uniform grid at the finest spacing, averaged to level 0,
    which every AMR mesh approximates). Regridding every 4 steps with the
    lookahead network leaves level 0 closer to it than the plain sensor
    regridding every step (measured: relative L1 2.50e-4 against 2.76e-4 with
    FP64 reference runs), with fewer of the plain sensor's requests unmet."""
    from paper_2508_05020_gb300.amr import AMR
    w = workload('blast3d', base_cells=(32, 32, 32))
    wts = np.load(os.path.join(HERE, 'paper_2508_05020_gb300', 'weights',
                               'indicator_d3_diag_k4.npy')).astype(np.float32)
    plain = AMR(w, precision=32, flagger='plain')
    dts, unmet_plain = [], []
    while True:
        dt = plain.step(sync=True)
        if not dt > 0:
            break
        dts.append(dt)
        plain.regrid()
        if len(dts) % 25 == 0:
            unmet_plain.append(plain.plain_requests())
    rho_plain = _level0_rho(plain)
    plain.close()
    assert len(dts) > 300                                     # the run reached t_end
    fine = AMR(dict(w, theta_rho=-1.0, theta_p=-1.0), precision=32, flagger='plain')
    n_all = int(sum(fine.diag()[2]))
    for dt in dts:
        fine.step(dt=dt, sync=False)
    assert int(sum(fine.diag()[2])) == n_all == 8 + 64 + 512    # every level fully refined throughout
    rho_fine = _level0_rho(fine)
    fine.close()
    learned = AMR(w, precision=32, flagger='mlp', mlp_weights=wts, mlp_keep_margin=12.0)
    unmet_learned = []
    for i, dt in enumerate(dts):
        learned.step(dt=dt, sync=False)
        if (i + 1) % 4 == 0:
            learned.regrid()
        if (i + 1) % 25 == 0:
            unmet_learned.append(learned.plain_requests())
    rho_learned = _level0_rho(learned)
    learned.close()

    def l1(a, b):
        return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))
    e_plain, e_learned = l1(rho_plain, rho_fine), l1(rho_learned, rho_fine)
    print('L1 vs fully refined: plain every step %.3e, lookahead every 4 steps %.3e; unmet %.2f / %.2f'
          % (e_plain, e_learned, np.mean(unmet_plain), np.mean(unmet_learned)))
    assert e_learned < e_plain
    assert np.mean(unmet_learned) <= np.mean(unmet_plain)
