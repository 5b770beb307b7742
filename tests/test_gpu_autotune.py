"""The launch-parameter autotuner (amr_autotune): it changes how the batched
step is launched, never what it computes."""
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


def snapshot(a):
    out = []
    for l in range(a.L):
        c, x = a.get_level(l)
        out.append((c.copy(), x.copy()))
    return out, a.diag()


@pytest.mark.parametrize('name,base,precision', [('riemann2d', (64, 64, 1), 64), ('blast3d', (32, 32, 32), 32),
                                                 ('dmr', (128, 32, 1), 64)])
def test_autotune_leaves_results_unchanged(name, base, precision):
    from paper_2508_05020_gb300.amr import AMR, TUNE_NAMES
    w = workload(name, base_cells=base)
    a = AMR(w, precision=precision)
    b = AMR(w, precision=precision, autotune=True)
    pa, ta = a.tuning()
    pb, tb = b.tuning()
    # defaults before tuning; candidates of the tuner after it, each with a measured time
    assert pa == {'ghost_ctas_per_sm': 16, 'ghost_cells_per_item': 128, 'rhs_ctas_per_sm': 2,
                  'reflux_ctas_per_sm': 4, 'restrict_ctas_per_sm': 8, 'cfl_ctas_per_sm': 8, 'flag_ctas_per_sm': 4,
                  'rhs_tile_shape': 0}
    assert pb['ghost_ctas_per_sm'] in (4, 8, 16, 32) and pb['ghost_cells_per_item'] in (64, 128, 256, 512, 1024)
    assert pb['rhs_ctas_per_sm'] in (1, 2, 3, 4, 6, 8, 12, 16)
    assert pb['rhs_tile_shape'] in ((0, 1, 2, 3, 4) if (w['dim'], w['patch'], precision) == (3, 16, 32) else (0,))
    assert all(tb[k] > 0 for k in TUNE_NAMES)
    # tuning again leaves the state, time and dt untouched
    s0, d0 = snapshot(b)
    b.autotune()
    s1, d1 = snapshot(b)
    for (c0, x0), (c1, x1) in zip(s0, s1):
        assert np.array_equal(c0, c1) and np.array_equal(x0, x1)
    assert d0[0] == d1[0] and np.array_equal(d0[1], d1[1])
    # and the run is bit-identical with and without tuned launches
    for _ in range(3):
        assert a.step() == b.step()
        a.regrid()
        b.regrid()
    sa, da = snapshot(a)
    sb, db = snapshot(b)
    for (ca, xa), (cb, xb) in zip(sa, sb):
        assert np.array_equal(ca, cb) and np.array_equal(xa, xb)
    assert da[0] == db[0]
    a.close()
    b.close()


def test_every_rhs_tile_shape_gives_the_same_bits():
    """The fused RHS's tile-shape candidates of FP32 3D 16^3 patches (four-,
    two- and eight-plane z chunks; four- and eight-plane chunks with the halo
    planes copied by TMA) and other grids, set by amr_set_tuning: the same
    results bit for bit; parameters out of range are refused."""
    from paper_2508_05020_gb300.amr import AMR, AMRError
    w = workload('blast3d', base_cells=(32, 32, 32))
    runs = []
    for shape, grid in ((0, 2), (1, 3), (2, 1), (1, 1), (3, 2), (4, 1), (3, 12)):
        a = AMR(w, precision=32)
        a.set_tuning({'rhs_tile_shape': shape, 'rhs_ctas_per_sm': grid})
        assert a.tuning()[0]['rhs_tile_shape'] == shape
        for _ in range(3):
            a.step()
            a.regrid()
        runs.append(snapshot(a))
        if shape == 0:
            for bad in ({'rhs_tile_shape': 5}, {'rhs_tile_shape': -1}, {'ghost_cells_per_item': 16},
                        {'cfl_ctas_per_sm': 0}):
                with pytest.raises(AMRError):
                    a.set_tuning(bad)
            assert a.tuning()[0]['rhs_tile_shape'] == 0
        a.close()
    s0, d0 = runs[0]
    for s1, d1 in runs[1:]:
        for (c0, x0), (c1, x1) in zip(s0, s1):
            assert np.array_equal(c0, c1) and np.array_equal(x0, x1)
        assert d0[0] == d1[0]
    # FP64 and 2D grids compile one shape
    b = AMR(workload('riemann2d', base_cells=(64, 64, 1)), precision=64)
    with pytest.raises(AMRError):
        b.set_tuning({'rhs_tile_shape': 1})
    b.close()
