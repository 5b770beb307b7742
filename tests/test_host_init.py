"""amr_init's argument checks through the C ABI, which run on the host before
any CUDA call (no GPU needed), and, on a machine without a GPU, the loud
failure of a valid call: there is no CPU fallback."""
import ctypes as C

import numpy as np
import pytest

from synth import workload


@pytest.fixture(scope='module')
def amr():
    from paper_2508_05020_gb300 import build
    build.build()
    from paper_2508_05020_gb300 import amr
    return amr


def init(amr, w, levels=None, ratio=2, patch=None, ic=None, gamma=None, **opt):
    """amr_init with host memory options (no PyTorch stream); returns (rc, message)."""
    lib = amr.load()
    o, keep = amr.make_options(torch_memory=False, cfl=w['cfl'], t_end=w['t_end'],
                               **{k: v for k, v in opt.items() if k in ('precision', 'flagger', 'max_patches', 'mode',
                                                                       'flux', 'mlp_keep_margin', 'theta_switch',
                                                                       'mlp_refine_margin')})
    for k in ('raw_flagger', 'raw_mode', 'raw_precision', 'raw_flux', 'raw_cfl'):
        if k in opt:
            setattr(o, k[4:], opt[k])
    dom = amr.Domain()
    dom.dim = opt.get('dim', w['dim'])
    for d in range(3):
        dom.lo[d] = w['lo'][d]
        dom.hi[d] = opt.get('hi', w['hi'])[d]
        bc = opt.get('bc', w['bc'])[d]
        dom.bc_lo[d] = bc[0] if isinstance(bc[0], int) else amr.BC[bc[0]]
        dom.bc_hi[d] = bc[1] if isinstance(bc[1], int) else amr.BC[bc[1]]
    base = (C.c_int * 3)(*opt.get('base_cells', w['base_cells']))
    ctx = C.c_void_p()
    rc = lib.amr_init(C.byref(ctx), C.byref(dom), w['gamma'] if gamma is None else gamma, base,
                      w['levels'] if levels is None else levels, ratio, w['patch'] if patch is None else patch,
                      amr.IC[w['ic']] if ic is None else ic, C.byref(o))
    msg = lib.amr_last_error(ctx).decode() if ctx else ''
    if ctx:
        lib.amr_destroy(ctx)
    return rc, msg


def test_invalid_arguments_are_refused_before_any_device_call(amr):
    w2 = workload('riemann2d', base_cells=(32, 32, 1), patch=8)
    w1 = workload('sod')
    w3 = workload('blast3d', base_cells=(16, 16, 16), patch=8, levels=2)
    cases = [
        (w2, dict(dim=0), 'dim'),
        (w2, dict(dim=4), 'dim'),
        (w2, dict(ratio=3), 'ratio'),
        (w2, dict(patch=12), 'patch size'),
        (w3, dict(patch=32, base_cells=(32, 32, 32)), 'patch size'),
        (w2, dict(levels=0), 'levels'),
        (w2, dict(levels=9), 'levels'),
        (w2, dict(gamma=1.0), 'gamma'),
        (w2, dict(raw_precision=16), 'precision'),
        (w2, dict(ic=99), 'initial condition'),
        (w2, dict(raw_cfl=0.0), 'cfl'),
        (w2, dict(raw_flagger=7), 'flagger'),
        (w2, dict(raw_mode=5), 'mode'),
        (w2, dict(base_cells=(36, 32, 1)), 'multiples'),
        (w2, dict(base_cells=(4, 32, 1)), 'multiples'),
        (w2, dict(hi=(0.0, 1.0, 1.0)), 'empty domain'),
        (w2, dict(bc=((9, 0), (0, 0), (0, 0))), 'boundary kind'),
        (w2, dict(bc=(('periodic', 'outflow'), ('outflow', 'outflow'), ('outflow', 'outflow'))), 'periodic'),
        (w3, dict(bc=(('dmr_inflow', 'outflow'),) * 3), 'double-Mach'),
        (w2, dict(max_patches=8), 'pool smaller'),
        # the 20-bit key fields and the 31-bit pool size
        (w1, dict(base_cells=(1 << 17, 1, 1), levels=8), '2^20'),
        (w3, dict(base_cells=(8192, 8192, 8192), levels=2), '2^31'),
    ]
    for w, kw, word in cases:
        rc, msg = init(amr, w, **kw)
        assert rc == -1 and word in msg, (kw, rc, msg)


def test_options_out_of_range_are_refused(amr):
    w = workload('sod')
    for kw, word in ((dict(raw_flux=4), 'flux'), (dict(mlp_keep_margin=-1.0), 'margin'),
                     (dict(theta_switch=float('nan')), 'theta_switch'),
                     (dict(mlp_keep_margin=2.0, mlp_refine_margin=3.0), 'mlp_refine_margin'),
                     (dict(mlp_refine_margin=-1.0), 'mlp_refine_margin')):
        rc, msg = init(amr, w, **kw)
        assert rc == -1 and word in msg, (kw, rc, msg)


def test_no_cpu_fallback_without_a_gpu(amr):
    torch = pytest.importorskip('torch')
    if torch.cuda.is_available():
        pytest.skip('a CUDA device is present')
    rc, msg = init(amr, workload('riemann2d', base_cells=(32, 32, 1), patch=8))
    assert rc == -3 and 'CUDA' in msg, (rc, msg)
    # the standalone network calls need the device too (NULL options: cudaMalloc, legacy stream)
    X = np.zeros((4, amr.mlp_k(1)), dtype=np.float32)
    w = np.zeros(64 * amr.mlp_k(1) + 64 + 64 * 64 + 64 + 64 + 1, dtype=np.float32)
    z = np.zeros(4, dtype=np.float32)
    rc = amr.load().amr_mlp_infer(1, amr._ptr(X), 4, amr._ptr(w), amr._ptr(z), None)
    assert rc == -3, rc
