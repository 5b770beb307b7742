"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 bar: identical canonical patch lists and every conserved variable within
1e-9 relative max-norm (relative to the variable's max magnitude on that
level) after a run with a regrid after every step. FP32 bar: L1(rho) within
1e-5 of the oracle, relative to L1 of rho.
"""
import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def amr(w, **kw):
    from paper_2508_05020_gb300.amr import AMR
    return AMR(w, **kw)


def oracle(w):
    from oracle.amr import Oracle
    return Oracle(w)


def compare(gpu, ref, tol=TOL64):
    """Patch lists bit-exact, data within tol relative max-norm per variable."""
    worst = 0.0
    for l in range(ref.L):
        cg, xg = gpu.get_level(l)
        cr, xr = ref.get_level(l)
        assert np.array_equal(cg, cr), 'level %d patch lists differ' % l
        if len(cr) == 0:
            continue
        for v in range(ref.nv):
            scale = max(np.max(np.abs(xr[:, v])), 1e-300)
            err = np.max(np.abs(xg[:, v] - xr[:, v])) / scale
            worst = max(worst, err)
            assert err <= tol, (l, v, err)
    return worst


def run_both(w, steps, regrid=True, **kw):
    g = amr(w, **kw)
    r = oracle(w)
    compare(g, r, tol=1e-15)           # initial hierarchy and point-sampled state
    for _ in range(steps):
        dg = g.step()
        dr = r.step()
        assert abs(dg - dr) <= 1e-12 * dr, (dg, dr)
        if regrid:
            g.regrid()
            r.regrid()
    return g, r


# the FP64 path evaluates the oracle's expressions operation for operation
# (no FMA contraction, IEEE division and square root), so it reproduces the
# oracle bit for bit; only initial conditions with sin() (CUDA's sin against
# the host's) may differ in the last bit, and there the 1e-9 bar applies
@pytest.mark.parametrize('name,kw,steps,tol', [
    ('sod', {}, 25, 0.0),
    ('sod', dict(levels=2, patch=8, base_cells=(32, 1, 1)), 15, 0.0),
    ('shu_osher', {}, 6, TOL64),
    ('density_wave', dict(levels=2, patch=16), 5, TOL64),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8), 4, 0.0),
    ('riemann2d', dict(base_cells=(64, 64, 1)), 2, 0.0),
    ('dmr', dict(base_cells=(64, 16, 1), patch=8, levels=3), 3, 0.0),
    ('implosion', dict(base_cells=(32, 32, 1), patch=8, levels=3), 4, 0.0),
    ('constant', {}, 3, 0.0),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2), 2, 0.0),
    ('blast3d', dict(base_cells=(32, 32, 32), patch=16, levels=2), 1, 0.0),
    # the HLLC flux option
    ('sod', dict(flux='hllc'), 25, 0.0),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8, flux='hllc'), 4, 0.0),
    ('dmr', dict(base_cells=(64, 16, 1), patch=8, levels=3, flux='hllc'), 3, 0.0),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2, flux='hllc'), 2, 0.0),
    # the shock-free central schemes (Eqs. 8-9); Sod exercises their positivity guard
    ('density_wave', dict(levels=2, patch=16, flux='central'), 5, TOL64),
    ('sod', dict(flux='central'), 8, 0.0),
    ('shear2d', dict(base_cells=(32, 32, 1), patch=8, levels=3), 4, TOL64),
    ('shear2d', dict(base_cells=(64, 64, 1), patch=16, levels=3), 2, TOL64),
    # the hybrid flux: the central value where the shock sensor is quiet,
    # WENO5 + Rusanov at shocks, face by face
    ('sod', dict(flux='hybrid'), 25, 0.0),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8, flux='hybrid'), 4, 0.0),
    ('dmr', dict(base_cells=(64, 16, 1), patch=8, levels=3, flux='hybrid'), 3, 0.0),
    ('implosion', dict(base_cells=(32, 32, 1), patch=8, levels=3, flux='hybrid'), 4, 0.0),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2, flux='hybrid'), 2, 0.0),
    ('blast3d', dict(base_cells=(32, 32, 32), patch=16, levels=2, flux='hybrid'), 1, 0.0),
    ('shu_osher', dict(flux='hybrid', theta_switch=0.02), 6, TOL64),
    # 32-cell patches in 2D, a single level in 3D
    ('riemann2d', dict(base_cells=(128, 128, 1), patch=32, levels=2), 3, 0.0),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=1), 2, 0.0),
])
def test_fp64_matches_oracle(name, kw, steps, tol):
    w = workload(name, **kw)
    g, r = run_both(w, steps)
    compare(g, r, tol=tol)
    tg, cg, _ = g.diag()
    assert abs(tg - r.t) <= 1e-12 * r.t
    g.close()


def test_fp64_sod_to_t_end_matches_oracle_and_exact_solution():
    from oracle import riemann
    w = workload('sod')
    g = amr(w)
    r = oracle(w)
    while r.t < w['t_end'] - 1e-14:
        g.step()
        g.regrid()
        r.step()
        r.regrid()
    compare(g, r)
    rho = r.leaf_field(0)[0, 0]
    x = (np.arange(rho.size) + 0.5) / rho.size
    ex, _, _ = riemann.sample((1, 0, 1), (0.125, 0, 0.1), 1.4, x, 0.5, r.t)
    assert np.mean(np.abs(rho - ex)) < 0.006
    g.close()


def l1_rho_rel(gpu, ref):
    """Relative L1(rho) of the gpu state against the oracle on the finest composite."""
    num = den = 0.0
    for l in range(ref.L):
        cg, xg = gpu.get_level(l)
        cr, xr = ref.get_level(l)
        assert np.array_equal(cg, cr)
        vol = 1.0
        for d in range(ref.dim):
            vol *= ref.dx[l][d]
        keys = ref.mesh.level_list(l)
        for i, k in enumerate(keys):
            if ref.mesh.is_leaf(k):
                num += np.sum(np.abs(xg[i, 0] - xr[i, 0])) * vol
                den += np.sum(np.abs(xr[i, 0])) * vol
    return num / den


@pytest.mark.parametrize('name,kw,steps', [
    ('sod', {}, 60),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8), 6),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2), 2),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8, flux='hllc'), 6),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2, flux='hllc'), 2),
    ('blast3d', dict(base_cells=(32, 32, 32), patch=16, levels=2), 1),
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8, flux='hybrid'), 6),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2, flux='hybrid'), 2),
    ('blast3d', dict(base_cells=(32, 32, 32), patch=16, levels=2, flux='hybrid'), 1),
])
def test_fp32_l1_against_oracle(name, kw, steps):
    # same mesh sequence: both sides regrid from their own flags; a flag near
    # the threshold could differ, so the check runs without regrid
    w = workload(name, **kw)
    g = amr(w, precision=32)
    r = oracle(w)
    for _ in range(steps):
        dt = r.step()
        g.step(dt)
    err = l1_rho_rel(g, r)
    assert err <= 1e-5, err
    g.close()


def test_requests_bit_exact_given_identical_state():
    # the oracle's state after a few steps, uploaded as is: flags, requests and
    # the regrid outcome must match exactly
    w = workload('riemann2d', base_cells=(32, 32, 1), patch=8)
    r = oracle(w)
    for _ in range(3):
        r.step()
        r.regrid()
    g = amr(w)
    keys = r.mesh.canonical()
    levels = np.array([k[0] for k in keys])
    coords = np.array([[k[1][0], k[1][1]] for k in keys])
    data = np.stack([r.U[k][r.inner()].reshape((r.nv, r.N, r.N)) for k in keys])
    g.set_state(levels, coords, data, t=r.t)
    compare(g, r, tol=0.0)
    rg, cg = g.requests()
    rr, cr, _ = r.requests()
    assert [tuple(x) for x in rg] == [(k[0],) + k[1] for k in rr]
    assert [tuple(x) for x in cg] == [(k[0],) + k[1] for k in cr]
    g.regrid()
    r.regrid()
    compare(g, r, tol=0.0)
    g.close()


def test_conservation_periodic_fp64():
    w = workload('implosion', base_cells=(64, 64, 1), patch=16, levels=3)
    g = amr(w)
    _, c0, _ = g.diag()
    for _ in range(6):
        g.step()
        g.regrid()
    _, c1, ppl = g.diag()
    assert np.all(np.abs(c1 - c0) <= 1e-13 * np.maximum(np.abs(c0), 1.0)), (c0, c1)
    g.close()


def test_uniform_fine_equivalence_gpu():
    w = workload('riemann2d', base_cells=(32, 32, 1), patch=8, levels=2, theta_rho=-1.0, theta_p=-1.0)
    wu = workload('riemann2d', base_cells=(64, 64, 1), patch=8, levels=1)
    a = amr(w)
    b = amr(wu)
    for _ in range(3):
        assert a.step() == b.step()
        a.regrid()
    ca, xa = a.get_level(1)
    cb, xb = b.get_level(0)
    assert np.array_equal(ca, cb)
    assert np.array_equal(xa, xb)
    a.close()
    b.close()


@pytest.mark.parametrize('precision', [64, 32])
def test_modes_agree_bitwise(precision):
    # one launch per patch, batched without graph, batched with graph
    w = workload('dmr', base_cells=(64, 16, 1), patch=8, levels=3)
    runs = [amr(w, precision=precision, mode='per_patch'),
            amr(w, precision=precision, use_graph=False),
            amr(w, precision=precision)]
    for _ in range(3):
        dts = [x.step() for x in runs]
        assert dts[0] == dts[1] == dts[2]
        for x in runs:
            x.regrid()
    for l in range(w['levels']):
        ref = runs[0].get_level(l)
        for x in runs[1:]:
            c, d = x.get_level(l)
            assert np.array_equal(c, ref[0]) and np.array_equal(d, ref[1])
    for x in runs:
        x.close()


def test_pool_exhaustion_leaves_state_unchanged():
    # a uniform state builds no refinement; then the implosion data (level 0
    # only) asks for more patches than the pool holds
    from paper_2508_05020_gb300.amr import AMRError
    from oracle.amr import Oracle
    w = workload('implosion', base_cells=(32, 32, 1), patch=8, levels=3)
    g = amr(workload('implosion', base_cells=(32, 32, 1), patch=8, levels=3, ic='constant'), max_patches=24)
    r = Oracle(w, init=False)
    keys = r.mesh.canonical()
    data = np.stack([r.ic_fill(k)[r.inner()].reshape((4, 8, 8)) for k in keys])
    g.set_state(np.zeros(len(keys), dtype=np.int32), np.array([[k[1][0], k[1][1]] for k in keys]), data)
    keys0 = g.patch_keys()
    _, x0 = g.get_level(0)
    with pytest.raises(AMRError) as e:
        g.regrid()
    assert 'POOL' in str(e.value)
    assert g.patch_keys() == keys0
    _, x1 = g.get_level(0)
    assert np.array_equal(x0, x1)
    g.close()


def test_nonfinite_state_is_reported():
    from paper_2508_05020_gb300.amr import AMRError
    w = workload('sod', levels=1)
    g = amr(w)
    c, x = g.get_level(0)
    x[1, 0, 3] = -1.0                  # negative density in one cell
    g.set_state(np.zeros(len(c), dtype=np.int32), c, x)
    with pytest.raises(AMRError) as e:
        g.step()
    assert 'NONFINITE' in str(e.value)
    g.close()


def test_invalid_arguments_rejected():
    from paper_2508_05020_gb300.amr import AMRError
    with pytest.raises(AMRError):
        amr(workload('sod', patch=12))
    with pytest.raises(AMRError):
        amr(workload('sod', base_cells=(40, 1, 1)))
    g = amr(workload('riemann2d', base_cells=(32, 32, 1), patch=8))
    with pytest.raises(AMRError) as e:
        # a level-1 patch without its siblings breaks the tree structure
        g.set_state(np.array([0] * 16 + [1]), np.array([[i % 4, i // 4] for i in range(16)] + [[0, 0]]),
                    np.ones((17, 4, 8, 8)))
    assert 'MESH' in str(e.value)
    g.close()


def smooth3d_hierarchy(patch, levels, flux):
    """A refined 3D hierarchy (the shear layers, refined about y = -+0.15,
    which the domain places inside patches so that refinement is partial)
    carrying a smooth periodic field that varies along x, y and z, on the
    oracle."""
    w = workload('shear2d', dim=3, base_cells=(16, 16, 16), patch=patch, levels=levels, flux=flux,
                 lo=(-0.3, -0.35, -0.3), hi=(0.3, 0.25, 0.3), theta_rho=0.05, theta_p=0.05,
                 bc=(('periodic', 'periodic'),) * 3)
    r = oracle(w)
    from oracle import euler
    for k in r.mesh.canonical():
        _, X = r.cells(k, [0, 0, 0], [r.N] * 3)
        ph = 2.0 * np.pi * (X[0] + 2.0 * X[1] - X[2]) / 0.6
        rho = 1.0 + 0.2 * np.sin(ph)
        u = [0.3 + 0.1 * np.cos(ph), -0.2 + 0.05 * np.sin(2.0 * ph), 0.1 * np.cos(ph + 2.0 * np.pi * X[2] / 0.6)]
        pr = 1.0 + 0.1 * np.cos(ph)
        r.U[k][r.inner()] = np.stack(euler.conserved_from_primitive(rho, u, pr, 1.4))
    return w, r


@pytest.mark.parametrize('patch,levels,flux', [(8, 3, 'central'), (16, 2, 'central'), (16, 2, 'hybrid')])
def test_fp64_central_3d_bitwise_given_identical_state(patch, levels, flux):
    # every dimension's pencils see variation (the z pencils included); the
    # hybrid flux takes the central value at every face of this smooth field
    w, r = smooth3d_hierarchy(patch, levels, flux)
    n = [len(r.mesh.level_list(l)) for l in range(levels)]
    assert n[-1] > 0 and (levels == 2 or n[-1] < 8 * n[-2]), n
    g = amr(w)
    keys = r.mesh.canonical()
    g.set_state(np.array([k[0] for k in keys]), np.array([list(k[1]) for k in keys]),
                np.stack([r.U[k][r.inner()] for k in keys]), t=0.0)
    compare(g, r, tol=0.0)
    for _ in range(2):
        dr = r.step()
        dg = g.step()
        assert dg == dr
    compare(g, r, tol=0.0)
    g.close()


@pytest.mark.parametrize('name,kw,steps', [
    ('shear2d', dict(base_cells=(64, 64, 1), patch=16, levels=3), 4),
    ('density_wave', dict(levels=2, patch=16, flux='central'), 20),
])
def test_fp32_central_l1_rho(name, kw, steps):
    w = workload(name, **kw)
    g = amr(w, precision=32)
    r = oracle(w)
    for _ in range(steps):
        dt = r.step()
        g.step(dt)
        r.regrid()
        g.regrid()
    err = l1_rho_rel(g, r)
    assert err <= 1e-5, err
    g.close()


def test_fp32_central_3d_given_identical_state():
    # the FP32 central instantiation in 3D (four-plane chunks at N = 16) on
    # the smooth field of the refined 3D hierarchy
    w, r = smooth3d_hierarchy(16, 2, 'central')
    g = amr(w, precision=32)
    keys = r.mesh.canonical()
    g.set_state(np.array([k[0] for k in keys]), np.array([list(k[1]) for k in keys]),
                np.stack([r.U[k][r.inner()] for k in keys]), t=0.0)
    for _ in range(2):
        dt = r.step()
        g.step(dt)
    err = l1_rho_rel(g, r)
    assert err <= 1e-5, err
    g.close()
