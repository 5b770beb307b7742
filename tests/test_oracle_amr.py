"""Pins of the oracle's AMR solver: conservation, uniform-fine equivalence,
ghost fill, prolongation, restriction and the refinement sensor (no GPU)."""
import numpy as np
import pytest

from oracle import euler
from oracle.amr import G, Oracle, minmod
from synth import workload


def rel_change(s, s0):
    return np.abs(s - s0) / np.maximum(np.abs(s0), 1.0)


@pytest.mark.parametrize('base', [(32, 32, 1), (32, 16, 1)])
def test_conservation_periodic_with_regrid(base):
    # the implosion problem of Sec. 6 (Eq. 13) on a periodic box, 3 levels;
    # with 32 x 16 base cells dy = 2 dx, so the coarse-fine corrections of the
    # two dimensions differ in their cell size
    w = workload('implosion', base_cells=base, patch=8, levels=3)
    o = Oracle(w)
    s0 = o.cons_sums()
    meshes = set()
    # thresholds switch between the default, 'nothing flags' (coarsen) and
    # 'everything flags' (refine), so every regrid path runs
    for th in (0.05, 0.05, 10.0, 10.0, 0.05, -1.0, 0.05, 10.0):
        o.w['theta_rho'] = o.w['theta_p'] = th
        o.step()
        o.regrid()
        meshes.add(tuple(o.mesh.canonical()))
        assert np.all(rel_change(o.cons_sums(), s0) < 1e-13)
    assert len(meshes) > 3            # the hierarchy changed along the way


def test_conservation_reflecting_box_mass_energy():
    w = workload('implosion', base_cells=(16, 16, 1), patch=8, levels=3,
                 bc=(('reflect', 'reflect'), ('reflect', 'reflect'), ('outflow', 'outflow')),
                 lo=(-0.15, -0.3, 0.0), hi=(0.45, 0.3, 1.0))
    o = Oracle(w)
    s0 = o.cons_sums()
    for _ in range(10):
        o.step()
        o.regrid()
    s = o.cons_sums()
    assert rel_change(s, s0)[0] < 1e-13
    assert rel_change(s, s0)[3] < 1e-13


def test_conservation_3d_periodic():
    w = workload('blast3d', base_cells=(16, 16, 16), patch=8, levels=2,
                 bc=(('periodic', 'periodic'),) * 3)
    o = Oracle(w)
    s0 = o.cons_sums()
    for _ in range(2):
        o.step()
        o.regrid()
    assert np.all(rel_change(o.cons_sums(), s0) < 1e-13)


def finest_equals_uniform(name, levels, steps, **kw):
    """Refine everything (negative thresholds flag every cell) and compare the
    finest level with a single-level run at the finest spacing."""
    w = workload(name, theta_rho=-1.0, theta_p=-1.0, levels=levels, **kw)
    base_f = tuple(b * 2 ** (levels - 1) if d < w['dim'] else 1 for d, b in enumerate(w['base_cells']))
    wu = workload(name, levels=1, **dict(kw, base_cells=base_f))
    a = Oracle(w)
    b = Oracle(wu)
    n_f = 1
    for d in range(w['dim']):
        n_f *= base_f[d] // w['patch']
    assert len(a.mesh.level_list(levels - 1)) == n_f
    for _ in range(steps):
        da = a.step()
        a.regrid()
        db = b.step()
        assert da == db
    ca, xa = a.get_level(levels - 1)
    cb, xb = b.get_level(0)
    assert np.array_equal(ca, cb)
    assert np.array_equal(xa, xb)           # bitwise


def test_uniform_fine_equivalence_1d_sod():
    finest_equals_uniform('sod', 3, 6)


def test_uniform_fine_equivalence_2d_riemann():
    finest_equals_uniform('riemann2d', 2, 3, base_cells=(16, 16, 1), patch=8)


def test_uniform_fine_equivalence_2d_dmr_time_dependent_boundaries():
    finest_equals_uniform('dmr', 2, 3, base_cells=(32, 8, 1), patch=8)


def test_uniform_fine_equivalence_2d_periodic():
    finest_equals_uniform('implosion', 2, 3, base_cells=(16, 16, 1), patch=8)


def test_uniform_fine_equivalence_3d():
    # the seeded perturbation is keyed to base-level cells, which differ here
    finest_equals_uniform('blast3d', 2, 1, base_cells=(8, 8, 8), patch=8, amp=0.0)


@pytest.mark.parametrize('name,kw', [
    ('riemann2d', dict(base_cells=(32, 32, 1), patch=8, levels=3)),
    ('dmr', dict(base_cells=(64, 16, 1), patch=8, levels=3)),
    ('blast3d', dict(base_cells=(16, 16, 16), patch=8, levels=2)),
])
def test_halo_poisoning(name, kw):
    # every ghost cell of every patch is written by the fill: poison with NaN,
    # fill, and no NaN may remain anywhere in any slot
    o = Oracle(workload(name, **kw))
    for k in o.mesh.canonical():
        A = o.U[k]
        inner = A[o.inner()].copy()
        A[...] = np.nan
        A[o.inner()] = inner
    o.fill_ghosts(o.U, 0.0)
    for k in o.mesh.canonical():
        assert not np.any(np.isnan(o.U[k])), k


def test_minmod_rule():
    a = np.array([1.0, -1.0, 2.0, -3.0, 0.0, 1.0, 2.0])
    b = np.array([2.0, -3.0, 1.0, 1.0, 5.0, 1.0, -2.0])
    assert np.array_equal(minmod(a, b), [1.0, -1.0, 1.0, 0.0, 0.0, 1.0, 0.0])


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_prolongation_conservative_and_linear_exact(dim):
    w = workload({1: 'sod', 2: 'riemann2d', 3: 'blast3d'}[dim], levels=2,
                 base_cells=tuple(16 if d < dim else 1 for d in range(3)), patch=8)
    o = Oracle(w, init=False)
    for k in o.mesh.canonical():
        o.U[k] = o.ic_fill(k)
    rng = np.random.default_rng(3)
    key = (0, (0, 0, 0))
    A = o.U[key]
    # a positive linear state: prolongation reproduces it exactly
    sl = o.inner()
    Zs, Ys, Xs = A.shape[1:]
    zz, yy, xx = np.meshgrid(np.arange(Zs), np.arange(Ys), np.arange(Xs), indexing='ij')
    lin = 2.0 + 0.01 * xx + (0.02 * yy if dim >= 2 else 0) + (0.03 * zz if dim == 3 else 0)
    A[0] = lin
    for d in range(dim):
        A[1 + d] = 0.0
    A[dim + 1] = 10.0 * lin
    child = (1, (0, 0, 0))
    Gi, _ = o.cells(child, [0, 0, 0], [o.N] * 3)
    vals = o.prolong_cells(o.U, child, Gi)
    fine = vals.reshape((o.nv,) + Gi[0].shape)
    fx = (Gi[0] + 0.5) / 2.0 - 0.5 + G          # coarse slot coordinate of the fine centre
    fy = (Gi[1] + 0.5) / 2.0 - 0.5 + G
    fz = (Gi[2] + 0.5) / 2.0 - 0.5 + G
    exp = 2.0 + 0.01 * fx + (0.02 * fy if dim >= 2 else 0) + (0.03 * fz if dim == 3 else 0)
    assert np.allclose(fine[0], exp, rtol=1e-14)
    # random positive data: the mean of the 2^d children equals the coarse cell
    A[0] = 1.0 + rng.uniform(0, 1, A[0].shape)
    A[dim + 1] = 5.0 + rng.uniform(0, 1, A[0].shape)
    vals = o.prolong_cells(o.U, child, Gi).reshape((o.nv,) + Gi[0].shape)
    acc = 0.0
    for sz in ((0, 1) if dim == 3 else (None,)):
        for sy in ((0, 1) if dim >= 2 else (None,)):
            for sx in (0, 1):
                s = [slice(None)]
                for s_ in (sz, sy, sx):
                    s.append(slice(None) if s_ is None else slice(s_, None, 2))
                acc = acc + vals[tuple(s)]
    coarse = A[(slice(None),) + tuple(slice(G, G + o.N // 2) if d < dim else slice(None) for d in (2, 1, 0))]
    assert np.allclose(acc / 2 ** dim, coarse, rtol=1e-14)


def test_prolongation_positivity_fallback():
    w = workload('sod', levels=2, base_cells=(16, 1, 1), patch=8)
    o = Oracle(w, init=False)
    for k in o.mesh.canonical():
        o.U[k] = o.ic_fill(k)
    A = o.U[(0, (0, 0, 0))]
    # coarse densities 1, 1e-3, 1: minmod slope 0 -> plain copy; make a steep
    # monotone energy drop so a child pressure would turn negative
    A[0, 0, 0, G:G + 3] = [1.0, 1.0, 1.0]
    A[1, 0, 0, G:G + 3] = [0.0, 2.0, 4.0]
    A[2, 0, 0, G:G + 3] = [1.0, 2.5, 10.0]
    Gi, _ = o.cells((1, (0, 0, 0)), [2, 0, 0], [4, 1, 1])   # children of coarse cell 1
    vals = o.prolong_cells(o.U, (1, (0, 0, 0)), Gi)
    assert np.allclose(vals[:, 0], A[:, 0, 0, G + 1])
    assert np.allclose(vals[:, 1], A[:, 0, 0, G + 1])


def test_restriction_is_mean_of_children():
    w = workload('riemann2d', levels=2, base_cells=(16, 16, 1), patch=8, theta_rho=-1.0, theta_p=-1.0)
    o = Oracle(w)
    rng = np.random.default_rng(4)
    for k in o.mesh.level_list(1):
        o.U[k][o.inner()] = rng.uniform(1, 2, o.U[k][o.inner()].shape)
    o.restrict(o.U)
    pk = (0, (0, 0, 0))
    ch = o.U[(1, (0, 0, 0))][o.inner()]
    m = (ch[:, :, 0:2, 0:2]).reshape(o.nv, -1).mean(axis=1)
    assert np.allclose(o.U[pk][:, 0, G, G], m, rtol=1e-15)


def test_sensor_flags_only_around_a_jump():
    w = workload('sod', levels=1, base_cells=(64, 1, 1), patch=16)
    o = Oracle(w)
    o.fill_ghosts(o.U, 0.0)
    flagged = {k[1][0]: np.nonzero(o.patch_flags(k)[0, 0])[0] - 2 for k in o.mesh.canonical()}
    # jump between global cells 31 and 32: only cells 31 and 32 flag
    assert list(flagged[0]) == []
    assert list(flagged[1]) == [15, 16]     # local 15 (global 31) and band cell 16 (global 32)
    assert list(flagged[2]) == [-1, 0]
    assert list(flagged[3]) == []


def test_cfl_matches_definition():
    w = workload('sod', levels=1)
    o = Oracle(w)
    dt = o.cfl_dt()
    # left state: c = sqrt(1.4), dx = 1/64
    assert dt == pytest.approx(0.5 / (np.sqrt(1.4) * 64.0), rel=1e-14)
    rho, u, p, T = euler.primitives(o.U[(0, (0, 0, 0))][o.inner()], 1, 1.4)
    assert np.allclose(p, 1.0)


@pytest.mark.parametrize('dim', [2, 3])
def test_cfl_sums_over_dimensions_with_their_cell_sizes(dim):
    # uniform rho = 1, u = (0.3, -0.2, 0.1), p = 1 on the unit box with 8, 16
    # and 32 cells along x, y, z: dt = CFL / sum_d (|u_d| + c) n_d, c = sqrt(1.4)
    base = (8, 16, 32 if dim == 3 else 1)
    bc = tuple(('periodic', 'periodic') for _ in range(3))
    o = Oracle(workload('constant', dim=dim, base_cells=base, patch=8, levels=1, bc=bc))
    c = np.sqrt(1.4)
    lam = sum((abs(v) + c) * n for v, n in zip((0.3, -0.2, 0.1)[:dim], base[:dim]))
    assert o.cfl_dt() == pytest.approx(0.5 / lam, rel=1e-14)


def test_four_quadrant_keeps_its_diagonal_symmetry_through_regrids():
    # the four-quadrant states are symmetric under x <-> y (with u <-> v) and
    # so are the outflow boundaries: flags, Algorithm 1 and the coarsening rule
    # (both independent of the order of their inputs) give a symmetric mesh
    # at every regrid, and the fields stay symmetric to round-off (the
    # prolongation, the face corrections and the restriction visit x before y)
    w = workload('riemann2d', base_cells=(32, 32, 1), patch=8, levels=3)
    o = Oracle(w)
    for _ in range(8):
        o.step()
        o.regrid()
        assert {(l, (c[1], c[0], c[2])) for l, c in o.mesh.patches} == o.mesh.patches
        F = [o.leaf_field(v)[0] for v in range(4)]
        for a, b in ((0, 0), (3, 3), (1, 2)):
            assert np.max(np.abs(F[a] - F[b].T)) <= 1e-13 * np.max(np.abs(F[a]))
    assert 0 < len(o.mesh.level_list(2)) < 4 * 4 * 16          # partly refined


def test_unperturbed_blast_keeps_the_cube_symmetries():
    # the blast without its density perturbation is symmetric under every
    # exchange of two axes (with the momentum components exchanged alike); on
    # 3^3 base patches, partly refined, the mesh keeps every symmetry exactly
    # and the fields to round-off
    w = workload('blast3d', base_cells=(24, 24, 24), patch=8, levels=2, amp=0.0)
    o = Oracle(w)
    for _ in range(3):
        o.step()
        o.regrid()
        for perm in ((1, 0, 2), (0, 2, 1), (2, 1, 0)):
            assert {(l, tuple(c[perm[d]] for d in range(3))) for l, c in o.mesh.patches} == o.mesh.patches
        F = [o.leaf_field(v) for v in range(5)]                  # axes (z, y, x)
        for axes, (ma, mb) in (((0, 2, 1), (1, 2)), ((2, 1, 0), (1, 3)), ((1, 0, 2), (2, 3))):
            for a in range(5):
                b = mb if a == ma else (ma if a == mb else a)
                assert np.max(np.abs(F[a] - np.transpose(F[b], axes))) <= 1e-13 * np.max(np.abs(F[a])), (axes, a)
    assert 27 < len(o.mesh.patches) < 27 * 9


def test_stage_times_of_ssp_rk3(monkeypatch):
    # the Shu-Osher stages evaluate the right-hand side at t, t + dt and
    # t + dt/2 (the abscissae of SSP-RK3), so time-dependent boundaries are
    # filled at those times: the ghost fills of one step see exactly them
    o = Oracle(workload('dmr', base_cells=(32, 8, 1), patch=8, levels=1))
    o.t = 0.0125
    seen = []
    real = Oracle.fill_ghosts

    def spy(self, U, t):
        seen.append(t)
        return real(self, U, t)

    monkeypatch.setattr(Oracle, 'fill_ghosts', spy)
    dt = 1e-3
    o.step(dt)
    assert seen == [0.0125, 0.0125 + dt, 0.0125 + 0.5 * dt]
    assert o.t == 0.0125 + dt


def test_reflecting_wall_is_the_mirror_image():
    # method of images: a state on [0, 1] beside a reflecting wall at x = 0
    # evolves as the right half of the mirror-symmetric state on [-1, 1]
    # (density and energy even, momentum odd); with the Rusanov flux, which
    # keeps mirror symmetry exactly, the two runs agree bit for bit
    rng = np.random.default_rng(8)
    n = 64
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.5 * np.exp(-((x - 0.3) / 0.1) ** 2) + 0.05 * rng.uniform(size=n)
    u = 0.4 * np.sin(3.0 * x) + 0.05 * rng.uniform(size=n)
    p = 1.0 + 0.8 * (x < 0.2) + 0.05 * rng.uniform(size=n)
    U = np.stack(euler.conserved_from_primitive(rho, [u], p, 1.4))
    half = Oracle(workload('sod', levels=1, base_cells=(n, 1, 1),
                           bc=(('reflect', 'outflow'), ('outflow', 'outflow'), ('outflow', 'outflow'))))
    full = Oracle(workload('sod', levels=1, base_cells=(2 * n, 1, 1), lo=(-1.0, 0.0, 0.0)))
    M = np.concatenate([U[:, ::-1] * np.array([[1.0], [-1.0], [1.0]]), U], axis=1)

    def put(o, A):
        for k in o.mesh.canonical():
            c = k[1][0]
            o.U[k][o.inner()] = A[:, c * 16:(c + 1) * 16].reshape(o.U[k][o.inner()].shape)

    put(half, U)
    put(full, M)
    for _ in range(12):
        dt = half.step()
        assert full.step() == dt
    for v in range(3):
        assert np.array_equal(full.leaf_field(v)[0, 0, n:], half.leaf_field(v)[0, 0])


def test_conservation_periodic_hybrid_flux():
    # the face-by-face switch between the central value and WENO5 + Rusanov
    # keeps one value per face, so the sums over leaves telescope through the
    # coarse-fine corrections on a refined periodic implosion (which has both
    # quiet and shocked faces)
    w = workload('implosion', base_cells=(32, 32, 1), patch=8, levels=3, flux='hybrid')
    o = Oracle(w)
    s0 = o.cons_sums()
    for _ in range(6):
        o.step()
        o.regrid()
        assert np.all(rel_change(o.cons_sums(), s0) < 1e-13)
