"""Workload parameter tables.

Each workload is a plain dict of numbers and names. Both the oracle and the
CUDA library read these parameters; each side implements the initial
condition, the boundary rule and every numerical step on its own.

Fields
------
dim            spatial dimension d (1, 2 or 3)
lo, hi         domain corners (3 entries; unused dimensions are [0, 1])
bc             per dimension a pair (low side, high side) of boundary kinds:
               'outflow', 'reflect', 'periodic', 'dmr_inflow', 'dmr_bottom', 'dmr_top'
gamma          ratio of specific heats (R = 1 throughout, Sec. 6)
base_cells     level-0 cells per dimension (unused dimensions are 1)
levels         number of levels L, the base level included
patch          cells per patch side N (every patch has the same size, Sec. 4.2)
ic             initial-condition name
cfl            CFL number
t_end          final time (the time step is clipped to it)
theta_rho/p    thresholds of the relative-jump refinement sensor
flux           numerical flux at faces: 'rusanov' (Sec. 3.2), 'hllc' (an option),
               'central' (the shock-free central interpolation and 4th-order
               staggered divergence of Sec. 3.2, Eqs. 8-9) or 'hybrid' (the
               central face value where a shock sensor is quiet, WENO5 +
               Rusanov elsewhere, face by face)
theta_switch   threshold of the hybrid flux's shock sensor (relative jump of rho
               and p along the pencil; 0.05)
seed           seed of the +-1 % density perturbation (blast only)
amp            amplitude of that perturbation (blast only; 0.01)

The five named workloads are the shock-tube, shock-entropy, four-quadrant,
double-Mach-reflection and 3D blast problems; ``implosion`` is the periodic
demonstration problem of Sec. 6 (Eq. 13) and ``shear2d`` its second one.
"""
import copy

_OUT = ('outflow', 'outflow')
_PER = ('periodic', 'periodic')
_UNUSED = ('outflow', 'outflow')

WORKLOADS = {
    # 1D Sod shock tube: 64 base cells, 2 ratio-2 refinement levels above the base,
    # 16-cell patches, CFL 0.5, t_end 0.2.
    'sod': dict(dim=1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                bc=(_OUT, _UNUSED, _UNUSED), gamma=1.4,
                base_cells=(64, 1, 1), levels=3, patch=16, ic='sod',
                cfl=0.5, t_end=0.2, theta_rho=0.05, theta_p=0.05, seed=0),
    # 1D Shu-Osher shock-entropy interaction on [-5, 5]: 256 base cells, 4 levels,
    # 32-cell patches, t_end 1.8.
    'shu_osher': dict(dim=1, lo=(-5.0, 0.0, 0.0), hi=(5.0, 1.0, 1.0),
                      bc=(_OUT, _UNUSED, _UNUSED), gamma=1.4,
                      base_cells=(256, 1, 1), levels=4, patch=32, ic='shu_osher',
                      cfl=0.5, t_end=1.8, theta_rho=0.05, theta_p=0.05, seed=0),
    # 2D four-quadrant Riemann problem on [0,1]^2: 256^2 base, 3 levels, 16^2 patches,
    # t_end 0.3.
    'riemann2d': dict(dim=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                      bc=(_OUT, _OUT, _UNUSED), gamma=1.4,
                      base_cells=(256, 256, 1), levels=3, patch=16, ic='riemann2d',
                      cfl=0.5, t_end=0.3, theta_rho=0.05, theta_p=0.05, seed=0),
    # 2D Mach-10 double Mach reflection on [0,4]x[0,1]: 512x128 base, 4 levels,
    # 16^2 patches, t_end 0.2.
    'dmr': dict(dim=2, lo=(0.0, 0.0, 0.0), hi=(4.0, 1.0, 1.0),
                bc=(('dmr_inflow', 'outflow'), ('dmr_bottom', 'dmr_top'), _UNUSED),
                gamma=1.4, base_cells=(512, 128, 1), levels=4, patch=16, ic='dmr',
                cfl=0.5, t_end=0.2, theta_rho=0.05, theta_p=0.05, seed=0),
    # 3D spherical blast in the unit box: 128^3 base, 3 levels, 16^3 patches,
    # t_end 0.05, +-1 % seeded density perturbation (seed 0).
    'blast3d': dict(dim=3, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                    bc=(_OUT, _OUT, _OUT), gamma=1.4,
                    base_cells=(128, 128, 128), levels=3, patch=16, ic='blast3d',
                    cfl=0.5, t_end=0.05, theta_rho=0.05, theta_p=0.05, seed=0, amp=0.01),
    # Implosion demonstration (Sec. 6, Eq. 13): periodic (-0.3, 0.3)^2, CFL 0.45.
    # 1024^2 finest-equivalent cells = 256^2 base with 3 levels.
    'implosion': dict(dim=2, lo=(-0.3, -0.3, 0.0), hi=(0.3, 0.3, 1.0),
                      bc=(_PER, _PER, _UNUSED), gamma=1.4,
                      base_cells=(256, 256, 1), levels=3, patch=16, ic='implosion',
                      cfl=0.45, t_end=0.0, theta_rho=0.05, theta_p=0.05, seed=0),
    # Smooth density wave rho = 1 + 0.2 sin(2 pi (x - t)), u = 1, p = 1 (periodic).
    'density_wave': dict(dim=1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                         bc=(_PER, _UNUSED, _UNUSED), gamma=1.4,
                         base_cells=(64, 1, 1), levels=1, patch=16, ic='density_wave',
                         cfl=0.5, t_end=0.0, theta_rho=0.05, theta_p=0.05, seed=0),
    # Periodic shear layers (Sec. 6, second demonstration): (-0.3, 0.3)^2, density
    # ratio 2, convective Mach number 0.7, perturbation with 5 periods across the
    # domain; shock-free, so the central schemes of Sec. 3.2 (flux 'central').
    # 1024^2 finest-equivalent cells = 256^2 base with 3 levels; CFL 0.45 as the
    # implosion. Sensor thresholds 0.01: the tanh layers (width 0.01, about 4
    # base cells) give relative jumps near 0.04 on level 0 and 0.02 on level 1,
    # so both coarse levels refine about them.
    'shear2d': dict(dim=2, lo=(-0.3, -0.3, 0.0), hi=(0.3, 0.3, 1.0),
                    bc=(_PER, _PER, _UNUSED), gamma=1.4,
                    base_cells=(256, 256, 1), levels=3, patch=16, ic='shear_layer',
                    cfl=0.45, t_end=0.0, theta_rho=0.01, theta_p=0.01, seed=0, flux='central'),
    # Uniform state rho = 1, u = (0.3, -0.2, 0.1), p = 1 (for constant preservation).
    'constant': dict(dim=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                     bc=(_PER, _OUT, _UNUSED), gamma=1.4,
                     base_cells=(32, 32, 1), levels=2, patch=8, ic='constant',
                     cfl=0.5, t_end=0.0, theta_rho=0.05, theta_p=0.05, seed=0),
}


def workload(name, **overrides):
    """Return a deep copy of a named workload with fields overridden."""
    w = copy.deepcopy(WORKLOADS[name])
    w['name'] = name
    w.setdefault('flux', 'rusanov')
    w.setdefault('theta_switch', 0.05)
    for k, v in overrides.items():
        if k not in w:
            raise KeyError(k)
        w[k] = v
    return w


def reduced(name):
    """Small variants used where the full-size run is too long for the oracle.

    double Mach reflection: 128x32 base; 3D blast: 32^3 base; four-quadrant:
    64^2 base; the 1D problems keep their full size.
    """
    if name == 'dmr':
        return workload('dmr', base_cells=(128, 32, 1))
    if name == 'blast3d':
        return workload('blast3d', base_cells=(32, 32, 32))
    if name == 'riemann2d':
        return workload('riemann2d', base_cells=(64, 64, 1))
    if name == 'implosion':
        return workload('implosion', base_cells=(64, 64, 1))
    return workload(name)


def fine_equivalent_cells(w):
    """Cells of a uniform grid at the finest level: base cells x 2^(d (L-1))."""
    n = 1
    for d in range(w['dim']):
        n *= w['base_cells'][d] * 2 ** (w['levels'] - 1)
    return n
