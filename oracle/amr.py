"""The AMR solver of the oracle: ghost fill, stages, reflux, restriction, CFL,
refinement sensor and regrid, on the hierarchy of ``oracle.mesh``.

Test infrastructure (see ``oracle/__init__``). FP64 numpy, one slot array per
patch with g = 3 ghost layers in every active dimension (the patch region of
Sec. 4.2 spans interior and ghost points). Array axis 3 - d holds dimension d.

Readings where the paper is silent (each is stated where it is used):
  * nodes are cell centres, x_i = lo + (i + 1/2) dx_l, dx_l = dx_0 / 2^l;
  * all levels advance with the same dt inside each SSP-RK3 stage (no subcycling);
  * ghost fill per level, coarse to fine: same-level copy, else limited-linear
    prolongation from level l-1, then physical boundaries (dims x, y, z in turn);
  * after each stage: reflux (coarse face flux replaced by the mean of the fine
    face fluxes, applied as a correction of the stage result), then conservative
    restriction from the finest level down;
  * refinement sensor: relative jump of rho and p over the patch band [-2, N+1]^d.
"""
import itertools
import math

import numpy as np

from . import euler
from .mesh import Mesh, canon

G = 3                                   # ghost layers (WENO5 needs i-2..i+3)
RK_A = (None, 0.75, 1.0 / 3.0)          # SSP-RK3 in Shu-Osher form (Sec. 3.2)
RK_B = (1.0, 0.25, 2.0 / 3.0)
GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


class OracleError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# initial conditions (Sec. 6, Eq. 13; shock-tube, shock-entropy, four-quadrant,
# double-Mach and blast set-ups), point-sampled at cell centres
# ---------------------------------------------------------------------------

def dmr_states(gamma):
    """Pre- and post-shock states of a Mach-10 shock entering gas at rest with
    (rho, p) = (1.4, 1), from the Rankine-Hugoniot relations of Eqs. 1-3. The
    post-shock velocity is normal to the shock line x = 1/6 + y/sqrt(3), i.e.
    along (cos 30deg, -sin 30deg). Returns ((rho, u, v, p) pre, post)."""
    M = 10.0
    r1, p1 = 1.4, 1.0
    c1 = math.sqrt(gamma * p1 / r1)
    W = M * c1
    r2 = r1 * (gamma + 1.0) * M * M / ((gamma - 1.0) * M * M + 2.0)
    p2 = p1 * (2.0 * gamma * M * M - (gamma - 1.0)) / (gamma + 1.0)
    un = W * (1.0 - r1 / r2)
    s3 = math.sqrt(3.0)
    return (r1, 0.0, 0.0, p1), (r2, un * (s3 * 0.5), -(un * 0.5), p2)


def splitmix64(seed, n):
    """Output n+1 of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014),
    mapped to [0, 1) with 53 bits. n is an int64 array of counters."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over='ignore'):
        z = np.uint64(seed) + (n + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def initial_primitive(w, X, Gidx, level):
    """(rho, [u_d], p) of a workload at cell centres X[d] (global cell indices
    Gidx[d] at `level`, used only by the seeded blast perturbation)."""
    dim = w['dim']
    ic = w['ic']
    shape = X[0].shape
    zero = np.zeros(shape)
    one = np.ones(shape)
    x = X[0]
    if ic == 'sod':
        left = x < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        u = [zero.copy() for _ in range(dim)]
    elif ic == 'shu_osher':
        left = x < -4.0
        rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
        u = [np.where(left, 2.629369, 0.0)] + [zero.copy() for _ in range(dim - 1)]
        p = np.where(left, 10.33333, 1.0)
    elif ic == 'riemann2d':
        y = X[1]
        east = x > 0.5
        north = y > 0.5
        # quadrant states (rho, u, v, p): NE, NW, SW, SE
        st = {(1, 1): (1.5, 0.0, 0.0, 1.5), (0, 1): (0.5323, 1.206, 0.0, 0.3),
              (0, 0): (0.138, 1.206, 1.206, 0.029), (1, 0): (0.5323, 0.0, 1.206, 0.3)}
        rho, ux, uy, p = zero.copy(), zero.copy(), zero.copy(), zero.copy()
        for (e, n), (r_, a_, b_, p_) in st.items():
            m = (east == bool(e)) & (north == bool(n))
            rho[m], ux[m], uy[m], p[m] = r_, a_, b_, p_
        u = [ux, uy] + [zero.copy() for _ in range(dim - 2)]
    elif ic == 'dmr':
        y = X[1]
        pre, post = dmr_states(w['gamma'])
        behind = x < 1.0 / 6.0 + y / math.sqrt(3.0)
        rho = np.where(behind, post[0], pre[0])
        u = [np.where(behind, post[1], pre[1]), np.where(behind, post[2], pre[2])]
        p = np.where(behind, post[3], pre[3])
    elif ic == 'blast3d':
        dxc = X[0] - 0.5
        dyc = X[1] - 0.5
        dzc = X[2] - 0.5
        r2 = dxc * dxc + dyc * dyc + dzc * dzc
        p = np.where(r2 < 0.01, 100.0, 0.1)
        nb = w['base_cells']
        ib = [Gidx[d] >> level for d in range(3)]
        lin = (ib[2] * nb[1] + ib[1]) * nb[0] + ib[0]
        xi = splitmix64(w['seed'], lin)
        rho = 1.0 + w['amp'] * (2.0 * xi - 1.0)
        u = [zero.copy() for _ in range(dim)]
    elif ic == 'implosion':
        inside = np.abs(X[0]) + np.abs(X[1]) < 0.15
        rho = np.where(inside, 0.125, 1.0)
        p = np.where(inside, 0.140, 1.0)
        u = [zero.copy() for _ in range(dim)]
    elif ic == 'density_wave':
        rho = 1.0 + 0.2 * np.sin(2.0 * math.pi * x)
        u = [one.copy()] + [zero.copy() for _ in range(dim - 1)]
        p = one.copy()
    elif ic == 'shear_layer':
        # two periodic shear layers at y = -0.15, 0.15 (Sec. 6): band |y| < 0.15
        # moves with +dU/2 at rho 1, the rest with -dU/2 at rho 2 (density ratio
        # 2), p = 1; dU = Mc (c1 + c2) for convective Mach number Mc = 0.7;
        # tanh profiles of thickness 0.01; the transverse velocity is perturbed
        # with 5 periods across the domain, Gaussian (width 0.02) about each layer
        y = X[1]
        g = w['gamma']
        c1 = math.sqrt(g * 1.0 / 1.0)
        c2 = math.sqrt(g * 1.0 / 2.0)
        du = 0.7 * (c1 + c2)
        f = 0.5 * (np.tanh((y + 0.15) / 0.01) - np.tanh((y - 0.15) / 0.01))
        rho = 2.0 + (1.0 - 2.0) * f
        ux = -0.5 * du + du * f
        a = (y - 0.15) / 0.02
        b = (y + 0.15) / 0.02
        uy = 0.05 * np.sin(2.0 * math.pi * 5.0 * (x + 0.3) / 0.6) * (np.exp(-(a * a)) + np.exp(-(b * b)))
        u = [ux, uy] + [zero.copy() for _ in range(dim - 2)]
        p = one.copy()
    elif ic == 'constant':
        vel = (0.3, -0.2, 0.1)
        rho = one.copy()
        u = [one * vel[d] for d in range(dim)]
        p = one.copy()
    else:
        raise OracleError('unknown initial condition ' + ic)
    return rho, u, p


def minmod(a, b):
    """0 if a b <= 0, else the argument of smaller magnitude (ties: the first)."""
    pick = np.where(np.abs(a) <= np.abs(b), a, b)
    return np.where(a * b <= 0.0, 0.0, pick)


class Oracle:
    """FP64 reference of the whole per-step path on one workload dict."""

    def __init__(self, w, init=True):
        self.w = w
        self.dim = w['dim']
        self.N = w['patch']
        self.L = w['levels']
        self.gamma = w['gamma']
        self.nv = self.dim + 2
        for d in range(self.dim):
            if w['base_cells'][d] % self.N:
                raise OracleError('base cells must be a multiple of the patch size')
        base_patches = [w['base_cells'][d] // self.N if d < self.dim else 1 for d in range(3)]
        self.periodic = tuple(w['bc'][d][0] == 'periodic' if d < self.dim else False for d in range(3))
        self.mesh = Mesh(self.dim, base_patches, self.periodic, self.L - 1)
        self.dx = [[(w['hi'][d] - w['lo'][d]) / float(w['base_cells'][d] * 2 ** l) for d in range(3)]
                   for l in range(self.L)]
        self.t = 0.0
        self.steps = 0
        self.U = {}
        self.flag_override = None       # callable(key, slot array) -> bool, e.g. a learned flagger
        if init:
            self.initialise()

    # ---- layout helpers -------------------------------------------------
    def slot_shape(self):
        return (self.nv,) + tuple(self.N + 2 * G if d < self.dim else 1 for d in (2, 1, 0))

    def inner(self):
        return tuple([slice(None)] + [slice(G, G + self.N) if d < self.dim else slice(None)
                                      for d in (2, 1, 0)])

    def cells(self, key, lo_local, hi_local):
        """Global cell indices and centres of a box of local indices [lo, hi)."""
        l, c = key
        rng = []
        for d in range(3):
            if d < self.dim:
                rng.append(np.arange(lo_local[d], hi_local[d]) + c[d] * self.N)
            else:
                rng.append(np.zeros(1, dtype=np.int64))
        Gz, Gy, Gx = np.meshgrid(rng[2], rng[1], rng[0], indexing='ij')
        Gi = [Gx, Gy, Gz]
        X = [self.w['lo'][d] + (Gi[d] + 0.5) * self.dx[l][d] for d in range(3)]
        return Gi, X

    def ic_fill(self, key):
        """Point-sample the initial condition into a patch interior."""
        l, _ = key
        Gi, X = self.cells(key, [0, 0, 0], [self.N] * 3)
        rho, u, p = initial_primitive(self.w, X, Gi, l)
        Uc = euler.conserved_from_primitive(rho, u, p, self.gamma)
        A = np.zeros(self.slot_shape())
        A[self.inner()] = np.stack(Uc)
        return A

    # ---- initial hierarchy --------------------------------------------------
    def initialise(self):
        """Level 0 with the initial condition, then L-1 rounds of flag -> regrid
        with the initial condition re-sampled on new patches."""
        for k in self.mesh.canonical():
            self.U[k] = self.ic_fill(k)
        for _ in range(self.L - 1):
            self.regrid(resample_ic=True)

    # ---- ghost fill ---------------------------------------------------------
    def _block(self, o):
        """Local index range [lo, hi) per dimension of the ghost block at offset o."""
        lo, hi = [], []
        for d in range(3):
            if d >= self.dim:
                lo.append(0)
                hi.append(1)
            elif o[d] < 0:
                lo.append(-G)
                hi.append(0)
            elif o[d] == 0:
                lo.append(0)
                hi.append(self.N)
            else:
                lo.append(self.N)
                hi.append(self.N + G)
        return lo, hi

    def _slot_slice(self, lo, hi):
        return tuple([slice(None)] + [slice(lo[d] + G, hi[d] + G) if d < self.dim else slice(None)
                                      for d in (2, 1, 0)])

    def _outside(self, key, o):
        l, c = key
        ext = self.mesh.extent(l)
        for d in range(self.dim):
            if self.periodic[d]:
                continue
            if o[d] < 0 and c[d] == 0:
                return True
            if o[d] > 0 and c[d] == ext[d] - 1:
                return True
        return False

    def prolong_cells(self, U, key, Gi):
        """Limited-linear coarse-to-fine prolongation of the conserved variables
        at fine cells with global (unwrapped) indices Gi of patch `key`.

        Coarse cell C = G // 2 with minmod slopes s_d of the neighbouring
        differences (ties take the first argument, U_{C+1} - U_C); the child at
        sub-offset sigma in {0,1}^d is U_C + sum_d (sigma_d ? +1 : -1) s_d / 4,
        dims in order. If any of the 2^d children of C has rho <= 0 or p <= 0,
        every child takes U_C. Returns (nv, ncells)."""
        l, c = key
        pc = [c[d] // 2 for d in range(3)]
        flatG = [Gi[d].ravel() for d in range(3)]
        ncell = flatG[0].size
        Gc = [flatG[d] // 2 for d in range(3)]
        sub = [flatG[d] - 2 * Gc[d] for d in range(3)]
        off = [Gc[d] // self.N - pc[d] if d < self.dim else np.zeros(ncell, dtype=np.int64)
               for d in range(3)]
        out = np.empty((self.nv, ncell))
        combos = set(zip(off[0].tolist(), off[1].tolist(), off[2].tolist()))
        for oc in combos:
            sel = (off[0] == oc[0]) & (off[1] == oc[1]) & (off[2] == oc[2])
            qc = self.mesh.wrap(l - 1, tuple(pc[d] + oc[d] for d in range(3)))
            qkey = (l - 1, qc)
            if qc is None or qkey not in U:
                raise OracleError('prolongation source missing: R2 violated at %r' % (key,))
            Q = U[qkey]
            Lc = [(Gc[d][sel] - (pc[d] + oc[d]) * self.N) if d < self.dim else np.zeros(sel.sum(), dtype=np.int64)
                  for d in range(3)]
            sg = [sub[d][sel] for d in range(3)]
            out[:, sel] = self._prolong_from(Q, Lc, sg)
        return out

    def _prolong_from(self, Q, Lc, sg):
        dim = self.dim

        def gather(shift_d, s):
            idx = []
            for d in (2, 1, 0):
                if d < dim:
                    idx.append(Lc[d] + G + (s if d == shift_d else 0))
                else:
                    idx.append(np.zeros_like(Lc[0]))
            return Q[:, idx[0], idx[1], idx[2]]

        UC = gather(-1, 0)
        slopes = []
        for d in range(dim):
            a = gather(d, 1) - UC
            b = UC - gather(d, -1)
            slopes.append(minmod(a, b))
        ok = np.ones(UC.shape[1], dtype=bool)
        chosen = np.empty_like(UC)
        for sig in itertools.product((0, 1), repeat=dim):
            sig = tuple(reversed(sig))          # x fastest; only the set matters
            v = UC
            for d in range(dim):
                if sig[d]:
                    v = v + 0.25 * slopes[d]
                else:
                    v = v - 0.25 * slopes[d]
            rho, u, p, T = euler.primitives(v, dim, self.gamma)
            ok &= (rho > 0.0) & (p > 0.0)
            m = np.ones(UC.shape[1], dtype=bool)
            for d in range(dim):
                m &= sg[d] == sig[d]
            chosen[:, m] = v[:, m]
        return np.where(ok[None, :], chosen, UC)

    def fill_interior_ghosts(self, U, key):
        """Same-level copy where the neighbour exists, else prolongation."""
        l, c = key
        A = U[key]
        for o in self.mesh.offsets():
            if self._outside(key, o):
                continue
            lo, hi = self._block(o)
            nk = (l, self.mesh.wrap(l, tuple(c[d] + o[d] for d in range(3))))
            if nk in U:
                slo = [lo[d] - o[d] * self.N for d in range(3)]
                shi = [hi[d] - o[d] * self.N for d in range(3)]
                A[self._slot_slice(lo, hi)] = U[nk][self._slot_slice(slo, shi)]
            else:
                if l == 0:
                    raise OracleError('missing level-0 neighbour')
                Gi, _ = self.cells(key, lo, hi)
                vals = self.prolong_cells(U, key, Gi)
                A[self._slot_slice(lo, hi)] = vals.reshape((self.nv,) + Gi[0].shape)

    def _dirichlet(self, kind, X, t):
        """Boundary states of the double Mach reflection (None where the rule is
        a reflection): left inflow and bottom x < 1/6 take the post-shock state;
        the top follows the exact shock x_s(t) = 1/6 + (1 + 20 t)/sqrt(3)."""
        pre, post = dmr_states(self.gamma)
        x = X[0]
        if kind == 'dmr_inflow':
            behind = np.ones(x.shape, dtype=bool)
            use = behind
        elif kind == 'dmr_bottom':
            behind = x < 1.0 / 6.0
            use = behind
        elif kind == 'dmr_top':
            behind = x < 1.0 / 6.0 + (1.0 + 20.0 * t) / math.sqrt(3.0)
            use = np.ones(x.shape, dtype=bool)
        else:
            raise OracleError(kind)
        st = [np.where(behind, post[j], pre[j]) for j in range(4)]
        Uc = euler.conserved_from_primitive(st[0], [st[1], st[2]], st[3], self.gamma)
        return np.stack(Uc), use

    def fill_physical(self, U, key, t):
        """Physical boundaries, one dimension after the other (x, y, z), each
        over the whole slot extent of the other dimensions: outflow copies the
        nearest interior layer, reflection mirrors ghost k <-> interior -1-k and
        negates the normal momentum, the double-Mach kinds set fixed states."""
        l, c = key
        A = U[key]
        ext = self.mesh.extent(l)
        N = self.N
        for d in range(self.dim):
            ax = 3 - d
            for side in (0, 1):
                kind = self.w['bc'][d][side]
                if kind == 'periodic':
                    continue
                if (side == 0 and c[d] != 0) or (side == 1 and c[d] != ext[d] - 1):
                    continue
                for k in range(G):
                    gl = -1 - k if side == 0 else N + k          # ghost local index
                    if kind == 'outflow':
                        src = 0 if side == 0 else N - 1
                        neg = False
                    else:
                        src = k if side == 0 else N - 1 - k      # mirror
                        neg = True
                    dst_sl = [slice(None)] * 4
                    src_sl = [slice(None)] * 4
                    dst_sl[ax] = gl + G
                    src_sl[ax] = src + G
                    vals = A[tuple(src_sl)].copy()
                    if neg:
                        vals[1 + d] = -vals[1 + d]
                    if kind in ('dmr_inflow', 'dmr_bottom', 'dmr_top'):
                        lo = [-G if e < self.dim else 0 for e in range(3)]
                        hi = [N + G if e < self.dim else 1 for e in range(3)]
                        lo[d], hi[d] = gl, gl + 1
                        _, X = self.cells(key, lo, hi)
                        X = [np.squeeze(X[e], axis=2 - d) for e in range(3)]
                        st, m = self._dirichlet(kind, X, t)
                        vals = np.where(m[None], st, vals)
                    A[tuple(dst_sl)] = vals

    def fill_ghosts(self, U, t):
        for l in range(self.L):
            keys = self.mesh.level_list(l)
            for k in keys:
                self.fill_interior_ghosts(U, k)
            for k in keys:
                self.fill_physical(U, k, t)

    # ---- one SSP-RK3 step ---------------------------------------------------
    def cfl_dt(self):
        """dt = CFL / max over leaf cells of sum_d (|u_d| + c) / dx_d (Sec. 3.1, Eq. 7:
        c sets the step size), clipped to t_end."""
        lam_max = 0.0
        for k in self.mesh.canonical():
            if not self.mesh.is_leaf(k):
                continue
            A = self.U[k][self.inner()]
            rho, u, p, T = euler.primitives(A, self.dim, self.gamma)
            if not (np.all(rho > 0.0) and np.all(p > 0.0)):
                raise OracleError('non-positive density or pressure')
            c = euler.sound_speed(p, rho, self.gamma)
            lam = None
            for d in range(self.dim):
                term = (np.abs(u[d]) + c) / self.dx[k[0]][d]
                lam = term if lam is None else lam + term
            lam_max = max(lam_max, float(np.max(lam)))
        if not math.isfinite(lam_max) or lam_max <= 0.0:
            raise OracleError('non-finite wave speed')
        dt = self.w['cfl'] / lam_max
        if self.w['t_end'] > 0.0:
            dt = min(dt, self.w['t_end'] - self.t)
        return dt

    def stage(self, s, dt, src, dst, U0, t_stage):
        """One SSP-RK3 stage over all patches of all levels."""
        self.fill_ghosts(src, t_stage)
        keys = self.mesh.canonical()
        inner = self.inner()
        faces = {}
        for k in keys:
            R, faces[k] = euler.patch_rhs(src[k], self.dim, self.N, G, self.dx[k[0]], self.gamma,
                                          self.w.get('flux', 'rusanov'), self.w.get('theta_switch', 0.05))
            Us = src[k][inner]
            if s == 0:
                new = Us + dt * R
            else:
                new = RK_A[s] * U0[k][inner] + RK_B[s] * (Us + dt * R)
            if k not in dst:
                dst[k] = np.zeros(self.slot_shape())
            dst[k][inner] = new
        self.reflux(dst, faces, RK_B[s], dt)
        self.restrict(dst)

    def step(self, dt=None):
        if dt is None or dt <= 0.0:
            dt = self.cfl_dt()
        t = self.t
        U0 = self.U
        U1, U2 = {}, {}
        self.stage(0, dt, U0, U1, U0, t)
        self.stage(1, dt, U1, U2, U0, t + dt)
        U3 = {}
        self.stage(2, dt, U2, U3, U0, t + 0.5 * dt)
        for k in U3:
            U0[k][self.inner()] = U3[k][self.inner()]
        self.t = t + dt
        self.steps += 1
        return dt

    # ---- reflux and restriction ---------------------------------------------
    def reflux(self, U, faces, b, dt):
        """At faces between a leaf patch and a same-level patch with children,
        the coarse flux F_c is replaced by the mean of the 2^(d-1) fine fluxes
        on that face (summed in lexicographic z, y, x order, times 2^-(d-1)).
        Applied to the stage result as U -/+ b dt (F_f - F_c) / dx (high/low
        face), per leaf patch in canonical order, faces x-, x+, y-, y+, z-, z+."""
        N = self.N
        for k in self.mesh.canonical():
            if not self.mesh.is_leaf(k):
                continue
            l, c = k
            A = U[k]
            for d in range(self.dim):
                ax = 3 - d
                for side in (0, 1):
                    o = [0, 0, 0]
                    o[d] = -1 if side == 0 else 1
                    bc_ = self.mesh.wrap(l, tuple(c[e] + o[e] for e in range(3)))
                    if bc_ is None:
                        continue
                    nb = (l, bc_)
                    if nb not in self.mesh.patches or self.mesh.is_leaf(nb):
                        continue
                    Fc = faces[k][d][side]
                    Ff = self._fine_face(faces, nb, d, side)
                    diff = (Ff - Fc) / self.dx[l][d]
                    sl = [slice(None)] + [slice(G, G + N) if e < self.dim else slice(None) for e in (2, 1, 0)]
                    sl[ax] = G if side == 0 else G + N - 1
                    sl = tuple(sl)
                    if side == 1:
                        A[sl] = A[sl] - b * (dt * diff)
                    else:
                        A[sl] = A[sl] + b * (dt * diff)

    def _fine_face(self, faces, nb, d, side):
        """Mean fine flux on the face of coarse patch `nb` seen from its neighbour
        at `side`, at coarse resolution: the children of nb on that face."""
        l, c = nb
        N = self.N
        fd = 2 * c[d] + (1 if side == 0 else 0)      # fine layer adjacent to the face
        fine_side = 1 if side == 0 else 0            # the children's face on that side
        tdims = [e for e in (2, 1, 0) if e != d]     # array axes order (z, y, x) minus d
        act = [e for e in tdims if e < self.dim]
        shape = [self.nv] + [2 * N if e < self.dim else 1 for e in tdims]
        full = np.empty(shape)
        for sub in itertools.product(*[(0, 1) for _ in act]):
            fc = [0, 0, 0]
            fc[d] = fd
            sl = [slice(None)]
            sd = dict(zip(act, sub))
            for e in range(3):
                if e != d:
                    fc[e] = 2 * c[e] + sd.get(e, 0) if e < self.dim else 0
            for e in tdims:
                if e < self.dim:
                    sl.append(slice(sd[e] * N, sd[e] * N + N))
                else:
                    sl.append(slice(None))
            full[tuple(sl)] = faces[(l + 1, tuple(fc))][d][fine_side]
        # 2^(d-1) fine faces per coarse face, lexicographic order, last axis fastest
        subs = list(itertools.product(*[(0, 1) for _ in act]))
        acc = None
        for sub in subs:
            sl = [slice(None)]
            sd = dict(zip(act, sub))
            for e in tdims:
                sl.append(slice(sd[e], None, 2) if e < self.dim else slice(None))
            v = full[tuple(sl)]
            acc = v if acc is None else acc + v
        return acc * (0.5 ** (self.dim - 1))

    def restrict(self, U):
        """Covered coarse cells take the mean of their 2^d children (sum in
        lexicographic z, y, x order, times 2^-d), finest level first."""
        N = self.N
        h = N // 2
        for l in range(self.L - 1, 0, -1):
            for k in self.mesh.level_list(l):
                pk = Mesh.parent(k)
                F = U[k][self.inner()]
                acc = None
                for sz in ((0, 1) if self.dim == 3 else (None,)):
                    for sy in ((0, 1) if self.dim >= 2 else (None,)):
                        for sx in (0, 1):
                            sl = [slice(None)]
                            for s_ in (sz, sy, sx):
                                sl.append(slice(None) if s_ is None else slice(s_, None, 2))
                            v = F[tuple(sl)]
                            acc = v if acc is None else acc + v
                val = acc * (0.5 ** self.dim)
                cs = [k[1][d] - 2 * pk[1][d] for d in range(3)]
                sl = [slice(None)]
                for d in (2, 1, 0):
                    sl.append(slice(G + cs[d] * h, G + cs[d] * h + h) if d < self.dim else slice(None))
                U[pk][tuple(sl)] = val

    # ---- refinement sensor and regrid -----------------------------------------
    def patch_flags(self, key):
        """Cell flags on the patch band [-2, N+1]^d (in-domain cells only): for
        phi in (rho, p) and each dimension, the relative jump
        s = |phi_+ - phi_-| / (phi_+ + 2 phi_0 + phi_-) exceeds theta, evaluated
        without the division as |phi_+ - phi_-| > theta (phi_+ + 2 phi_0 + phi_-)
        (the same test for positive rho and p). Requires filled ghosts."""
        A = self.U[key]
        rho, u, p, T = euler.primitives(A, self.dim, self.gamma)
        l, c = key
        ext = self.mesh.extent(l)
        N = self.N
        band = [slice(G - 2, G + N + 2) if d < self.dim else slice(None) for d in (2, 1, 0)]
        flag = None
        for phi, th in ((rho, self.w['theta_rho']), (p, self.w['theta_p'])):
            for d in range(self.dim):
                ax = 2 - d
                slm, sl0, slp = list(band), list(band), list(band)
                slm[ax] = slice(G - 3, G + N + 1)
                slp[ax] = slice(G - 1, G + N + 3)
                fm, f0, fp = phi[tuple(slm)], phi[tuple(sl0)], phi[tuple(slp)]
                f = np.abs(fp - fm) > th * (fp + 2.0 * f0 + fm)
                flag = f if flag is None else (flag | f)
        # in-domain mask
        mask = np.ones(flag.shape, dtype=bool)
        for d in range(self.dim):
            if self.periodic[d]:
                continue
            gidx = c[d] * N + np.arange(-2, N + 2)
            ok = (gidx >= 0) & (gidx < ext[d] * N)
            shp = [1, 1, 1]
            shp[2 - d] = N + 4
            mask &= ok.reshape(shp)
        return flag & mask

    def anyflag(self, key):
        """(refine, keep) flags of a leaf: refine requests refinement; keep
        blocks the coarsening of its parent. The plain sensor gives one flag
        for both; a learned flagger may return a pair (a hysteresis margin)."""
        if self.flag_override is not None:
            f = self.flag_override(self, key)
            return (bool(f[0]), bool(f[1])) if isinstance(f, tuple) else (bool(f), bool(f))
        f = bool(np.any(self.patch_flags(key)))
        return f, f

    def requests(self):
        """Refinement requests (leaves below the finest level with a flag) and
        coarsening candidates (patches whose children are unflagged leaves),
        from the current state. Fills ghosts first."""
        self.fill_ghosts(self.U, self.t)
        leaves = [k for k in self.mesh.canonical() if self.mesh.is_leaf(k)]
        af = {k: self.anyflag(k) for k in leaves}
        req = [k for k in leaves if k[0] < self.L - 1 and af[k][0]]
        cand = []
        for k in self.mesh.canonical():
            if self.mesh.is_leaf(k):
                continue
            ch = self.mesh.children(k)
            if all(self.mesh.is_leaf(x) for x in ch) and not any(af[x][1] for x in ch):
                cand.append(k)
        return req, cand, {k: v[0] for k, v in af.items()}

    def regrid(self, resample_ic=False):
        """Flag, close under R2 (Algorithm 1), coarsen (Sec. 4.3 rule), then fill
        new patches by prolongation from their parents (or the initial condition
        while the initial hierarchy is built)."""
        req, cand, _ = self.requests()
        created = self.mesh.refine(req)
        deleted = self.mesh.coarsen(cand, created)
        for k in deleted:
            del self.U[k]
        for k in sorted(created, key=canon):
            if resample_ic:
                self.U[k] = self.ic_fill(k)
            else:
                A = np.zeros(self.slot_shape())
                Gi, _ = self.cells(k, [0, 0, 0], [self.N] * 3)
                vals = self.prolong_cells(self.U, k, Gi)
                A[self.inner()] = vals.reshape((self.nv,) + Gi[0].shape)
                self.U[k] = A
        return created, deleted

    # ---- outputs ----------------------------------------------------------------
    def get_level(self, l):
        """Canonical patch list of level l: (coords (n, dim) int, interiors
        (n, nv, [N]*dim in z, y, x order))."""
        keys = self.mesh.level_list(l)
        coords = np.array([[k[1][d] for d in range(self.dim)] for k in keys], dtype=np.int64).reshape(-1, self.dim)
        shp = (self.nv,) + (self.N,) * self.dim
        data = np.stack([self.U[k][self.inner()].reshape(shp) for k in keys]) if keys \
            else np.zeros((0,) + shp)
        return coords, data

    def cons_sums(self):
        """sum over leaf cells of U times the cell volume, per variable."""
        tot = np.zeros(self.nv)
        for k in self.mesh.canonical():
            if not self.mesh.is_leaf(k):
                continue
            vol = 1.0
            for d in range(self.dim):
                vol *= self.dx[k[0]][d]
            A = self.U[k][self.inner()]
            tot += A.reshape(self.nv, -1).sum(axis=1) * vol
        return tot

    def leaf_field(self, var=0):
        """Composite field on the finest uniform grid (leaf values injected into
        all finest cells they cover); shape [n_z, n_y, n_x] of the finest level."""
        Lf = self.L - 1
        n = [self.w['base_cells'][d] * 2 ** Lf if d < self.dim else 1 for d in range(3)]
        out = np.full((n[2], n[1], n[0]), np.nan)
        for k in self.mesh.canonical():
            if not self.mesh.is_leaf(k):
                continue
            l, c = k
            r = 2 ** (Lf - l)
            A = self.U[k][self.inner()][var]
            for ax in range(3):
                if (2 - ax) < self.dim:
                    A = np.repeat(A, r, axis=ax)
            sl = []
            for d in (2, 1, 0):
                if d < self.dim:
                    sl.append(slice(c[d] * self.N * r, (c[d] + 1) * self.N * r))
                else:
                    sl.append(slice(None))
            out[tuple(sl)] = A
        return out
