"""Python binding of libamr (include/amr.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module
converts workload dicts to the C structs, passes PyTorch's caching allocator
and current CUDA stream to the library, and copies results into numpy
arrays. It never computes any part of the method itself, and it raises if
the compiled library is missing.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, '_lib', 'libamr.so')

OK = 0
ERRORS = {-1: 'AMR_ERR_ARG', -2: 'AMR_ERR_POOL', -3: 'AMR_ERR_CUDA', -4: 'AMR_ERR_NONFINITE',
          -5: 'AMR_ERR_TIMEOUT', -6: 'AMR_ERR_STATE', -7: 'AMR_ERR_MESH', -8: 'AMR_ERR_IO'}
BC = {'outflow': 0, 'reflect': 1, 'periodic': 2, 'dmr_inflow': 3, 'dmr_bottom': 4, 'dmr_top': 5}
IC = {'sod': 0, 'shu_osher': 1, 'riemann2d': 2, 'dmr': 3, 'blast3d': 4, 'implosion': 5,
      'density_wave': 6, 'constant': 7, 'shear_layer': 8}
FLAGGER = {'plain': 0, 'mlp': 1}
MODE = {'batched': 0, 'per_patch': 1}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Domain(C.Structure):
    _fields_ = [('dim', C.c_int), ('lo', C.c_double * 3), ('hi', C.c_double * 3),
                ('bc_lo', C.c_int * 3), ('bc_hi', C.c_int * 3)]


class Options(C.Structure):
    _fields_ = [('precision', C.c_int), ('cfl', C.c_double), ('t_end', C.c_double),
                ('flagger', C.c_int), ('theta_rho', C.c_double), ('theta_p', C.c_double),
                ('max_patches', C.c_int), ('seed', C.c_uint64), ('amp', C.c_double),
                ('mode', C.c_int), ('use_graph', C.c_int),
                ('dev_alloc', ALLOC_FN), ('dev_free', FREE_FN), ('user', C.c_void_p),
                ('stream', C.c_void_p), ('mlp_weights', C.c_void_p), ('mlp_n_weights', C.c_long),
                ('autotune', C.c_int), ('flux', C.c_int),
                ('mlp_keep_margin', C.c_double), ('theta_switch', C.c_double), ('mlp_refine_margin', C.c_double)]

FLUX = {'rusanov': 0, 'hllc': 1, 'central': 2, 'hybrid': 3}

TUNE_NAMES = ('ghost_ctas_per_sm', 'ghost_cells_per_item', 'rhs_ctas_per_sm', 'reflux_ctas_per_sm',
              'restrict_ctas_per_sm', 'cfl_ctas_per_sm', 'flag_ctas_per_sm', 'rhs_tile_shape')


class AMRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (ERRORS.get(code, code), msg))
        self.code = code


_lib = None

# (name, restype, argtypes) of every exported entry point of include/amr.h
SIGNATURES = [
    ('amr_default_options', None, [C.POINTER(Options)]),
    ('amr_init', C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Domain), C.c_double, C.POINTER(C.c_int),
                           C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(Options)]),
    ('amr_step', C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    ('amr_regrid', C.c_int, [C.c_void_p]),
    ('amr_advance', C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ('amr_get_level', C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p]),
    ('amr_get_diag', C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    ('amr_set_state', C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]),
    ('amr_get_requests', C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.POINTER(C.c_int),
                                   C.c_void_p]),
    ('amr_mesh_close', C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                 C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p,
                                 C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ('amr_mesh_tables', C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_longlong)]),
    ('amr_checkpoint', C.c_int, [C.c_void_p, C.c_char_p]),
    ('amr_restore', C.c_int, [C.c_void_p, C.c_char_p]),
    ('amr_set_mlp', C.c_int, [C.c_void_p, C.c_void_p, C.c_long]),
    ('amr_flag_stats', C.c_int, [C.c_void_p, C.c_void_p]),
    ('amr_plain_requests', C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ('amr_harvest', C.c_int, [C.c_void_p, C.POINTER(C.c_long), C.c_void_p, C.c_void_p]),
    ('amr_get_counters', C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_longlong)]),
    ('amr_set_timing', C.c_int, [C.c_void_p, C.c_int]),
    ('amr_autotune', C.c_int, [C.c_void_p]),
    ('amr_get_tuning', C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ('amr_set_tuning', C.c_int, [C.c_void_p, C.c_void_p]),
    ('amr_get_timing', C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ('amr_destroy', None, [C.c_void_p]),
    ('amr_last_error', C.c_char_p, [C.c_void_p]),
    ('amr_mlp_k', C.c_int, [C.c_int]),
    ('amr_mlp_features', C.c_int, [C.c_int, C.c_double, C.c_void_p, C.c_long, C.c_void_p,
                                   C.POINTER(Options)]),
    ('amr_mlp_infer', C.c_int, [C.c_int, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p,
                                C.POINTER(Options)]),
    ('amr_mlp_grad', C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_long, C.c_float, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.POINTER(Options)]),
    ('amr_mlp_train', C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_long, C.c_float, C.c_int, C.c_int,
                                C.c_float, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(Options)]),
    ('amr_mlp_grad_noalloc', C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_long, C.c_float, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
]


def load():
    """Load libamr.so (built by paper_2508_05020_gb300.build). Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError('libamr.so is not built (%s); run paper_2508_05020_gb300.build.build()' % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _TorchMemory:
    """Device allocator hooks backed by PyTorch's caching allocator."""

    def __init__(self, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.device = torch.cuda.current_device()
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:      # out of memory -> the library reports AMR_ERR_CUDA
            return None

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


def make_options(precision=64, cfl=0.5, t_end=0.0, flagger='plain', theta_rho=0.05, theta_p=0.05,
                 max_patches=0, seed=0, amp=0.01, mode='batched', use_graph=True, torch_memory=True,
                 autotune=False, flux='rusanov', mlp_keep_margin=0.0, theta_switch=0.05, mlp_refine_margin=0.0):
    """Options struct plus the objects that must outlive it."""
    lib = load()
    o = Options()
    lib.amr_default_options(C.byref(o))
    o.precision = precision
    o.cfl = cfl
    o.t_end = t_end
    o.flagger = FLAGGER[flagger]
    o.theta_rho = theta_rho
    o.theta_p = theta_p
    o.max_patches = max_patches
    o.seed = seed
    o.amp = amp
    o.mode = MODE[mode]
    o.use_graph = 1 if use_graph else 0
    o.autotune = 1 if autotune else 0
    o.flux = FLUX[flux]
    o.mlp_keep_margin = mlp_keep_margin
    o.theta_switch = theta_switch
    o.mlp_refine_margin = mlp_refine_margin
    keep = []
    if torch_memory:
        import torch
        stream = torch.cuda.Stream()        # the library's own (capturable) stream
        mem = _TorchMemory(stream)
        o.dev_alloc = mem.alloc
        o.dev_free = mem.free
        o.stream = C.c_void_p(stream.cuda_stream)
        keep += [mem, stream]
    return o, keep


class AMR:
    """One hierarchy on the current CUDA device (see include/amr.h)."""

    def __init__(self, w, precision=64, flagger='plain', mode='batched', use_graph=True,
                 max_patches=0, torch_memory=True, mlp_weights=None, autotune=False, mlp_keep_margin=0.0,
                 mlp_refine_margin=0.0):
        self.lib = load()
        self.w = dict(w)
        self.dim = w['dim']
        self.N = w['patch']
        self.L = w['levels']
        self.nv = self.dim + 2
        dom = Domain()
        dom.dim = self.dim
        for d in range(3):
            dom.lo[d] = w['lo'][d]
            dom.hi[d] = w['hi'][d]
            dom.bc_lo[d] = BC[w['bc'][d][0]]
            dom.bc_hi[d] = BC[w['bc'][d][1]]
        self.opt, self._keep = make_options(precision, w['cfl'], w['t_end'], flagger, w['theta_rho'],
                                            w['theta_p'], max_patches, w.get('seed', 0), w.get('amp', 0.01),
                                            mode, use_graph, torch_memory, autotune, w.get('flux', 'rusanov'),
                                            mlp_keep_margin, w.get('theta_switch', 0.05), mlp_refine_margin)
        if mlp_weights is not None:
            self._w_host = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            self.opt.mlp_weights = _ptr(self._w_host)
            self.opt.mlp_n_weights = self._w_host.size
        base = (C.c_int * 3)(*w['base_cells'])
        ctx = C.c_void_p()
        rc = self.lib.amr_init(C.byref(ctx), C.byref(dom), w['gamma'], base, self.L, 2, self.N,
                               IC[w['ic']], C.byref(self.opt))
        self.ctx = ctx
        if rc != OK:
            msg = self.lib.amr_last_error(ctx).decode() if ctx else ''
            if ctx:
                self.lib.amr_destroy(ctx)
                self.ctx = None
            raise AMRError(rc, msg)

    def _check(self, rc):
        if rc != OK:
            raise AMRError(rc, self.lib.amr_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, 'ctx', None):
            self.lib.amr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt=0.0, sync=True):
        """One SSP-RK3 step; dt <= 0 takes the CFL step. Returns dt (sync=True)."""
        out = C.c_double()
        self._check(self.lib.amr_step(self.ctx, float(dt), C.byref(out) if sync else None))
        return out.value if sync else None

    def regrid(self):
        self._check(self.lib.amr_regrid(self.ctx))

    def advance(self, n_steps, regrid=True):
        """n_steps CFL steps (amr_advance). regrid: True (after every step),
        False (never) or the regrid interval K (after every K-th step)."""
        k = (1 if regrid else 0) if isinstance(regrid, bool) else int(regrid)
        self._check(self.lib.amr_advance(self.ctx, int(n_steps), k))

    def get_level(self, level, data=True, out=None):
        """Patch coordinates and interiors of a level (amr_get_level). `out`: a
        C-contiguous float64 array of the right shape to receive the
        interiors (for instance in pinned host memory)."""
        n = C.c_int()
        self._check(self.lib.amr_get_level(self.ctx, level, C.byref(n), None, None))
        coords = np.zeros((n.value, self.dim), dtype=np.int32)
        shape = (n.value, self.nv) + (self.N,) * self.dim
        if out is not None:
            if out.shape != shape or out.dtype != np.float64 or not out.flags['C_CONTIGUOUS']:
                raise ValueError('out must be a C-contiguous float64 array of shape %s' % (shape,))
            arr = out
        else:
            arr = np.zeros(shape) if data else None
        if n.value:
            self._check(self.lib.amr_get_level(self.ctx, level, C.byref(n), _ptr(coords), _ptr(arr)))
        return coords.astype(np.int64), arr

    def diag(self):
        t = C.c_double()
        cons = np.zeros(5)
        ppl = np.zeros(8, dtype=np.int32)
        self._check(self.lib.amr_get_diag(self.ctx, C.byref(t), _ptr(cons), _ptr(ppl)))
        return t.value, cons[:self.nv].copy(), ppl[:self.L].copy()

    def set_state(self, levels, coords, data, t=0.0):
        levels = np.ascontiguousarray(levels, dtype=np.int32)
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        data = np.ascontiguousarray(data, dtype=np.float64)
        self._check(self.lib.amr_set_state(self.ctx, len(levels), _ptr(levels), _ptr(coords), _ptr(data),
                                           float(t)))

    def requests(self):
        nr, nc = C.c_int(), C.c_int()
        self._check(self.lib.amr_get_requests(self.ctx, C.byref(nr), None, C.byref(nc), None))
        r = np.zeros((nr.value, 4), dtype=np.int32)
        c = np.zeros((nc.value, 4), dtype=np.int32)
        self._check(self.lib.amr_get_requests(self.ctx, C.byref(nr), _ptr(r), C.byref(nc), _ptr(c)))
        return r, c

    def checkpoint(self, path):
        """Write the hierarchy, state and time to a file (amr_checkpoint)."""
        self._check(self.lib.amr_checkpoint(self.ctx, os.fsencode(path)))

    def restore(self, path):
        """Replace the hierarchy, state and time by a checkpoint's (amr_restore)."""
        self._check(self.lib.amr_restore(self.ctx, os.fsencode(path)))

    def set_mlp(self, weights):
        wv = np.ascontiguousarray(weights, dtype=np.float32)
        self._check(self.lib.amr_set_mlp(self.ctx, _ptr(wv), wv.size))

    def plain_requests(self):
        """Refinement requests of the plain sensor on the current hierarchy
        (amr_plain_requests): the unmet requests of a learned or infrequent
        regrid."""
        n = C.c_int()
        self._check(self.lib.amr_plain_requests(self.ctx, C.byref(n)))
        return n.value

    def flag_stats(self):
        out = np.zeros(4, dtype=np.int64)
        self._check(self.lib.amr_flag_stats(self.ctx, _ptr(out)))
        return out

    def harvest(self):
        n = C.c_long()
        self._check(self.lib.amr_harvest(self.ctx, C.byref(n), None, None))
        smp = np.zeros((n.value, 5, 3))
        lab = np.zeros(n.value, dtype=np.uint8)
        self._check(self.lib.amr_harvest(self.ctx, C.byref(n), _ptr(smp), _ptr(lab)))
        return smp[:n.value], lab[:n.value]

    def counters(self):
        a, b, k = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self._check(self.lib.amr_get_counters(self.ctx, C.byref(a), C.byref(b), C.byref(k)))
        return a.value, b.value, k.value

    def autotune(self):
        self._check(self.lib.amr_autotune(self.ctx))

    def tuning(self):
        """Launch parameters in use and the autotuner's best times (ms), by TUNE_NAMES."""
        p = np.zeros(len(TUNE_NAMES), dtype=np.int32)
        ms = np.zeros(len(TUNE_NAMES), dtype=np.float32)
        self._check(self.lib.amr_get_tuning(self.ctx, _ptr(p), _ptr(ms)))
        return dict(zip(TUNE_NAMES, p.tolist())), dict(zip(TUNE_NAMES, ms.tolist()))

    def set_tuning(self, params):
        """Set the launch parameters (a dict by TUNE_NAMES, as tuning() returns
        them; missing names keep their value) (amr_set_tuning)."""
        cur, _ = self.tuning()
        cur.update(params)
        p = np.array([cur[k] for k in TUNE_NAMES], dtype=np.int32)
        self._check(self.lib.amr_set_tuning(self.ctx, _ptr(p)))

    def set_timing(self, enable=True):
        self._check(self.lib.amr_set_timing(self.ctx, 1 if enable else 0))

    TIMING_SLOTS = ('ghost', 'rhs', 'reflux', 'restrict', 'cfl', 'flag', 'closure', 'upload_fill',
                    'regrid_ghost', 'flag_phase_wall')

    def timing(self):
        """Milliseconds of the last step (slots 0-4) and regrid (5-9), named by
        TIMING_SLOTS, and the kernel launches behind each slot."""
        ms = np.zeros(len(self.TIMING_SLOTS))
        n = np.zeros(len(self.TIMING_SLOTS), dtype=np.int32)
        self._check(self.lib.amr_get_timing(self.ctx, _ptr(ms), _ptr(n)))
        return ms, n

    def patch_keys(self):
        """Canonical (level, x, y, z) keys of every patch."""
        out = []
        for l in range(self.L):
            coords, _ = self.get_level(l, data=False)
            for c in coords:
                cc = list(c) + [0] * (3 - self.dim)
                out.append((l, tuple(cc)))
        return out


# ---------------------------------------------------------------------------
# host-only mesh planning
# ---------------------------------------------------------------------------
def _key_rows(keys):
    a = np.ascontiguousarray(np.asarray(keys, dtype=np.int32).reshape(-1, 4))
    return a, a.shape[0]


def mesh_close(dim, base_patches, periodic, max_level, keys, refine=(), candidates=()):
    """The mesh half of a regrid on the host (amr_mesh_close): Algorithm 1 on
    the refinement requests, then the coarsening rule on the candidates.
    keys, refine, candidates: rows (level, cx, cy, cz). Returns (hierarchy as
    an (n, 4) int32 array in canonical order, patches created, deleted)."""
    lib = load()
    bp = np.array([int(base_patches[d]) if d < len(base_patches) else 1 for d in range(3)], dtype=np.int32)
    per = np.array([1 if d < len(periodic) and periodic[d] else 0 for d in range(3)], dtype=np.int32)
    k, n = _key_rows(keys)
    r, nr = _key_rows(refine)
    cnd, nc = _key_rows(candidates)
    n_out, n_cr, n_del = C.c_int(0), C.c_int(0), C.c_int(0)
    cap = max(n, 1) * 2
    while True:
        out = np.zeros((cap, 4), dtype=np.int32)
        rc = lib.amr_mesh_close(dim, _ptr(bp), _ptr(per), max_level, n, _ptr(k), nr, _ptr(r), nc, _ptr(cnd), cap,
                                C.byref(n_out), _ptr(out), C.byref(n_cr), C.byref(n_del))
        if rc == -2 and n_out.value > cap:                  # AMR_ERR_POOL: room for the result
            cap = n_out.value
            continue
        _check_free(rc, 'amr_mesh_close')
        return out[:n_out.value], n_cr.value, n_del.value


def mesh_tables(dim, base_patches, periodic, max_level, keys):
    """The metadata tables of a hierarchy (amr_mesh_tables; slot = canonical
    index), split into a dict of named int32 arrays by the layout of
    include/amr.h."""
    lib = load()
    bp = np.array([int(base_patches[d]) if d < len(base_patches) else 1 for d in range(3)], dtype=np.int32)
    per = np.array([1 if d < len(periodic) and periodic[d] else 0 for d in range(3)], dtype=np.int32)
    k, n = _key_rows(keys)
    size = C.c_longlong(0)
    _check_free(lib.amr_mesh_tables(dim, _ptr(bp), _ptr(per), max_level, n, _ptr(k), None, C.byref(size)),
                'amr_mesh_tables')
    out = np.zeros(size.value, dtype=np.int32)
    _check_free(lib.amr_mesh_tables(dim, _ptr(bp), _ptr(per), max_level, n, _ptr(k), _ptr(out), C.byref(size)),
                'amr_mesh_tables')
    parts, o = {}, 0
    for name, width in (('level', n), ('coord', 3 * n), ('nbr', 27 * n), ('parent', n), ('child', 8 * n),
                        ('pflag', n), ('all_list', n), ('level_off', 9), ('leaf_list', n), ('counts', 4),
                        ('reflux_list', n), ('reflux_fine', 24 * n), ('new_list', n)):
        parts[name] = out[o:o + width]
        o += width
    assert o == out.size
    return parts


# ---------------------------------------------------------------------------
# standalone learned-indicator calls
# ---------------------------------------------------------------------------
def _check_free(rc, what):
    if rc != OK:
        raise AMRError(rc, what)


def mlp_k(dim):
    return load().amr_mlp_k(dim)


def mlp_features(dim, gamma, samples):
    lib = load()
    samples = np.ascontiguousarray(samples, dtype=np.float64)
    n = samples.shape[0]
    X = np.zeros((n * 2 * dim, mlp_k(dim)), dtype=np.float32)
    o, keep = make_options()
    _check_free(lib.amr_mlp_features(dim, gamma, _ptr(samples), n, _ptr(X), C.byref(o)), 'amr_mlp_features')
    return X


def mlp_infer(dim, X, weights):
    lib = load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    z = np.zeros(X.shape[0], dtype=np.float32)
    o, keep = make_options()
    _check_free(lib.amr_mlp_infer(dim, _ptr(X), X.shape[0], _ptr(w), _ptr(z), C.byref(o)), 'amr_mlp_infer')
    return z


def mlp_grad(dim, X, y, pos_weight, weights):
    lib = load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    g = np.zeros_like(w)
    loss = np.zeros(1, dtype=np.float32)
    o, keep = make_options()
    _check_free(lib.amr_mlp_grad(dim, _ptr(X), _ptr(y), X.shape[0], float(pos_weight), _ptr(w), _ptr(g),
                                 _ptr(loss), C.byref(o)), 'amr_mlp_grad')
    return float(loss[0]), g


def mlp_train(dim, X, y, pos_weight, weights, epochs, batch, lr, seed=1):
    lib = load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = np.array(weights, dtype=np.float32, copy=True)
    hist = np.zeros(epochs, dtype=np.float32)
    o, keep = make_options()
    _check_free(lib.amr_mlp_train(dim, _ptr(X), _ptr(y), X.shape[0], float(pos_weight), epochs, batch,
                                  float(lr), seed, _ptr(w), _ptr(hist), C.byref(o)), 'amr_mlp_train')
    return w, hist
