#!/usr/bin/env python
"""Throughput benchmark of the AMR Euler hot path on GB300.

A step is one pass of the whole hot path over the hierarchy: CFL reduction,
three SSP-RK3 stages (ghost fill, fused WENO5/Rusanov RHS + stage update,
reflux, restriction) over every leaf patch of every level, and a regrid
(flagging, closure, new patches) after every K-th step. The default workload
is the 3D blast problem (128^3 base cells, 3 levels, 16^3 patches, FP32
fields, t_end = 0.05; its inputs exceed L2). The metric is fine-equivalent
cell-updates per second: (base cells x 2^(d (L-1))) x steps / seconds; the
leaf cell-updates per second (cells actually advanced) are reported beside it.

The blast's refined region grows as it expands (about 1.4 k leaf patches at
t = 0, 8 k at t_end), so the run goes from t = 0 to t_end in one context:
three windows of exactly K steps (after W warm-up steps each) are timed at
t = 0, at t_end / 2 and just before t_end, the one at t_end / 2 giving the
headline `value`, and the whole run's device time gives the whole-run rate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank advances its own replica (no collective on the
data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import workload  # noqa: E402
from synth.workloads import fine_equivalent_cells  # noqa: E402

METRIC = 'fine-equiv cell-updates/s per GB300, batched FP32+learned vs plain FP64, at stated L1(rho)'
UNIT = 'cell-updates/s'
PEAKS_FILE = os.path.join(ROOT, 'MEASURED_PEAKS.json')
FLOPS_FILE = os.path.join(ROOT, 'oracle', 'flop_counts.json')
WEIGHTS_DIR = os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights')

# DRAM bytes of one stage-1 k_rhs launch per RHS tile shape (ncu,
# dram__bytes_read.sum + dram__bytes_write.sum; None: not captured) on the
# default workload at t_end / 2 (4656 leaf
# patches, the state a checkpoint of the default run holds at the start of its
# headline window), valid while the sources of the kernel (the regions below:
# EOS, WENO5, face fluxes, the kernel and its launch) hash as recorded. Leaves
# are independent work items, so a launch over another hierarchy of the same
# workload moves this figure per leaf times its leaves.
RHS_TRAFFIC = {'bytes': {0: 1132389888 + 414993152, 2: 969363200 + 412371456, 3: 1134521856 + 417061376,
                         4: 962697984 + 413609984}, 'leaves': 4656, 'workload': 'blast3d', 'base': 128, 'levels': 3,
               'regions': [('paper_2508_05020_gb300/csrc/amr_kernels.cuh', 'template <typename T> struct Num;',
                            '// Metadata of one patch staged'),
                           ('paper_2508_05020_gb300/csrc/amr_kernels.cuh', '// K4: fused right-hand side',
                            '// K5: coarse-fine flux correction'),
                           ('paper_2508_05020_gb300/csrc/amr_launch.cuh', 'template <typename T, int D, int N, int V = 0> struct RhsCfg',
                            'template <typename T>\ncudaError_t Kernels<T>::prepare')],
               'hash': '2e0f7a645a629b19'}


def rhs_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f, a, b in RHS_TRAFFIC['regions']:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        i = text.index(a)
        h.update(text[i:text.index(b, i)].encode())
    return h.hexdigest()[:16]


def rhs_traffic(workload_name, base, levels, leaves=None, shape=0):
    """DRAM bytes of one stage-1 RHS launch of tile shape `shape` over `leaves`
    leaf patches (the captured launch's own count if None), or None when no
    capture applies."""
    if workload_name != RHS_TRAFFIC['workload'] or base not in (0, RHS_TRAFFIC['base']) or \
            levels not in (0, RHS_TRAFFIC['levels']):
        return None
    try:
        if rhs_source_hash() != RHS_TRAFFIC['hash']:
            return None
    except ValueError:
        return None
    b = RHS_TRAFFIC['bytes'].get(shape)
    if b is None:
        return None
    if leaves is None:
        return b
    return int(round(b * leaves / RHS_TRAFFIC['leaves']))


def parse_tuning(text):
    """`name=value[,name=value]` (launch parameter names of amr.TUNE_NAMES,
    integer values) as a dict; ValueError on a malformed item."""
    out = {}
    for item in text.split(','):
        item = item.strip()
        if not item:
            continue
        name, sep, value = item.partition('=')
        if not sep or not name.strip():
            raise ValueError('launch parameter %r is not name=value' % item)
        out[name.strip()] = int(value)
    return out


def load_json(path, default):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return default


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    QUERY = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
             'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
             'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', self.gpu, '--query-gpu=' + self.QUERY,
                                          '--format=csv,noheader,nounits', '-lms', '50'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(',')]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace('.', '').isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == 'active'})
        sm_sorted = sorted(sm)
        return {'sm_mhz': sm_sorted[len(sm_sorted) // 2] if sm else None,
                'sm_max_mhz': max(mx) if mx else None, 'reasons': reasons, 'samples': len(sm)}


# ----------------------------------------------------------------------------- hierarchy counts
def leaf_patches(w, ppl):
    """Leaves of a hierarchy with ppl patches per level: every patch above
    the base level has 2^d - 1 siblings and one parent, which is not a leaf."""
    ppl = [int(x) for x in ppl[:w['levels']]]
    return sum(ppl) - sum(ppl[1:]) // (2 ** w['dim'])


def cell_counts(w, ppl):
    """Cells one step updates: the leaf patches (a patch with children is
    restricted from them, not updated), all patches (whose ghosts are
    filled), and the fine-equivalent count."""
    n = w['patch'] ** w['dim']
    leaves = leaf_patches(w, ppl) * n
    return {'leaf_cells': leaves, 'all_patch_cells': int(sum(ppl)) * n,
            'fine_equivalent': int(fine_equivalent_cells(w)), 'stage_updates_per_step': 3 * leaves}


def rhs_flops_per_launch(amr, w, flops):
    """Algorithmic FLOPs of one fused RHS launch: faces x FLOP/face + cells x
    FLOP/cell (central: N + 3 face fluxes and N + 1 conservative face values
    per row); None for a flux without a count (HLLC)."""
    d = w['dim']
    N = w['patch']
    _, _, ppl = amr.diag()
    n_patch = leaf_patches(w, ppl)                 # the kernel updates leaves only
    rows = n_patch * d * N ** (d - 1)
    cells = n_patch * N ** d
    f = flops[str(d)]
    flux = w.get('flux', 'rusanov')
    if flux == 'central':
        return rows * ((N + 3) * f['face_central'] + (N + 1) * f['face_combine_central']) + cells * f['cell']
    if flux != 'rusanov':
        return None
    return rows * (N + 1) * f['face'] + cells * f['cell']


# ----------------------------------------------------------------------------- CPU oracle
def _oracle_ppl(o):
    ppl = [0] * o.L
    for l, _ in o.mesh.patches:
        ppl[l] += 1
    return ppl


def oracle_sample(steps, base=32):
    """The FP64 CPU oracle, as it stands, on the same problem at base^3 cells
    on one core: (fine-equivalent cell-updates/s, leaf cell-updates/s,
    seconds, description)."""
    from oracle.amr import Oracle
    w = workload('blast3d', base_cells=(base, base, base))
    o = Oracle(w)
    leaves = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        leaves += leaf_patches(w, _oracle_ppl(o)) * w['patch'] ** 3
        o.step()
        o.regrid()
    dt = time.perf_counter() - t0
    fe = fine_equivalent_cells(w)
    desc = ('oracle (numpy FP64) on the same 3D blast problem at %d^3 base cells, 3 levels, 16^3 patches, '
            'plain flags: %d step(s) of step + regrid from t = 0' % (base, steps))
    return fe * steps / dt, leaves / dt, dt, desc


def _oracle_worker(base, steps, barrier, q):
    """One replica of the oracle sample (all-core timing): initialise, report
    ready, then for each step wait for the common start and time one step +
    regrid of its own run."""
    sys.path.insert(0, ROOT)
    from oracle.amr import Oracle
    w = workload('blast3d', base_cells=(base, base, base))
    o = Oracle(w)
    q.put(('ready', 0.0, 0))
    for _ in range(steps):
        barrier.wait()
        leaves = leaf_patches(w, _oracle_ppl(o)) * w['patch'] ** 3
        t0 = time.perf_counter()
        o.step()
        o.regrid()
        q.put(('done', time.perf_counter() - t0, leaves))


def oracle_all_cores(base=32, steps=1, procs=None):
    """The oracle on every host core: one independent replica of the sample
    per core (spawned processes, one thread each), each step started on all
    of them together. Returns per step (fine-equivalent cell-updates/s, leaf
    cell-updates/s, seconds) and the number of cores."""
    import multiprocessing as mp
    n = procs or host_cores()
    ctx = mp.get_context('spawn')
    barrier = ctx.Barrier(n + 1)
    q = ctx.Queue()
    env_keep = {k: os.environ.get(k) for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS')}
    for k in env_keep:
        os.environ[k] = '1'
    ps = [ctx.Process(target=_oracle_worker, args=(base, steps, barrier, q)) for _ in range(n)]
    for p in ps:
        p.start()
    for k, v in env_keep.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    for _ in ps:
        q.get(timeout=1200)
    fe = fine_equivalent_cells(workload('blast3d', base_cells=(base, base, base)))
    out = []
    for _ in range(steps):
        barrier.wait()
        res = [q.get(timeout=1200) for _ in ps]
        wall = max(r[1] for r in res)
        out.append((n * fe / wall, sum(r[2] for r in res) / wall, wall))
    for p in ps:
        p.join(timeout=60)
    return out, n


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands on every host core (one
    replica per core), each timed step one step + regrid of the 3D blast at
    16^3 base cells (about a second of CPU work per replica)."""
    if rank != 0:
        return 0
    base = 16
    res, cores = oracle_all_cores(base, steps=args.warmup + args.steps)
    per_step = [r[2] for r in res[args.warmup:]]
    leaf_rates = [r[1] for r in res[args.warmup:]]
    w = workload('blast3d', base_cells=(base, base, base))
    fe = fine_equivalent_cells(w) * cores
    total = sum(per_step)
    val = fe * len(per_step) / total if per_step else 0.0
    desc = ('the FP64 CPU oracle (numpy), as it stands, plain flags, on the 3D blast at %d^3 base cells, 3 levels, '
            '16^3 patches: %d independent replicas, one per host core, each timed step one step + regrid from t = 0'
            % (base, cores))
    line = {'impl': 'reference', 'metric': METRIC, 'value': val, 'unit': UNIT, 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': 1000.0 * total / len(per_step) if per_step else 0.0,
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic',
            'config': {'workload': 'blast3d base 16x16x16, 3 levels, 16^3 patches, FP64, plain flags, rusanov flux, '
                                   'CPU oracle x %d replicas' % cores,
                       'sample_of': 'blast3d base 128x128x128, 3 levels, 16^3 patches (the GPU arm\'s workload)',
                       'leaf_cell_updates_per_s': sum(leaf_rates) / len(leaf_rates) if leaf_rates else 0.0},
            'cpu_baseline': {'value': val, 'unit': UNIT, 'cores': cores, 'kind': 'oracle', 'sample': desc},
            'e2e': {'value': val, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ranks
def combine_ranks(elapsed, units, dist=None, device='cpu'):
    """Whole-job timing over ranks: (max elapsed, total units). Each rank runs its
    own replica, so the only exchange is this scalar reduction after the timed
    region (gloo on CPU in tests, NCCL under torchrun on GPUs)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed, units
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- GPU run to t_end
def plan_chunk(remaining_t, dt_est, cap):
    """Steps to issue next when `remaining_t` of simulated time is left at an
    estimated step dt_est: at most `cap`, one at a time near the end (the last
    step is clipped to t_end, so no step is spent after it)."""
    if remaining_t <= 0.0:
        return 0
    est = remaining_t / dt_est if dt_est > 0 else 1.0
    if est <= 3.0:
        return 1
    return max(1, min(cap, int(est) - 2))


class Run:
    """One context advanced to t_end in event-timed segments of amr_advance;
    every step of the run lies in exactly one segment, so the segments' device
    time is the run's."""

    def __init__(self, amr, w, regrid_every, sample_every=0):
        import torch
        self.torch = torch
        self.amr = amr
        self.w = w
        self.K = regrid_every
        self.sample_every = sample_every
        self.stream = amr._keep[1]
        self.ms = 0.0
        self.steps = 0
        self.leaf_steps = 0               # leaf patches x steps (at the start of each segment)
        self.unmet = []
        self.t_end = w['t_end']
        self.t, self.dt_est = 0.0, 0.0
        self._refresh()

    def _refresh(self):
        t, _, ppl = self.amr.diag()
        self.leaves = leaf_patches(self.w, ppl)
        self.ppl = [int(x) for x in ppl]
        return t

    def seg(self, n):
        torch = self.torch
        if n <= 0:
            return 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = self.t
        leaves0 = self.leaves
        e0.record(self.stream)
        self.amr.advance(n, regrid=self.K)
        e1.record(self.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        self.ms += ms
        self.steps += n
        self.t = self._refresh()
        self.leaf_steps += n * 0.5 * (leaves0 + self.leaves)
        if self.t > t0:
            self.dt_est = (self.t - t0) / n
        return ms

    def done(self):
        return self.t >= self.t_end * (1.0 - 1e-12)

    def advance_to(self, target, cap=100):
        """Advance until t >= target (t_end at most), sampling the unmet plain
        requests every `sample_every` steps when asked."""
        target = min(target, self.t_end)
        while self.t < target * (1.0 - 1e-12) and not self.done():
            if self.dt_est <= 0.0:
                n = 1
            else:
                n = plan_chunk(target - self.t, self.dt_est, self.sample_every or cap) if target >= self.t_end \
                    else max(1, min(self.sample_every or cap, int(math.ceil((target - self.t) / self.dt_est))))
            self.seg(n)
            if self.sample_every and not self.done():
                self.unmet.append(self.amr.plain_requests())

    def advance_until_left(self, n_left):
        """Advance until about n_left steps remain before t_end (the step dt
        drifts, so the estimate is renewed after every chunk)."""
        while not self.done():
            extra = self.steps_left() - n_left
            if extra < 1.0:
                break
            self.seg(max(1, min(self.sample_every or 100, int(extra))))
            if self.sample_every and not self.done():
                self.unmet.append(self.amr.plain_requests())

    def steps_left(self):
        return (self.t_end - self.t) / self.dt_est if self.dt_est > 0 else float('inf')

    def summary(self, fe, N):
        s = self.ms / 1000.0
        cells = N ** self.w['dim']
        out = {'steps': self.steps, 't': self.t, 'device_s': s,
               'fine_equivalent_cell_updates_per_s': fe * self.steps / s if s > 0 else None,
               'leaf_cell_updates_per_s': self.leaf_steps * cells / s if s > 0 else None,
               'mean_ms_per_step': self.ms / max(self.steps, 1),
               'patches_per_level_end': self.ppl, 'leaf_patches_end': self.leaves}
        if self.unmet:
            out['unmet_plain_requests_per_step'] = float(sum(self.unmet) / len(self.unmet))
            out['unmet_plain_requests_max'] = int(max(self.unmet))
            out['unmet_samples'] = len(self.unmet)
        return out


def make_amr(AMR, w, args, flagger, weights, precision=32, mode='batched'):
    return AMR(w, precision=precision, flagger=flagger, mlp_weights=weights if flagger == 'mlp' else None,
               max_patches=args.max_patches, autotune=not args.no_autotune and mode == 'batched', mode=mode,
               mlp_keep_margin=args.keep_margin if flagger == 'mlp' else 0.0)


def host_state(amr, pinned=True):
    """The whole hierarchy and its interiors in (pinned) host memory."""
    import numpy as np
    import torch
    lv, co, da = [], [], []
    for l in range(amr.L):
        c, x = amr.get_level(l)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c.astype(np.int32))
        da.append(x)
    out = []
    for a in (np.concatenate(lv), np.concatenate(co), np.concatenate(da)):
        if pinned:
            t = torch.empty(a.shape, dtype={np.dtype(np.float64): torch.float64,
                                            np.dtype(np.int32): torch.int32}[a.dtype], pin_memory=True).numpy()
            t[...] = a
            a = t
        out.append(a)
    return tuple(out) + (amr.diag()[0],)


def load_weights(name, dim):
    import numpy as np
    return np.load(os.path.join(WEIGHTS_DIR, name.format(d=dim))).astype(np.float32)


# variants of the regrid-interval comparison: (label, flagger, weights file, K)
VARIANTS = [('fp32_plain_every_1', 'plain', None, 1),
            ('fp32_plain_every_4', 'plain', None, 4),
            ('fp32_learned_every_1', 'mlp', 'indicator_d{d}.npy', 1),
            ('fp32_lookahead_every_4', 'mlp', 'indicator_d{d}_diag_k4.npy', 4)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=5)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--workload', default='blast3d')
    ap.add_argument('--base', type=int, default=0, help='override base cells per dimension')
    ap.add_argument('--levels', type=int, default=0, help='override the number of levels')
    ap.add_argument('--precision', type=int, default=32)
    ap.add_argument('--flagger', default='mlp', choices=['plain', 'mlp'])
    ap.add_argument('--weights', default=None,
                    help='float32 .npy weights of the learned indicator ({d} stands for the dimension)')
    ap.add_argument('--regrid-every', type=int, default=None,
                    help='regrid interval K (default: 4 with the learned lookahead network, else 1)')
    ap.add_argument('--keep-margin', type=float, default=12.0,
                    help='learned flags: a leaf blocks the coarsening of its parent while a band logit is above '
                         'minus this margin (refinement still needs a logit above 0)')
    ap.add_argument('--window', type=float, default=0.5,
                    help='start of the headline window as a fraction of t_end (workloads without t_end: 0)')
    ap.add_argument('--sample-every', type=int, default=25, help='steps between unmet-request samples (0: none)')
    ap.add_argument('--max-patches', type=int, default=0, help='pool capacity (0: every level fully refined)')
    ap.add_argument('--checkpoint', default=None,
                    help='write the state reached at the start of the headline window to this file (amr_checkpoint)')
    ap.add_argument('--restore', default=None,
                    help='start from this checkpoint (amr_restore) instead of t = 0: the headline window only, no '
                         'other window and no whole-run figures (for profiling the mid-run state)')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-autotune', action='store_true', help='default launch parameters instead of tuned ones')
    ap.add_argument('--set-tuning', default='',
                    help='launch parameters to pin after any tuning, as name=value[,name=value] with the names of '
                         'amr.TUNE_NAMES (e.g. rhs_tile_shape=2,rhs_ctas_per_sm=1, to profile one tile shape)')
    ap.add_argument('--no-compare', action='store_true',
                    help='skip the regrid-interval variants, the FP64 paths and the L1(rho) comparison')
    args = ap.parse_args()

    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    if args.impl == 'reference':
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import __graft_entry__
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    __graft_entry__.build()
    from paper_2508_05020_gb300.amr import AMR

    w = workload(args.workload)
    if args.base:
        w['base_cells'] = tuple(args.base if d < w['dim'] else 1 for d in range(3))
    if args.levels:
        w['levels'] = args.levels
    has_end = w['t_end'] > 0
    weights_name = args.weights or ('indicator_d{d}_diag_k4.npy' if args.flagger == 'mlp' else None)
    weights = load_weights(weights_name, w['dim']) if args.flagger == 'mlp' else None
    K_r = args.regrid_every or (4 if weights_name and '_k4' in weights_name else 1)
    amr = make_amr(AMR, w, args, args.flagger, weights, precision=args.precision)
    pinned = parse_tuning(args.set_tuning)
    if pinned:
        amr.set_tuning(pinned)
    tuned, tuned_ms = amr.tuning()
    fe = fine_equivalent_cells(w)
    N = w['patch']
    run = Run(amr, w, K_r, sample_every=args.sample_every if has_end else 0)
    K, W = args.steps, args.warmup
    windows = {}

    def window(name):
        run.seg(W)
        torch.cuda.synchronize()
        leaves, t_start = run.leaves, run.t
        ms = run.seg(K)
        windows[name] = {'t_start': t_start, 'steps': K, 'ms_per_step': ms / K,
                         'fine_equivalent_cell_updates_per_s': fe * K / (ms / 1000.0),
                         'leaf_cell_updates_per_s': 0.5 * (leaves + run.leaves) * N ** w['dim'] * K / (ms / 1000.0),
                         'leaf_patches': run.leaves}

    if args.restore:                          # profiling: straight to the saved state
        amr.restore(args.restore)
        run.t = run._refresh()
        has_end = False
    else:
        # 1. t = 0
        window('t0')
        # 2. the headline window at window * t_end: state saved for the e2e and FP64 legs
        if has_end:
            run.advance_to(args.window * w['t_end'])
        if args.checkpoint:
            amr.checkpoint(args.checkpoint)
    # the tuner again on the hierarchy of the headline window (untimed; it
    # leaves the state, time and dt as they are): the mesh has grown since t = 0
    if not args.no_autotune:
        amr.autotune()
    if pinned:
        amr.set_tuning(pinned)
    tuned_half = amr.tuning()[0]
    mid_state = host_state(amr) if (rank == 0 and (not args.no_e2e or not args.no_compare)) else None
    t_h = run.t
    amr.set_timing(True)
    run.seg(W)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    _, _, k0 = amr.counters()
    _, cons0, _ = amr.diag()                   # conserved sums before the timed steps
    leaves0 = run.leaves
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    ms = run.seg(K)                           # amr_advance: K steps, a regrid every K_r, no return in between
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    kinds, nlaunch = amr.timing()             # last timed step and its regrid
    amr.set_timing(False)
    _, _, k1 = amr.counters()
    t_now, cons, ppl = amr.diag()
    elapsed = ms / 1000.0
    elapsed, units = combine_ranks(elapsed, float(fe * K), dist, device='cuda')
    if dist:
        dist.barrier()
    value = units / elapsed
    windows['half'] = {'t_start': t_h, 'steps': K, 'ms_per_step': 1000.0 * elapsed / K,
                       'fine_equivalent_cell_updates_per_s': value,
                       'leaf_cell_updates_per_s': 0.5 * (leaves0 + run.leaves) * N ** w['dim'] * K / elapsed,
                       'leaf_patches': run.leaves}
    flops = load_json(FLOPS_FILE, None)
    rhs_ms = kinds[1] / max(nlaunch[1], 1)
    flops_rhs = rhs_flops_per_launch(amr, w, flops) if flops else None
    nv = w['dim'] + 2
    # mass and energy: relative change; momenta (whose totals can vanish by symmetry): change per unit mass
    drift = [float(abs(cons[v] - cons0[v]) / max(abs(cons0[v] if v in (0, nv - 1) else cons0[0]), 1e-300))
             for v in range(nv)]
    # 3. just before t_end, then the rest of the run
    if has_end:
        run.advance_until_left(W + K + 2)
        if run.steps_left() >= W + K:
            window('t_end')
        run.advance_to(w['t_end'])
    whole = run.summary(fe, N) if not args.restore else None
    learned = None
    if args.flagger == 'mlp':
        c = amr.flag_stats()                      # learned vs plain sensor on the final state, per band cell
        learned = {'tp': int(c[0]), 'fp': int(c[1]), 'fn': int(c[2]), 'tn': int(c[3]),
                   'recall': float(c[0] / max(1, c[0] + c[2])), 'precision': float(c[0] / max(1, c[0] + c[1])),
                   'state': 'at the end of the run (t = %.4g)' % run.t, 'weights': weights_name.format(d=w['dim'])}
    amr.close()

    peaks = load_json(PEAKS_FILE, {})
    sm_max = float(peaks.get('sm_max_mhz', 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 FLOP
    roof = None
    if flops_rhs:
        achieved = float(flops_rhs) / (rhs_ms / 1000.0) / 1e12
        scheme = ('central interpolation + 4th-order staggered divergence' if w.get('flux') == 'central'
                  else 'WENO5 + Rusanov')
        roof = {'bound': 'alu', 'kernel': 'k_rhs (fused %s + SSP-RK3 stage)' % scheme,
                'achieved': achieved, 'peak': fp32_peak, 'unit': 'TFLOP/s', 'frac': achieved / fp32_peak,
                'traffic': rhs_traffic(args.workload, args.base, args.levels, leaf_patches(w, ppl),
                                       tuned_half['rhs_tile_shape']),
                'traffic_unit': 'DRAM bytes per launch (stage 1, RHS tile shape %d; ncu capture at %d leaf patches '
                                'scaled to this launch\'s %d)' % (tuned_half['rhs_tile_shape'], RHS_TRAFFIC['leaves'],
                                                                  leaf_patches(w, ppl)),
                'avg_launch_ms': rhs_ms, 'flop_per_launch': flops_rhs,
                'peak_basis': 'FP32 ALU: 152 SMs x 128 lanes x 2 FLOP x %.0f MHz (of the measured maximum SM clock)'
                              % sm_max}

    wl = '%s base %s, %d levels, %d^%d patches, FP%d, %s flags, %s flux, regrid every %d step%s' % (
        args.workload, 'x'.join(str(b) for b in w['base_cells'][:w['dim']]), w['levels'], w['patch'], w['dim'],
        args.precision, args.flagger if args.flagger == 'plain' else 'learned (%s)' % weights_name.format(d=w['dim']),
        w.get('flux', 'rusanov'), K_r, '' if K_r == 1 else 's')
    line = {'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world, 'steps': K,
            'warmup': W, 'ms_per_step': 1000.0 * elapsed / K, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32' if args.precision == 32 else 'f64',
            'data': 'synthetic',
            'config': {'workload': wl,
                       'timed_window': ('the %d steps after %d warm-up steps from t = %.4g (%.2f t_end), reached by '
                                        'running the problem from t = 0' % (K, W, t_h, t_h / w['t_end']))
                       if has_end else ('the %d steps after %d warm-up steps from the checkpoint %s (t = %.4g)'
                                        % (K, W, args.restore, t_h) if args.restore
                                        else 'the %d steps after %d warm-up steps from t = 0' % (K, W)),
                       'fine_equivalent_cells': fe, 'patches_per_level': [int(x) for x in ppl],
                       'l2': 'inputs larger than L2 (state arrays of several GB)',
                       'parallelism': 'replicas (dp%d, no data-path collective)' % world,
                       'launch_parameters': tuned_half, 'launch_parameters_t0': tuned,
                       'autotuned': ('at t = 0 and again at the start of the timed window' if not args.no_autotune
                                     else False),
                       'mlp_keep_margin': args.keep_margin if args.flagger == 'mlp' else None,
                       'regrid_every': K_r,
                       'cells_per_step': cell_counts(w, ppl)},
            'clocks': clk, 'gpu_launches': int(k1 - k0), 'roofline': roof,
            'leaf_cell_updates_per_s': windows['half']['leaf_cell_updates_per_s'],
            'windows': windows, 'whole_run': whole,
            'conservation': {'relative_drift_over_timed_steps': drift,
                             'variables': ['rho'] + ['rho u%d' % d for d in range(w['dim'])] + ['rho E'],
                             'note': 'sums over leaf cells times cell volume (FP64); mass and energy relative to their '
                                     'totals, momenta relative to the total mass; outflow boundaries, so the sums '
                                     'change once the blast reaches them'},
            'phase_ms_last_step': dict(zip(AMR.TIMING_SLOTS, [float(x) for x in kinds])),
            'wall_s': wall}
    if learned:
        line['learned_indicator'] = learned
    # the end-to-end leg first, on a GPU in the state the headline window saw
    # (after the long comparison legs it measured half the rate)
    if rank == 0 and not args.no_e2e and mid_state is not None:
        line['e2e'] = e2e_measure(AMR, w, args, fe, weights, K_r, mid_state, local)
    if rank == 0 and not args.no_compare and has_end:
        line['compare'] = compare(AMR, w, args, fe, K_r, weights_name, whole, mid_state, value)
        line['l1_rho_at_t_end'] = line['compare']['l1_rho_at_t_end_reduced'].get('fp32_headline')
    if rank == 0 and not args.no_cpu_baseline:
        v1, lv1, dt1, desc1 = oracle_sample(1)
        res, cores = oracle_all_cores(32)
        va, lva, dta = res[0]
        line['cpu_baseline'] = {'value': va, 'unit': UNIT, 'cores': cores, 'kind': 'oracle',
                                'sample': 'oracle (numpy FP64) on the 3D blast at 32^3 base cells, 3 levels, 16^3 '
                                          'patches, plain flags: %d independent replicas, one per host core, each one '
                                          'step + regrid from t = 0 (%.1f s)' % (cores, dta),
                                'leaf_cell_updates_per_s': lva,
                                'single_thread': {'value': v1, 'leaf_cell_updates_per_s': lv1, 'cores': 1,
                                                  'seconds': dt1, 'sample': desc1},
                                'note': 'fine-equivalent rates depend on how sparse the refinement is; the leaf '
                                        'cell-update rates compare like with like (GPU: leaf_cell_updates_per_s)'}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def level0_rho(amr):
    """Density of level 0 (the conservative average of the whole hierarchy)
    as one array over the level's cells, (z, y, x) order."""
    import numpy as np
    coords, x = amr.get_level(0)
    d, N = amr.dim, amr.N
    ext = [int(coords[:, k].max()) + 1 if k < d else 1 for k in range(3)]
    out = np.zeros(tuple(ext[k] * (N if k < d else 1) for k in (2, 1, 0)))
    for c, patch in zip(coords, x[:, 0]):
        sl = tuple(slice(int(c[k]) * N, int(c[k]) * N + N) if k < d else slice(None) for k in (2, 1, 0))
        out[sl] = patch.reshape(out[sl].shape)
    return out


def l1_rel(a, b):
    import numpy as np
    return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))


def compare(AMR, w, args, fe, K_r, weights_name, whole, mid_state, value):
    """The rest of the measurement beside the headline run:

    * the regrid-interval variants on the same workload, each run from t = 0
      to t_end (whole-run rates, unmet plain requests sampled every
      `sample_every` steps); the headline run is one of them;
    * the plain FP64 paths (per-patch: one launch per patch and kernel class;
      batched) timed from the headline window's state;
    * L1(rho) at t_end of every FP32 variant against the batched FP64 plain
      run (bit for bit the oracle's method) on the same problem at 32^3 base
      cells, with that run's dt sequence (the full-size FP64 run to t_end
      would take about half an hour)."""
    import numpy as np
    import torch
    out = {'regrid_interval': {}}
    head_label = None
    for label, flagger, wname, K in VARIANTS:
        is_head = (flagger == args.flagger and K == K_r and
                   (flagger == 'plain' or wname == weights_name))
        if is_head:
            head_label = label
            out['regrid_interval'][label] = dict(whole, headline=True)
            continue
        wts = load_weights(wname, w['dim']) if flagger == 'mlp' else None
        a = make_amr(AMR, w, args, flagger, wts)
        r = Run(a, w, K, sample_every=args.sample_every)
        r.advance_to(w['t_end'])
        out['regrid_interval'][label] = r.summary(fe, w['patch'])
        a.close()
    if head_label is None:
        out['regrid_interval']['headline'] = dict(whole, headline=True)
    # FP64 plain paths from the headline window's state (per-patch: one step)
    lv, co, da, t_mid = mid_state
    for name, mode, steps in (('plain_fp64_per_patch', 'per_patch', 1), ('plain_fp64_batched', 'batched', 3)):
        a = make_amr(AMR, w, args, 'plain', None, precision=64, mode=mode)
        a.set_state(lv, co, da, t=t_mid)
        if mode == 'batched':
            a.step(sync=True)                        # warm-up (graph capture); the per-patch mode has no graph
            a.regrid()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            a.step(sync=mode == 'per_patch')
            a.regrid()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        a.close()
        out[name] = {'value': fe * steps / el, 'unit': UNIT, 'ms_per_step': 1000.0 * el / steps, 'steps': steps,
                     'timing': 'host wall clock around step + regrid from the headline window\'s state (t = %.4g)'
                               % t_mid}
    out['speedup_vs_plain_fp64_per_patch'] = value / out['plain_fp64_per_patch']['value']
    out['speedup_vs_plain_fp64_batched'] = value / out['plain_fp64_batched']['value']
    # L1(rho) at t_end on the reduced problem (same dt sequence for every run)
    wr = dict(w)
    wr['base_cells'] = tuple(32 if d < w['dim'] else 1 for d in range(3))
    ref = AMR(wr, precision=64, flagger='plain', autotune=False)
    dts = []
    while True:
        dt = ref.step(sync=True)
        if not dt > 0:
            break
        dts.append(dt)
        ref.regrid()
    rho64 = level0_rho(ref)
    ref.close()
    # every cell refined to the finest level (thresholds below zero flag every
    # cell), FP64, the same dt sequence: the finest level is the uniform grid
    # at the finest spacing, the discrete solution every AMR mesh approximates
    # (uniform-fine equivalence, bit for bit in the oracle's pins), and its
    # level 0 is that solution averaged over each level-0 cell
    uni = AMR(dict(wr, theta_rho=-1.0, theta_p=-1.0), precision=64, flagger='plain', autotune=False)
    for dt in dts:
        uni.step(dt=dt, sync=False)
    rho_uni = level0_rho(uni)
    r_fine = 2 ** (w['levels'] - 1)
    uni.close()
    l1 = {'fp64_plain_every_1': {'l1_rho_vs_uniform_fine': l1_rel(rho64, rho_uni)}}
    for label, flagger, wname, K in VARIANTS:
        wts = load_weights(wname, w['dim']) if flagger == 'mlp' else None
        a = AMR(wr, precision=32, flagger=flagger, mlp_weights=wts, mlp_keep_margin=args.keep_margin)
        unmet = []
        for i, dt in enumerate(dts):
            a.step(dt=dt, sync=False)
            if (i + 1) % K == 0:
                a.regrid()
            if (i + 1) % args.sample_every == 0:
                unmet.append(a.plain_requests())
        r0 = level0_rho(a)
        l1[label] = {'l1_rho': l1_rel(r0, rho64), 'l1_rho_vs_uniform_fine': l1_rel(r0, rho_uni),
                     'unmet_plain_requests_per_step': float(np.mean(unmet)) if unmet else None}
        a.close()
        if label == head_label:
            l1['fp32_headline'] = l1[label]
    if head_label is None:
        l1['fp32_headline'] = None
    out['l1_rho_at_t_end_reduced'] = l1
    out['l1_note'] = ('relative L1 of rho on level 0 (the conservative average of the whole hierarchy) at t_end = %g '
                      'after %d steps of the same problem at 32^%d base cells, every run with the dt sequence of the '
                      'batched FP64 plain run (regrid every step): l1_rho against that run (FP32 plain every step '
                      'isolates the FP32 storage and arithmetic, the other rows add their mesh choices), '
                      'l1_rho_vs_uniform_fine against the FP64 uniform grid at the finest spacing (%d^%d cells, every '
                      'cell refined) averaged to level 0: the discretisation error a mesh choice leaves'
                      % (w['t_end'], len(dts), w['dim'], 32 * r_fine, w['dim']))
    return out


def e2e_measure(AMR, w, args, fe, weights, K_r, mid_state, gpu_index=0):
    """The same metric through the public API with host buffers, on the
    headline window's state: the hierarchy is uploaded from pinned host
    memory (amr_set_state), every step calls amr_advance(1) (a regrid every
    K_r steps) + amr_get_diag (time and conservation sums read back), and the
    final state is read back into pinned host memory (amr_get_level), all
    inside the timed region. Same options and launch parameters as the timed
    run."""
    import numpy as np
    import torch
    lv, co, da, t_mid = mid_state
    amr = make_amr(AMR, w, args, args.flagger, weights, precision=args.precision)
    res = torch.empty(2 * da.size, dtype=torch.float64, pin_memory=True).numpy()   # room for the final state
    clocks = ClockSampler(gpu_index)             # started before the warm-up: its start-up is not timed
    clocks.start()
    for _ in range(args.warmup):
        amr.advance(1, regrid=K_r)
        amr.diag()
    h0, d0, _ = amr.counters()
    t0 = time.perf_counter()
    amr.set_state(lv, co, da, t=t_mid)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        amr.advance(1, regrid=K_r)
        amr.diag()
    t2 = time.perf_counter()
    off = 0
    for l in range(w['levels']):
        c, _ = amr.get_level(l, data=False)
        shape = (len(c), w['dim'] + 2) + (w['patch'],) * w['dim']
        n = int(np.prod(shape))
        amr.get_level(l, out=res[off:off + n].reshape(shape) if off + n <= res.size else None)
        off += n
    t3 = time.perf_counter()
    clk = clocks.stop()
    el = t3 - t0
    h1, d1, _ = amr.counters()
    amr.close()
    return {'value': fe * args.steps / el, 'unit': UNIT,
            'h2d_bytes_per_step': int((h1 - h0) / args.steps), 'd2h_bytes_per_step': int((d1 - d0) / args.steps),
            'parts_s': {'set_state': t1 - t0, 'steps': t2 - t1, 'readback': t3 - t2}, 'clocks': clk,
            'note': 'state of the headline window (t = %.4g) uploaded and final state read back inside the timed '
                    'region (amortised over the steps); per step amr_advance(1) + amr_get_diag' % t_mid}


if __name__ == '__main__':
    sys.exit(main())
