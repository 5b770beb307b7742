#!/usr/bin/env python
"""Throughput benchmark of the AMR Euler hot path on GB300.

A step is one pass of the whole hot path over the hierarchy: CFL reduction,
three SSP-RK3 stages (ghost fill, fused WENO5/Rusanov RHS + stage update,
reflux, restriction) over every patch of every level, then flagging and
regrid. The default workload is the 3D blast problem (128^3 base cells, 3
levels, 16^3 patches, FP32 fields; its inputs exceed L2). The metric is
fine-equivalent cell-updates per second: (base cells x 2^(d (L-1))) x steps /
seconds.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank advances its own replica (no collective on the
data path); rank 0 prints one JSON line.
"""
import argparse
import json
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

# DRAM bytes of one stage-1 k_rhs launch (ncu, dram__bytes_read.sum +
# dram__bytes_write.sum; the capture summarised in
# profiles/k_rhs_blast3d_128_fp32.md) on the default workload, valid while the
# sources of the kernel (the regions below: EOS, WENO5, face fluxes, the
# kernel and its launch) hash as recorded
RHS_TRAFFIC = {'bytes': 320362496 + 152754688, 'workload': 'blast3d', 'base': 128, 'levels': 3,
               'regions': [('paper_2508_05020_gb300/csrc/amr_kernels.cuh', 'template <typename T> struct Num;',
                            '// Metadata of one patch staged'),
                           ('paper_2508_05020_gb300/csrc/amr_kernels.cuh', '// K4: fused right-hand side',
                            '// K5: coarse-fine flux correction'),
                           ('paper_2508_05020_gb300/csrc/amr_launch.cuh', 'template <typename T, int D, int N> struct RhsCfg',
                            'template <typename T>\ncudaError_t Kernels<T>::prepare')],
               'hash': '3a9f979e10e4a37b'}


def rhs_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f, a, b in RHS_TRAFFIC['regions']:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        i = text.index(a)
        h.update(text[i:text.index(b, i)].encode())
    return h.hexdigest()[:16]


def rhs_traffic(workload_name, base, levels):
    if workload_name != RHS_TRAFFIC['workload'] or base not in (0, RHS_TRAFFIC['base']) or \
            levels not in (0, RHS_TRAFFIC['levels']):
        return None
    try:
        if rhs_source_hash() != RHS_TRAFFIC['hash']:
            return None
    except ValueError:
        return None
    return RHS_TRAFFIC['bytes']


def load_json(path, default):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return default


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


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(steps, base=32):
    """The FP64 CPU oracle, as it stands, on the same problem at base^3 cells:
    returns (fine-equivalent cell-updates/s, seconds, description)."""
    from oracle.amr import Oracle
    w = workload('blast3d', base_cells=(base, base, base))
    o = Oracle(w)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
        o.regrid()
    dt = time.perf_counter() - t0
    fe = fine_equivalent_cells(w)
    desc = ('oracle (numpy FP64, single thread) on the same 3D blast problem at %d^3 base cells, 3 levels, '
            '16^3 patches: %d step(s) of step + regrid from t = 0' % (base, steps))
    return fe * steps / dt, dt, desc


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    # each step a bounded sample: the same problem at 16^3 base cells (about a
    # second of CPU work), so that --steps K --warmup W ends within minutes
    per_step = []
    for i in range(args.warmup + args.steps):
        v, dt, desc = oracle_sample(1, base=16)
        if i >= args.warmup:
            per_step.append(dt)
    w = workload('blast3d', base_cells=(16, 16, 16))
    fe = fine_equivalent_cells(w)
    total = sum(per_step)
    val = fe * len(per_step) / total
    line = {'impl': 'reference', 'metric': METRIC, 'value': val, 'unit': UNIT, 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': 1000.0 * total / len(per_step),
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic', 'config': {'workload': 'blast3d base 128x128x128, 3 levels, 16^3 patches, FP32, '
                                                        'mlp flags, rusanov flux',
                                            'reference_sample': 'the FP64 CPU oracle (plain flags) on the same '
                                                                'problem at 16^3 base cells per timed step'},
            'cpu_baseline': {'value': val, 'unit': UNIT, 'cores': 1, 'kind': 'oracle', 'sample': desc},
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


# ----------------------------------------------------------------------------- GPU
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=40)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--workload', default='blast3d')
    ap.add_argument('--base', type=int, default=0, help='override base cells per dimension')
    ap.add_argument('--levels', type=int, default=0, help='override the number of levels')
    ap.add_argument('--precision', type=int, default=32)
    ap.add_argument('--flagger', default='mlp', choices=['plain', 'mlp'])
    ap.add_argument('--weights', default=None, help='float32 .npy weights of the learned indicator')
    ap.add_argument('--keep-margin', type=float, default=12.0,
                    help='learned flags: a leaf blocks the coarsening of its parent while a band logit is above '
                         'minus this margin (refinement still needs a logit above 0)')
    ap.add_argument('--max-patches', type=int, default=0, help='pool capacity (0: every level fully refined)')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-autotune', action='store_true', help='default launch parameters instead of tuned ones')
    ap.add_argument('--no-compare', action='store_true',
                    help='skip the plain FP64 per-patch path and the L1(rho) comparison')
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
    weights = None
    if args.flagger == 'mlp':
        path = args.weights or os.path.join(ROOT, 'paper_2508_05020_gb300', 'weights', 'indicator_d%d.npy' % w['dim'])
        weights = np.load(path).astype(np.float32)
    amr = AMR(w, precision=args.precision, flagger=args.flagger, mlp_weights=weights, max_patches=args.max_patches,
              autotune=not args.no_autotune, mlp_keep_margin=args.keep_margin)
    tuned, tuned_ms = amr.tuning()
    stream = amr._keep[1]
    amr.set_timing(True)

    def one_step():
        amr.step(sync=False)
        amr.regrid()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    _, _, k0 = amr.counters()
    _, cons0, _ = amr.diag()                   # conserved sums before the timed steps
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    flops = load_json(FLOPS_FILE, None)
    # no host synchronisation inside the loop but the regrid's own read-back of
    # the refinement requests; the per-class CUDA events are event nodes of the
    # captured step graph and are read once, after the loop, for the last step
    amr.advance(args.steps)                 # amr_advance: step + regrid per step, no return in between
    ev1.record(stream)
    torch.cuda.synchronize()
    kinds, nlaunch = amr.timing()           # last timed step and its regrid
    rhs_ms = [kinds[1] / max(nlaunch[1], 1)]
    flops_rhs = [rhs_flops_per_launch(amr, w, flops)] if flops else []
    if flops_rhs and flops_rhs[0] is None:
        flops_rhs = []
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    _, _, k1 = amr.counters()
    fe = fine_equivalent_cells(w)
    elapsed, units = combine_ranks(elapsed, float(fe * args.steps), dist, device='cuda')
    if dist:
        dist.barrier()
    value = units / elapsed
    t_now, cons, ppl = amr.diag()
    # mass and energy: relative change; momenta (whose totals can vanish by symmetry): change per unit mass
    nv = w['dim'] + 2
    drift = [float(abs(cons[v] - cons0[v]) / max(abs(cons0[v] if v in (0, nv - 1) else cons0[0]), 1e-300))
             for v in range(nv)]

    peaks = load_json(PEAKS_FILE, {})
    sm_max = float(peaks.get('sm_max_mhz', 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 FLOP
    roof = None
    if flops_rhs:
        avg_ms = float(np.mean(rhs_ms))
        achieved = float(np.mean(flops_rhs)) / (avg_ms / 1000.0) / 1e12
        scheme = ('central interpolation + 4th-order staggered divergence' if w.get('flux') == 'central'
                  else 'WENO5 + Rusanov')
        roof = {'bound': 'alu', 'kernel': 'k_rhs (fused %s + SSP-RK3 stage)' % scheme,
                'achieved': achieved, 'peak': fp32_peak, 'unit': 'TFLOP/s', 'frac': achieved / fp32_peak,
                'traffic': rhs_traffic(args.workload, args.base, args.levels), 'traffic_unit': 'bytes per launch (stage 1)',
                'avg_launch_ms': avg_ms,
                'peak_basis': 'FP32 ALU: 152 SMs x 128 lanes x 2 FLOP x %.0f MHz' % sm_max}

    line = {'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': 1000.0 * elapsed / args.steps, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32' if args.precision == 32 else 'f64',
            'data': 'synthetic',
            'config': {'workload': '%s base %s, %d levels, %d^%d patches, FP%d, %s flags, %s flux' % (
                args.workload, 'x'.join(str(b) for b in w['base_cells'][:w['dim']]), w['levels'], w['patch'],
                w['dim'], args.precision, args.flagger, w.get('flux', 'rusanov')),
                'fine_equivalent_cells': fe, 'patches_per_level': [int(x) for x in ppl],
                'l2': 'inputs larger than L2 (state arrays of several GB)',
                'parallelism': 'replicas (dp%d, no data-path collective)' % world,
                'launch_parameters': tuned, 'autotuned': not args.no_autotune,
                'mlp_keep_margin': args.keep_margin if args.flagger == 'mlp' else None,
                'cells_per_step': cell_counts(w, ppl)},
            'clocks': clk, 'gpu_launches': int(k1 - k0), 'roofline': roof,
            'conservation': {'relative_drift_over_timed_steps': drift,
                             'variables': ['rho'] + ['rho u%d' % d for d in range(w['dim'])] + ['rho E'],
                             'note': 'sums over leaf cells times cell volume (FP64); mass and energy relative to their '
                                     'totals, momenta relative to the total mass; exact conservation on periodic or '
                                     'closed domains up to round-off'},
            'phase_ms_last_step': dict(zip(AMR.TIMING_SLOTS, [float(x) for x in kinds])),
            'wall_s': wall}

    if args.flagger == 'mlp':
        c = amr.flag_stats()                      # learned vs plain sensor on the final state, per band cell
        line['learned_indicator'] = {'tp': int(c[0]), 'fp': int(c[1]), 'fn': int(c[2]), 'tn': int(c[3]),
                                     'recall': float(c[0] / max(1, c[0] + c[2])),
                                     'precision': float(c[0] / max(1, c[0] + c[1])),
                                     'state': 'after the timed steps'}
    amr.close()
    if rank == 0 and not args.no_compare:
        line['compare'] = compare_fp64_plain(AMR, w, args, fe, weights, value)
    if rank == 0 and not args.no_e2e:
        line['e2e'] = e2e_measure(AMR, w, args, fe, weights)
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, desc = oracle_sample(1)
        line['cpu_baseline'] = {'value': v, 'unit': UNIT, 'cores': 1, 'kind': 'oracle', 'sample': desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


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


def level0_rho(amr):
    _, x = amr.get_level(0)
    return x[:, 0]


def compare_fp64_plain(AMR, w, args, fe, weights, value):
    """The plain per-patch FP64 GPU path beside the batched one: its
    throughput on the same workload (one launch per patch and kernel class,
    plain sensor, FP64 fields), and L1(rho) on level 0 (the conservative
    average of the whole hierarchy) of the batched FP32 runs, with learned and
    with plain flags, against it after the same steps with the same dt."""
    import numpy as np
    import torch
    steps = max(2, min(args.steps, 5))
    ref = AMR(w, precision=64, flagger='plain', mode='per_patch')
    dts = []
    for _ in range(1):                             # warm-up (launch paths, allocator)
        dts.append(ref.step(sync=True))
        ref.regrid()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dts.append(ref.step(sync=True))
        ref.regrid()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    rho64 = level0_rho(ref)
    ref.close()
    out = {'plain_fp64_per_patch': {'value': fe * steps / el, 'unit': UNIT, 'ms_per_step': 1000.0 * el / steps,
                                    'steps': steps, 'timing': 'host wall clock around steps + regrids (dt read '
                                    'back every step)'},
           'speedup_batched_fp32_learned': value / (fe * steps / el)}
    # the batched FP64 plain path, for the share of the gain that batching alone gives
    b64 = AMR(w, precision=64, flagger='plain', autotune=True)
    b64.step(sync=True)
    b64.regrid()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b64.step(sync=False)
        b64.regrid()
    torch.cuda.synchronize()
    el64 = time.perf_counter() - t0
    b64.close()
    out['plain_fp64_batched'] = {'value': fe * steps / el64, 'unit': UNIT, 'ms_per_step': 1000.0 * el64 / steps,
                                 'steps': steps, 'timing': 'host wall clock around steps + regrids'}
    l1 = {}
    for name, prec, flagger in (('fp32_learned', 32, 'mlp'), ('fp32_plain', 32, 'plain'), ('fp64_batched_plain', 64, 'plain')):
        a = AMR(w, precision=prec, flagger=flagger, mlp_weights=weights if flagger == 'mlp' else None,
                mlp_keep_margin=args.keep_margin)
        for dt in dts:
            a.step(dt=dt)
            a.regrid()
        r = level0_rho(a)
        a.close()
        l1[name] = float(np.sum(np.abs(r - rho64)) / np.sum(np.abs(rho64)))
    out['l1_rho_vs_plain_fp64'] = l1
    out['l1_rho_note'] = ('relative L1 of rho on level 0 after %d steps (t = %.4g) with the per-patch FP64 '
                          "plain run's dt sequence" % (len(dts), float(sum(dts))))
    return out


def e2e_measure(AMR, w, args, fe, weights=None):
    """The same metric through the public API with host buffers: the initial
    hierarchy is uploaded from host memory (amr_set_state), every step calls
    amr_advance(1) (step + regrid) + amr_get_diag (time and conservation sums
    read back), and the final state is read back to host memory
    (amr_get_level). Same options and launch parameters as the timed run."""
    import numpy as np
    import torch

    def pinned(a):
        t = torch.empty(a.shape, dtype={np.dtype(np.float64): torch.float64, np.dtype(np.int32): torch.int32}[a.dtype],
                        pin_memory=True).numpy()
        t[...] = a
        return t

    amr = AMR(w, precision=args.precision, flagger=args.flagger, mlp_weights=weights, mlp_keep_margin=args.keep_margin,
              max_patches=args.max_patches, autotune=not args.no_autotune)
    lv, co, da = [], [], []
    for l in range(w['levels']):
        c, x = amr.get_level(l)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c.astype(np.int32))
        da.append(x)
    lv = pinned(np.concatenate(lv))                 # the inputs and outputs in pinned host memory
    co = pinned(np.concatenate(co))
    da = pinned(np.concatenate(da))
    res = torch.empty(2 * da.size, dtype=torch.float64, pin_memory=True).numpy()   # room for the final state
    for _ in range(args.warmup):
        amr.advance(1)
        amr.diag()
    h0, d0, _ = amr.counters()
    t0 = time.perf_counter()
    amr.set_state(lv, co, da, t=0.0)
    for _ in range(args.steps):
        amr.advance(1)
        amr.diag()
    off = 0
    for l in range(w['levels']):
        c, _ = amr.get_level(l, data=False)
        shape = (len(c), w['dim'] + 2) + (w['patch'],) * w['dim']
        n = int(np.prod(shape))
        amr.get_level(l, out=res[off:off + n].reshape(shape) if off + n <= res.size else None)
        off += n
    el = time.perf_counter() - t0
    h1, d1, _ = amr.counters()
    amr.close()
    return {'value': fe * args.steps / el, 'unit': UNIT,
            'h2d_bytes_per_step': int((h1 - h0) / args.steps), 'd2h_bytes_per_step': int((d1 - d0) / args.steps),
            'note': 'initial state uploaded and final state read back inside the timed region (amortised over '
                    'the steps); per step amr_advance(1) (step + regrid) + amr_get_diag'}


if __name__ == '__main__':
    sys.exit(main())
