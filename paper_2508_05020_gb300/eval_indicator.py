"""Evaluate weights of the learned refinement indicator on the GPU.

Two measurements, each printed and written as JSON:

agreement  Cell-level agreement of each weight set with the plain sensor
           (amr_flag_stats: true and false positives and negatives over the
           in-domain band cells of every leaf). The state comes from running
           the 3D blast for 20 steps, and the four-quadrant problem and the
           double Mach reflection for 40 steps each, with the plain sensor,
           in FP32.

unmet      The hierarchy is regridded only every K steps. The measure is the
           mean number of patches per step that the plain sensor would refine
           on the current hierarchy but that are not refined. It is taken for
           the plain sensor regridded every step and every K steps, and for
           each weight set regridded every K steps. The run is FP64. A second
           context with the plain sensor reads the requests from an uploaded
           copy of the state.

Weight sets are given as LABEL=PATTERN, where {d} in PATTERN stands for the
dimension, for example net=paper_2508_05020_gb300/weights/indicator_d{d}.npy.

    python -m paper_2508_05020_gb300.eval_indicator agreement --weights LABEL=PATTERN ... --out FILE
    python -m paper_2508_05020_gb300.eval_indicator unmet -k 4 --weights LABEL=PATTERN ... --out FILE
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

AGREEMENT_CASES = [('blast3d', {}, 20), ('riemann2d', {}, 40), ('dmr', {}, 40)]
UNMET_CASES = [('sod', {}, 80), ('shu_osher', {}, 200), ('riemann2d', dict(base_cells=(64, 64, 1)), 80),
               ('dmr', dict(base_cells=(128, 32, 1)), 80), ('blast3d', dict(base_cells=(32, 32, 32)), 24)]


def parse_weights(specs):
    """[(label, pattern)] from LABEL=PATTERN strings; the pattern must hold {d}."""
    out = []
    for s in specs:
        label, sep, pattern = s.partition('=')
        if not sep or not label or '{d}' not in pattern:
            raise ValueError('weights must be LABEL=PATTERN with {d} in the pattern: %r' % s)
        out.append((label, pattern))
    return out


def load_weights(pattern, dim):
    path = pattern.format(d=dim)
    if not os.path.isabs(path):
        path = os.path.join(ROOT, path)
    return np.load(path).astype(np.float32) if os.path.exists(path) else None


def agreement(weights, cases=AGREEMENT_CASES):
    from paper_2508_05020_gb300.amr import AMR
    from synth import workload
    res = {}
    for name, kw, steps in cases:
        w = workload(name, **kw)
        sets = [(label, load_weights(p, w['dim'])) for label, p in weights]
        sets = [(label, x) for label, x in sets if x is not None]
        if not sets:
            continue
        a = AMR(w, precision=32, flagger='plain')
        a.advance(steps)
        out = {}
        for label, x in sets:
            a.set_mlp(x)
            c = a.flag_stats()
            out[label] = {'recall': float(c[0] / max(1, c[0] + c[2])), 'precision': float(c[0] / max(1, c[0] + c[1])),
                          'counts': [int(v) for v in c]}
        a.close()
        res[name] = out
        print(name, json.dumps(out), flush=True)
    return res


def _state(a):
    lv, co, da = [], [], []
    for l in range(a.L):
        c, x = a.get_level(l)
        lv.append(np.full(len(c), l, dtype=np.int32))
        co.append(c)
        da.append(x)
    return np.concatenate(lv), np.concatenate(co), np.concatenate(da)


def _unmet_run(w, flagger, wts, every, steps):
    from paper_2508_05020_gb300.amr import AMR
    a = AMR(w, precision=64, flagger=flagger, mlp_weights=wts)
    plain = AMR(w, precision=64, flagger='plain')
    miss, patches = [], []
    for i in range(steps):
        a.step()
        lv, co, da = _state(a)
        plain.set_state(lv, co, da, t=a.diag()[0])
        r, _ = plain.requests()
        miss.append(len(r))
        patches.append(int(sum(a.diag()[2])))
        if (i + 1) % every == 0:
            a.regrid()
    a.close()
    plain.close()
    return {'missed_refinements_per_step': float(np.mean(miss)), 'max_missed': int(np.max(miss)),
            'mean_patches': float(np.mean(patches))}


def unmet(k, weights, cases=UNMET_CASES):
    from synth import workload
    res = {}
    for name, kw, steps in cases:
        w = workload(name, **kw)
        out = {'plain_every_1': _unmet_run(w, 'plain', None, 1, steps),
               'plain_every_%d' % k: _unmet_run(w, 'plain', None, k, steps)}
        for label, p in weights:
            x = load_weights(p, w['dim'])
            if x is not None:
                out['%s_every_%d' % (label, k)] = _unmet_run(w, 'mlp', x, k, steps)
        res[name] = out
        print(name, json.dumps(out), flush=True)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split('\n\n')[0])
    ap.add_argument('what', choices=('agreement', 'unmet'))
    ap.add_argument('--weights', nargs='+', required=True, help='LABEL=PATTERN, {d} = dimension')
    ap.add_argument('-k', type=int, default=4, help='regrid interval of the unmet measurement')
    ap.add_argument('--out', required=True)
    args = ap.parse_args(argv)
    weights = parse_weights(args.weights)
    if args.k < 1:
        ap.error('-k must be at least 1')
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    res = agreement(weights) if args.what == 'agreement' else unmet(args.k, weights)
    with open(args.out, 'w') as f:
        json.dump(res, f, indent=1)
    return 0


if __name__ == '__main__':
    sys.exit(main())
