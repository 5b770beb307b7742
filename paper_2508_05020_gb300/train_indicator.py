"""Train the learned refinement indicator on flags of the plain sensor.

Training data: the 1D shock-tube and shock-entropy problems run on the GPU
with the plain relative-jump sensor; every few steps the 5-point (rho, u, p)
stencils of the leaf band cells and their plain flags are harvested
(amr_harvest). For a d-dimensional network each 1D sample is embedded as a
stencil constant across the other axes, along every axis and sign
(amr_mlp_features), and the network is trained with the library's own FP32
forward/backward kernels and Adam (amr_mlp_train). Weights are written as
float32 .npy files, one per dimension.

With --lookahead K the label of a cell is its plain flag at any of the next
K steps (the cell itself included now): the network then predicts where the
plain sensor is about to flag, so that a hierarchy regridded every K steps
stays refined ahead of moving fronts. These data come from single-level runs
at the finest resolution of each problem (a fixed set of cells, so that the
flags of later steps line up with the stencils of the current one).

    python -m paper_2508_05020_gb300.train_indicator --out DIR [--lookahead K]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def harvest(name, every, max_steps=100000):
    from paper_2508_05020_gb300.amr import AMR
    from synth import workload
    w = workload(name)
    a = AMR(w, precision=64)
    smp, lab = [], []
    step = 0
    t = 0.0
    while t < w['t_end'] - 1e-12 and step < max_steps:
        if step % every == 0:
            s, l = a.harvest()
            smp.append(s)
            lab.append(l)
        a.step(sync=False)
        a.regrid()
        step += 1
        t, _, _ = a.diag()
    a.close()
    return np.concatenate(smp), np.concatenate(lab)


def harvest_lookahead(name, k, max_steps=100000):
    """Stencils of every step of a single-level run at the problem's finest
    resolution, labelled with the OR of the plain flag over that step and the
    next k steps (the last k steps of the run only serve as later flags)."""
    from paper_2508_05020_gb300.amr import AMR
    from synth import workload
    w0 = workload(name)
    fine = tuple(b * 2 ** (w0['levels'] - 1) if d < w0['dim'] else 1 for d, b in enumerate(w0['base_cells']))
    w = workload(name, base_cells=fine, levels=1)
    a = AMR(w, precision=64)
    smp, lab = [], []
    step = 0
    t = 0.0
    while t < w['t_end'] - 1e-12 and step < max_steps:
        s, l = a.harvest()
        smp.append(s)
        lab.append(l)
        a.step(sync=False)
        step += 1
        t, _, _ = a.diag()
    a.close()
    L = np.stack(lab)                                      # (steps, cells); 255: out of the domain
    valid = L[0] != 255
    F = (L == 1)
    out_s, out_l = [], []
    for n in range(len(smp) - k):
        y = F[n:n + k + 1].any(axis=0)
        out_s.append(smp[n][valid])
        out_l.append(y[valid].astype(np.uint8))
    return np.concatenate(out_s), np.concatenate(out_l)


def train(dim, s, y, epochs, batch, lr, seed=0):
    from paper_2508_05020_gb300 import amr
    from synth import mlp_init
    X = amr.mlp_features(dim, 1.4, s)
    yy = np.repeat(y.astype(np.float32), 2 * dim)
    pos = float(yy.sum())
    pw = (len(yy) - pos) / max(pos, 1.0)
    p = mlp_init(seed, amr.mlp_k(dim))
    w0 = np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ('W1', 'b1', 'W2', 'b2', 'W3', 'b3')])
    w, hist = amr.mlp_train(dim, X, yy, pw, w0.astype(np.float32), epochs=epochs, batch=batch, lr=lr, seed=1)
    return w, hist, pw


def evaluate(dim, w, s, y):
    from paper_2508_05020_gb300 import amr
    X = amr.mlp_features(dim, 1.4, s)
    yy = np.repeat(y.astype(bool), 2 * dim)
    pred = amr.mlp_infer(dim, X, w) > 0
    tp = int(np.sum(pred & yy))
    fp = int(np.sum(pred & ~yy))
    fn = int(np.sum(~pred & yy))
    return {'recall': tp / max(1, tp + fn), 'precision': tp / max(1, tp + fp), 'rows': int(len(yy))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--out', required=True)
    ap.add_argument('--epochs', type=int, default=40)
    ap.add_argument('--batch', type=int, default=512)
    ap.add_argument('--lr', type=float, default=2e-3)
    ap.add_argument('--dims', default='1,2,3')
    ap.add_argument('--lookahead', type=int, default=0,
                    help='K > 0: label = plain flag within the next K steps (single-level finest runs)')
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    t0 = time.time()
    if args.lookahead > 0:
        s1, l1 = harvest_lookahead('sod', args.lookahead)
        s2, l2 = harvest_lookahead('shu_osher', args.lookahead)
    else:
        s1, l1 = harvest('sod', every=4)
        s2, l2 = harvest('shu_osher', every=8)
    s = np.concatenate([s1, s2])
    y = np.concatenate([l1, l2])
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(s))
    n_test = len(s) // 5
    te, tr = perm[:n_test], perm[n_test:]
    os.makedirs(args.out, exist_ok=True)
    report = {'samples': int(len(s)), 'positives': int(y.sum()), 'harvest_s': time.time() - t0,
              'lookahead': args.lookahead}
    suffix = '_k%d' % args.lookahead if args.lookahead > 0 else ''
    for dim in [int(x) for x in args.dims.split(',')]:
        t1 = time.time()
        w, hist, pw = train(dim, s[tr], y[tr], args.epochs, args.batch, args.lr)
        np.save(os.path.join(args.out, 'indicator_d%d%s.npy' % (dim, suffix)), w)
        report['d%d' % dim] = {'train_s': time.time() - t1, 'loss_first': float(hist[0]),
                               'loss_last': float(hist[-1]), 'pos_weight': pw,
                               'heldout': evaluate(dim, w, s[te], y[te])}
        print(json.dumps({'dim': dim, **report['d%d' % dim]}), flush=True)
    with open(os.path.join(args.out, 'indicator_report%s.json' % suffix), 'w') as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))


if __name__ == '__main__':
    main()
