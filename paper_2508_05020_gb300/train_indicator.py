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

With --embed diag (which --lookahead K may accompany) the d-dimensional
training stencils are planar waves of
the 1D profiles along the axes and along the face and body diagonals (offset
o of the 5^d stencil reads the profile at o . n for an integer direction n,
the velocity is u n / |n|): fronts oblique to the grid, as a spherical blast
has, are in the training set. The profiles come from single-level runs at the
finest resolution (13-cell windows of the whole level, read back every few
steps); the plain sensor compares the +-1 neighbours along each axis, which
are the profile's +-1 neighbours for every such direction, so the label is
the 1D flag of the profile.

    python -m paper_2508_05020_gb300.train_indicator --out DIR [--lookahead K] [--embed diag]
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


PROFILE = 13                                               # cells of a harvested 1D window (+-6)


def harvest_profiles(name, every, max_steps=100000, theta=0.05, lookahead=0):
    """13-cell (rho, u, p) windows around every interior cell of single-level
    runs at the problem's finest resolution, every `every` steps, and the
    plain flag of the centre cell (with lookahead K: the OR of its flags at
    that step and the next K steps; the cells of the level are fixed, so a
    window's later flags are those of the same cell)."""
    from paper_2508_05020_gb300.amr import AMR
    from synth import workload
    w0 = workload(name)
    fine = (w0['base_cells'][0] * 2 ** (w0['levels'] - 1), 1, 1)
    w = workload(name, base_cells=fine, levels=1)
    a = AMR(w, precision=64)
    gm1 = w['gamma'] - 1.0
    h = PROFILE // 2
    win, lab, at = [], [], []
    flags = []                                       # flags of every step (lookahead)
    step = 0
    t = 0.0
    while t < w['t_end'] - 1e-12 and step < max_steps:
        if step % every == 0 or lookahead > 0:
            c, x = a.get_level(0)
            order = np.argsort(c[:, 0])
            U = np.concatenate([x[i] for i in order], axis=1)     # (3, cells)
            rho = U[0]
            u = U[1] / rho
            p = gm1 * (U[2] - 0.5 * rho * u * u)
            n = rho.size
            idx = np.arange(h, n - h)[:, None] + np.arange(-h, h + 1)[None, :]
            prof = np.stack([rho[idx], u[idx], p[idx]], axis=2)   # (m, 13, 3)
            f = np.zeros(len(prof), dtype=bool)
            for k in (0, 2):
                fm, f0, fp = prof[:, h - 1, k], prof[:, h, k], prof[:, h + 1, k]
                f |= np.abs(fp - fm) > theta * (fp + 2.0 * f0 + fm)
            flags.append(f)
            if step % every == 0:
                win.append(prof)
                lab.append(f.astype(np.uint8))
                at.append(len(flags) - 1)
        a.step(sync=False)
        step += 1
        t, _, _ = a.diag()
    a.close()
    if lookahead > 0:
        for i, s in enumerate(at):
            later = flags[s:s + lookahead + 1]
            lab[i] = np.logical_or.reduce(later).astype(np.uint8)
    return np.concatenate(win), np.concatenate(lab)


def directions(dim):
    """Integer directions of the planar waves: the axes, and in 2D/3D the
    face diagonals, and in 3D the body diagonals (both signs)."""
    import itertools
    out = []
    for n in itertools.product((-1, 0, 1), repeat=dim):
        if any(n):
            out.append(np.array(n))
    return out


def embedded_features(prof, dim, dirs, gamma):
    """Centre-normalised 5^d stencil features (the network's input layout:
    k = j (d + 2) + f, stencil point j with x fastest, fields rho~, u~_d, p~)
    of the windows `prof` embedded along the directions `dirs` (one per row)."""
    import itertools
    h = PROFILE // 2
    F = dim + 2
    pts = list(itertools.product(range(-2, 3), repeat=dim))       # (.., oy, ox) with ox fastest
    pts = [tuple(reversed(q)) for q in pts]                       # as (ox, oy, oz)
    m = len(prof)
    X = np.empty((m, len(pts) * F))
    rho0, u0, p0 = prof[:, h, 0], prof[:, h, 1], prof[:, h, 2]
    c0 = np.sqrt(gamma * p0 / rho0)
    norm = np.sqrt(np.sum(dirs * dirs, axis=1))
    for j, o in enumerate(pts):
        k = h + np.sum(dirs * np.array(o)[None, :], axis=1)       # profile index of the point
        r = prof[np.arange(m), k, 0]
        u = prof[np.arange(m), k, 1]
        p = prof[np.arange(m), k, 2]
        X[:, j * F] = r / rho0 - 1.0
        for d in range(dim):
            X[:, j * F + 1 + d] = u * dirs[:, d] / norm / c0
        X[:, j * F + F - 1] = p / p0 - 1.0
    return X


def train_features(dim, X, yy, epochs, batch, lr, seed=0):
    from paper_2508_05020_gb300 import amr
    from synth import mlp_init
    pos = float(yy.sum())
    pw = (len(yy) - pos) / max(pos, 1.0)
    p = mlp_init(seed, amr.mlp_k(dim))
    w0 = np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ('W1', 'b1', 'W2', 'b2', 'W3', 'b3')])
    w, hist = amr.mlp_train(dim, X.astype(np.float32), yy.astype(np.float32), pw, w0.astype(np.float32),
                            epochs=epochs, batch=batch, lr=lr, seed=1)
    return w, hist, pw


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
    ap.add_argument('--embed', default='axes', choices=['axes', 'diag'],
                    help='diag: planar waves along axes and diagonals from 13-cell profiles')
    ap.add_argument('--rows', type=int, default=1500000, help='training rows per dimension (--embed diag)')
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    t0 = time.time()
    if args.embed == 'diag':
        return main_diag(args)
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


def main_diag(args):
    t0 = time.time()
    p1, l1 = harvest_profiles('sod', every=2, lookahead=args.lookahead)
    p2, l2 = harvest_profiles('shu_osher', every=4, lookahead=args.lookahead)
    prof = np.concatenate([p1, p2])
    y = np.concatenate([l1, l2])
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(prof))
    n_test = len(prof) // 5
    te, tr = perm[:n_test], perm[n_test:]
    os.makedirs(args.out, exist_ok=True)
    report = {'profiles': int(len(prof)), 'positives': int(y.sum()), 'harvest_s': time.time() - t0,
              'embed': 'axes and diagonals', 'lookahead': args.lookahead}
    suffix = '_k%d' % args.lookahead if args.lookahead > 0 else ''
    from paper_2508_05020_gb300 import amr
    for dim in [int(x) for x in args.dims.split(',')]:
        t1 = time.time()
        dirs = np.array(directions(dim))
        # rows: every positive profile and an equal share of the rest, each along a random direction
        pos = tr[y[tr] == 1]
        neg = tr[y[tr] == 0]
        n_rows = min(args.rows, 8 * len(pos) + len(neg))
        pick = np.concatenate([rng.choice(pos, size=min(len(pos) * 8, n_rows // 2)),
                               rng.choice(neg, size=n_rows - min(len(pos) * 8, n_rows // 2), replace=False)])
        dsel = dirs[rng.integers(0, len(dirs), size=len(pick))]
        X = embedded_features(prof[pick], dim, dsel, 1.4)
        w, hist, pw = train_features(dim, X, y[pick].astype(np.float32), args.epochs, args.batch, args.lr)
        np.save(os.path.join(args.out, 'indicator_d%d%s.npy' % (dim, suffix)), w)
        # held out: every direction of the test profiles
        tsel = te[: max(1, 200000 // len(dirs))]
        Xt = embedded_features(np.repeat(prof[tsel], len(dirs), axis=0), dim, np.tile(dirs, (len(tsel), 1)), 1.4)
        yt = np.repeat(y[tsel].astype(bool), len(dirs))
        pred = amr.mlp_infer(dim, Xt.astype(np.float32), w) > 0
        tp, fp, fn = int(np.sum(pred & yt)), int(np.sum(pred & ~yt)), int(np.sum(~pred & yt))
        report['d%d' % dim] = {'train_s': time.time() - t1, 'rows': int(len(pick)), 'loss_first': float(hist[0]),
                               'loss_last': float(hist[-1]), 'pos_weight': pw,
                               'heldout_all_directions': {'recall': tp / max(1, tp + fn),
                                                          'precision': tp / max(1, tp + fp), 'rows': int(len(yt))}}
        print(json.dumps({'dim': dim, **report['d%d' % dim]}), flush=True)
    with open(os.path.join(args.out, 'indicator_report%s.json' % suffix), 'w') as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))
    return 0


if __name__ == '__main__':
    main()
