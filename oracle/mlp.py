"""FP64 refinement-indicator network of the oracle (test infrastructure).

A cell's input is its 5^d stencil of primitive variables (rho, u_0..u_{d-1}, p),
normalised by the centre cell: rho/rho_0 - 1, u/c_0, p/p_0 - 1 with
c_0 = sqrt(gamma p_0 / rho_0). Stencil points are ordered lexicographically
(z, y, x; offsets -2..2, x fastest), features per point in the order
(rho, u_0..u_{d-1}, p), so K = 5^d (d + 2). The network is
K -> 64 -> 64 -> 1 with ReLU hidden layers; the logit z > 0 predicts the plain
relative-jump flag of the cell. Training minimises the weighted binary cross
entropy  mean(pw y softplus(-z) + (1 - y) softplus(z))  with Adam.

The paper has no learned component: the refinement criterion is left to "the
runtime program" (Sec. 4.2); this network is one such program.
"""
import itertools

import numpy as np

HIDDEN = 64


def k_in(dim):
    return 5 ** dim * (dim + 2)


def stencil_offsets(dim):
    """Offsets of the 5^d stencil, lexicographic (z, y, x) with x fastest,
    returned as tuples (ox, oy, oz)."""
    rng = [range(-2, 3) if d < dim else (0,) for d in (2, 1, 0)]
    return [(o[2], o[1], o[0]) for o in itertools.product(*rng)]


def features(rho, u, p, gamma):
    """Normalised features of stencils. rho, p: (n, S); u: list of d arrays
    (n, S), S = 5^d points in stencil order with the centre at S // 2.
    Returns (n, K) with per-point feature order (rho, u..., p)."""
    S = rho.shape[1]
    c = S // 2
    r0 = rho[:, c:c + 1]
    p0 = p[:, c:c + 1]
    c0 = np.sqrt(gamma * p0 / r0)
    cols = [rho / r0 - 1.0] + [ud / c0 for ud in u] + [p / p0 - 1.0]
    return np.stack(cols, axis=2).reshape(rho.shape[0], -1)


def embed_1d(samples, dim, axis, sign):
    """Embed 1D 5-point samples (n, 5, 3) of (rho, u, p) into d-dimensional
    stencils that are constant across the other axes: the point at offset o
    takes the sample value at index 2 + sign * o_axis, with velocity component
    `axis` equal to sign * u and the other components 0.
    Returns (rho (n, S), [u_d (n, S)], p (n, S))."""
    offs = stencil_offsets(dim)
    idx = np.array([2 + sign * o[axis] for o in offs])
    rho = samples[:, idx, 0]
    p = samples[:, idx, 2]
    u = []
    for d in range(dim):
        u.append(samples[:, idx, 1] * sign if d == axis else np.zeros_like(rho))
    return rho, u, p


def embedded_features(samples, dim, gamma):
    """All 2 d embeddings (axis x sign, axis-major, sign -1 then +1) of 1D
    samples, stacked sample-major: row 2 d i + 2 a + (s > 0)."""
    out = []
    for a in range(dim):
        for s in (-1, 1):
            rho, u, p = embed_1d(samples, dim, a, s)
            out.append(features(rho, u, p, gamma))
    X = np.stack(out, axis=1)                  # (n, 2d, K)
    return X.reshape(-1, X.shape[2])


def forward(params, X):
    """Logits and hidden activations for inputs X (n, K)."""
    a1 = X @ params['W1'].T + params['b1']
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params['W2'].T + params['b2']
    h2 = np.maximum(a2, 0.0)
    z = h2 @ params['W3'].T + params['b3']
    return z[:, 0], (h1, h2)


def softplus(x):
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def loss_and_grad(params, X, y, pw):
    """Weighted BCE of the logits (mean over samples) and its gradient."""
    n = X.shape[0]
    z, (h1, h2) = forward(params, X)
    loss = np.mean(pw * y * softplus(-z) + (1.0 - y) * softplus(z))
    sz = sigmoid(z)
    dz = (pw * y * (sz - 1.0) + (1.0 - y) * sz) / n          # (n,)
    g = {}
    g['W3'] = dz[None, :] @ h2
    g['b3'] = np.array([dz.sum()])
    dh2 = dz[:, None] * params['W3'][0][None, :]
    dh2 = dh2 * (h2 > 0.0)
    g['W2'] = dh2.T @ h1
    g['b2'] = dh2.sum(axis=0)
    dh1 = dh2 @ params['W2']
    dh1 = dh1 * (h1 > 0.0)
    g['W1'] = dh1.T @ X
    g['b1'] = dh1.sum(axis=0)
    return loss, g


ORDER = ('W1', 'b1', 'W2', 'b2', 'W3', 'b3')


def flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(vec, kin):
    shapes = {'W1': (HIDDEN, kin), 'b1': (HIDDEN,), 'W2': (HIDDEN, HIDDEN), 'b2': (HIDDEN,),
              'W3': (1, HIDDEN), 'b3': (1,)}
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.array(vec[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def adam(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) in place; state holds m, v, t."""
    state['t'] = state.get('t', 0) + 1
    t = state['t']
    for k in ORDER:
        m = state.setdefault('m_' + k, np.zeros_like(params[k]))
        v = state.setdefault('v_' + k, np.zeros_like(params[k]))
        g = grads[k]
        m[...] = b1 * m + (1.0 - b1) * g
        v[...] = b2 * v + (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def plain_flag_1d(samples, theta_rho, theta_p):
    """Plain relative-jump flag of the centre of 1D 5-point samples (n, 5, 3)."""
    out = np.zeros(samples.shape[0], dtype=bool)
    for j, th in ((0, theta_rho), (2, theta_p)):
        fm, f0, fp = samples[:, 1, j], samples[:, 2, j], samples[:, 3, j]
        out |= np.abs(fp - fm) > th * (fp + 2.0 * f0 + fm)
    return out


def cell_stencils(orc, key):
    """Primitive 5^d stencils of the band cells [-1, N]^d of a patch (ghosts must
    be filled). Returns (rho (n, S), [u_d], p, cell local indices (n, 3))."""
    from . import euler
    from .amr import G
    A = orc.U[key]
    rho, u, p, _ = euler.primitives(A, orc.dim, orc.gamma)
    N = orc.N
    dim = orc.dim
    offs = stencil_offsets(dim)
    rng = [range(-1, N + 1) if d < dim else (0,) for d in (2, 1, 0)]
    cells = [(c[2], c[1], c[0]) for c in itertools.product(*rng)]
    cz = np.array([c[2] for c in cells])
    cy = np.array([c[1] for c in cells])
    cx = np.array([c[0] for c in cells])

    def idx(o):
        iz = cz + o[2] + (G if dim == 3 else 0)
        iy = cy + o[1] + (G if dim >= 2 else 0)
        ix = cx + o[0] + G
        return iz, iy, ix

    R = np.stack([rho[idx(o)] for o in offs], axis=1)
    P = np.stack([p[idx(o)] for o in offs], axis=1)
    Us = [np.stack([u[d][idx(o)] for o in offs], axis=1) for d in range(dim)]
    return R, Us, P, np.stack([cx, cy, cz], axis=1)


def make_flagger(params, gamma, keep_margin=0.0, refine_margin=0.0):
    """A per-patch flagger for Oracle.flag_override: refine if any in-domain
    band cell [-1, N]^d has a logit > -R (R = refine_margin, 0 by default);
    with keep_margin H > R it returns (refine, keep), keep (which blocks the
    coarsening of the parent) if any such cell has a logit > -H (a hysteresis
    between refining and coarsening)."""
    def flag(orc, key):
        R, Us, P, cells = cell_stencils(orc, key)
        X = features(R, Us, P, gamma)
        z, _ = forward(params, X)
        l, c = key
        ext = orc.mesh.extent(l)
        ok = np.ones(len(z), dtype=bool)
        for d in range(orc.dim):
            if orc.periodic[d]:
                continue
            g = c[d] * orc.N + cells[:, d]
            ok &= (g >= 0) & (g < ext[d] * orc.N)
        refine = bool(np.any((z > -refine_margin) & ok))
        if keep_margin > refine_margin:
            return refine, bool(np.any((z > -keep_margin) & ok))
        return refine
    return flag


def gradient_fd(params, X, y, pw, h=1e-6, n_probe=20, seed=0):
    """Central finite differences of the loss at n_probe random parameters."""
    rng = np.random.default_rng(seed)
    vec = flatten(params)
    kin = params['W1'].shape[1]
    idx = rng.choice(vec.size, size=n_probe, replace=False)
    out = []
    for i in idx:
        vp = vec.copy()
        vm = vec.copy()
        vp[i] += h
        vm[i] -= h
        lp, _ = loss_and_grad(unflatten(vp, kin), X, y, pw)
        lm, _ = loss_and_grad(unflatten(vm, kin), X, y, pw)
        out.append((lp - lm) / (2.0 * h))
    return idx, np.array(out)


def bce_pos_weight(y):
    """Positive-class weight = negatives / positives."""
    pos = float(np.sum(y))
    return (len(y) - pos) / max(pos, 1.0)

