"""Exact solution of the 1D Riemann problem of the Euler equations (Eqs. 1-3)
for a calorically perfect gas (Eqs. 4-7). Test infrastructure.

The star pressure p* solves f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the
velocity jump across the K wave: the Rankine-Hugoniot shock relation for
p > p_K and the isentropic rarefaction relation for p <= p_K. Newton's method
from the two-rarefaction estimate; then the self-similar solution is sampled
at xi = (x - x0) / t.
"""
import math

import numpy as np


def _fK(p, rk, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (p + B))
    else:
        e = (g - 1.0) / (2.0 * g)
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0)
        df = 1.0 / (rk * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    e = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** e + cr / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(100):
        fl, dfl = _fK(p, rl, pl, cl, g)
        fr, dfr = _fK(p, rr, pr, cr, g)
        f = fl + fr + ur - ul
        pn = p - f / (dfl + dfr)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, cl, g)
    fr, _ = _fK(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def wave_structure(left, right, g):
    """Star state and wave speeds: dict with p*, u*, rho*_L, rho*_R and the
    speeds of the left wave (head, tail or shock), contact and right wave."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    out = {'p': ps, 'u': us, 'contact': us}
    gg = (g - 1.0) / (g + 1.0)
    if ps > pl:   # left shock
        out['rho_l'] = rl * (ps / pl + gg) / (gg * ps / pl + 1.0)
        out['left'] = ('shock', ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g)))
    else:
        out['rho_l'] = rl * (ps / pl) ** (1.0 / g)
        csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        out['left'] = ('rarefaction', ul - cl, us - csl)
    if ps > pr:   # right shock
        out['rho_r'] = rr * (ps / pr + gg) / (gg * ps / pr + 1.0)
        out['right'] = ('shock', ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g)))
    else:
        out['rho_r'] = rr * (ps / pr) ** (1.0 / g)
        csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
        out['right'] = ('rarefaction', us + csr, ur + cr)
    return out


def sample(left, right, g, x, x0, t):
    """(rho, u, p) of the exact solution at positions x (array) and time t > 0."""
    ws = wave_structure(left, right, g)
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for i, s in enumerate(xi.ravel()):
        if s <= ws['contact']:
            lw = ws['left']
            if lw[0] == 'shock':
                st = (rl, ul, pl) if s <= lw[1] else (ws['rho_l'], ws['u'], ws['p'])
            else:
                if s <= lw[1]:
                    st = (rl, ul, pl)
                elif s >= lw[2]:
                    st = (ws['rho_l'], ws['u'], ws['p'])
                else:
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    cc = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    rr_ = rl * (cc / cl) ** (2.0 / (g - 1.0))
                    st = (rr_, uu, pl * (cc / cl) ** (2.0 * g / (g - 1.0)))
        else:
            rw = ws['right']
            if rw[0] == 'shock':
                st = (rr, ur, pr) if s >= rw[1] else (ws['rho_r'], ws['u'], ws['p'])
            else:
                if s >= rw[2]:
                    st = (rr, ur, pr)
                elif s <= rw[1]:
                    st = (ws['rho_r'], ws['u'], ws['p'])
                else:
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    cc = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    rr_ = rr * (cc / cr) ** (2.0 / (g - 1.0))
                    st = (rr_, uu, pr * (cc / cr) ** (2.0 * g / (g - 1.0)))
        rho.flat[i], u.flat[i], p.flat[i] = st
    return rho, u, p
