"""Instrumented FLOP count of the oracle's face flux and cell update.

Test infrastructure (see ``oracle/__init__``). Runs ``euler.face_flux`` (Sec. 3.2,
Eqs. 10-12), ``euler.central_face_flux`` (Sec. 3.2, Eq. 8), the
primitive-variable conversion and the SSP-RK3 stage update on a scalar type
that counts every floating-point operation, and writes ``flop_counts.json``
beside this file. Each +, -, *, /, sqrt, |.| and max counts
as one FLOP (a fused multiply-add on the GPU performs two of them).

    python -m oracle.flopcount
"""
import json
import math
import os


class _Count:
    n = 0


class F(float):
    def _b(self, o, f):
        _Count.n += 1
        return F(f(float(self), float(o)))

    def __add__(self, o): return self._b(o, lambda a, b: a + b)
    def __radd__(self, o): return self._b(o, lambda a, b: b + a)
    def __sub__(self, o): return self._b(o, lambda a, b: a - b)
    def __rsub__(self, o): return self._b(o, lambda a, b: b - a)
    def __mul__(self, o): return self._b(o, lambda a, b: a * b)
    def __rmul__(self, o): return self._b(o, lambda a, b: b * a)
    def __truediv__(self, o): return self._b(o, lambda a, b: a / b)
    def __rtruediv__(self, o): return self._b(o, lambda a, b: b / a)
    def __neg__(self): return F(-float(self))


class _NpShim:
    """The numpy functions face_flux uses, on counted scalars."""
    @staticmethod
    def sqrt(x):
        _Count.n += 1
        return F(math.sqrt(float(x)))

    @staticmethod
    def abs(x):
        _Count.n += 1
        return F(abs(float(x)))

    @staticmethod
    def maximum(a, b):
        _Count.n += 1
        return F(max(float(a), float(b)))

    @staticmethod
    def any(x):
        return bool(x)

    @staticmethod
    def logical_not(x):
        return not x

    @staticmethod
    def where(c, a, b):
        return a if c else b


def count(dim, gamma=1.4):
    from . import euler
    saved = euler.np
    euler.np = _NpShim
    try:
        # a smooth positive pencil (no first-order fallback taken)
        P = []
        for k in range(6):
            P.append((F(1.0 + 0.01 * k), F(0.1 + 0.02 * k), [F(0.05 * k) for _ in range(dim - 1)],
                      F(1.2 - 0.01 * k)))
        _Count.n = 0
        euler.face_flux(P, dim, F(gamma))
        face = _Count.n
        _Count.n = 0
        euler.central_face_flux(P[1:5], dim, F(gamma))
        face_central = _Count.n
        # one conversion to primitives per cell
        U = [F(1.1)] + [F(0.1)] * dim + [F(2.6)]
        _Count.n = 0
        euler.primitives(U, dim, F(gamma))
        prim = _Count.n
    finally:
        euler.np = saved
    nv = dim + 2
    # divergence: per dimension and variable (F+ - F-) / dx accumulated into R
    div = dim * nv * 3
    # stage update a U0 + b (Us + dt R): 5 operations per variable
    upd = nv * 5
    # central: the conservative face value G = (26 F_f - F_{f-1} - F_{f+1}) / 24
    # of Eq. 9, 4 operations per variable on each of the N + 1 faces of a row
    return {'face': face, 'cell': prim + div + upd, 'primitives': prim, 'divergence': div, 'update': upd,
            'face_central': face_central, 'face_combine_central': nv * 4}


def main():
    out = {str(d): count(d) for d in (1, 2, 3)}
    out['note'] = ('FLOPs counted by running the oracle on a counting scalar: face = one Rusanov '
                   'face flux (characteristic WENO5-JS, Eqs. 10-12); cell = primitives + divergence + '
                   'SSP-RK3 stage update of one cell; face_central = one central face flux (Eq. 8), '
                   'N + 3 of them per row; face_combine_central = the conservative face value of '
                   'Eq. 9, N + 1 per row')
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'flop_counts.json')
    with open(path, 'w') as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == '__main__':
    main()
