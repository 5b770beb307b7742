"""Euler numerics of the oracle: EOS, characteristic variables, WENO5-JS, Rusanov.

Test infrastructure (see ``oracle/__init__``). FP64 numpy. Arrays carry the
conserved variables on their first axis: U = (rho, rho u_0 .. rho u_{d-1}, rho e)
(Sec. 3.1, Eqs. 1-3). The gas is calorically perfect with R = 1 (Sec. 6), so
T = p / rho.
"""
import numpy as np

# WENO5-JS constants (Sec. 3.2: 5-point WENO-JS nonlinear interpolation).
EPS_WENO = 1.0e-6
C13_12 = 13.0 / 12.0
D0, D1, D2 = 0.0625, 0.625, 0.3125      # linear weights (1, 10, 5) / 16


def primitives(U, dim, gamma):
    """Primitive variables from conserved ones (Sec. 3.1, Eqs. 4-6, R = 1).

    u_d = m_d / rho; p = (gamma - 1) (E - rho |u|^2 / 2); T = p / rho.
    Returns (rho, [u_0..u_{d-1}], p, T).
    """
    gm1 = gamma - 1.0
    rho = U[0]
    u = [U[1 + d] / rho for d in range(dim)]
    usq = u[0] * u[0]
    for d in range(1, dim):
        usq = usq + u[d] * u[d]
    p = gm1 * (U[dim + 1] - 0.5 * rho * usq)
    T = p / rho
    return rho, u, p, T


def conserved_from_primitive(rho, u, p, gamma):
    """U from (rho, u, p): E = p / (gamma - 1) + rho |u|^2 / 2 (Sec. 3.1, Eqs. 4, 6)."""
    gm1 = gamma - 1.0
    dim = len(u)
    usq = u[0] * u[0]
    for d in range(1, dim):
        usq = usq + u[d] * u[d]
    out = [rho]
    for d in range(dim):
        out.append(rho * u[d])
    out.append(p / gm1 + 0.5 * rho * usq)
    return out


def sound_speed(p, rho, gamma):
    """c = sqrt(gamma p / rho) (Sec. 3.1, Eq. 7)."""
    return np.sqrt(gamma * p / rho)


def weno5_left(a, b, c, d, e):
    """WENO5-JS nodal mid-point value at x_{i+1/2} from nodes i-2..i+2 (Sec. 3.2).

    Candidates are the quadratic Lagrange interpolants of the three 3-point
    sub-stencils evaluated at the mid-point; their linear combination with
    weights (1, 10, 5)/16 is the 5-point interpolant (3, -20, 90, 60, -5)/128.
    Smoothness indicators are the Jiang-Shu ones; alpha_k = d_k / (eps + beta_k)^2.
    """
    q0 = (3.0 * a - 10.0 * b + 15.0 * c) * 0.125
    q1 = (-b + 6.0 * c + 3.0 * d) * 0.125
    q2 = (3.0 * c + 6.0 * d - e) * 0.125
    t0 = a - 2.0 * b + c
    s0 = a - 4.0 * b + 3.0 * c
    t1 = b - 2.0 * c + d
    s1 = b - d
    t2 = c - 2.0 * d + e
    s2 = 3.0 * c - 4.0 * d + e
    b0 = C13_12 * (t0 * t0) + 0.25 * (s0 * s0)
    b1 = C13_12 * (t1 * t1) + 0.25 * (s1 * s1)
    b2 = C13_12 * (t2 * t2) + 0.25 * (s2 * s2)
    e0 = EPS_WENO + b0
    e1 = EPS_WENO + b1
    e2 = EPS_WENO + b2
    a0 = D0 / (e0 * e0)
    a1 = D1 / (e1 * e1)
    a2 = D2 / (e2 * e2)
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def frozen_state(p_i, T_i, p_j, T_j, gamma):
    """Frozen state of the characteristic projection at the face between nodes
    i and j = i+1 (reading of Sec. 3.2, where the projection is deferred to the
    authors' earlier work): pbar, Tbar are arithmetic means, rhobar = pbar / Tbar,
    cbar = sqrt(gamma Tbar) (R = 1). Returns (z = rhobar cbar,
    kappa = (gamma - 1) / (gamma rhobar))."""
    pbar = 0.5 * (p_i + p_j)
    Tbar = 0.5 * (T_i + T_j)
    rbar = pbar / Tbar
    cbar = np.sqrt(gamma * Tbar)
    z = rbar * cbar
    kap = (gamma - 1.0) / (gamma * rbar)
    return z, kap


def char_forward(q, z, kap):
    """Characteristic fields of a node q = (p, un, ut, T) of the linearised
    primitive system in (p, u, T): [p - z un, T - kappa p, ut..., p + z un]
    (left eigenvectors for speeds u - c, u, u..., u + c)."""
    p, un, ut, T = q
    return [p - z * un, T - kap * p] + list(ut) + [p + z * un]


def char_inverse(w, z, kap):
    """Inverse of char_forward: p = (w1 + w5)/2, un = (w5 - w1)/(2 z),
    T = w2 + kappa p, ut = w_t. Returns (p, un, ut, T)."""
    nf = len(w)
    p = 0.5 * (w[0] + w[nf - 1])
    un = (w[nf - 1] - w[0]) / (2.0 * z)
    T = w[1] + kap * p
    return p, un, list(w[2:nf - 1]), T


def hllc(left, right, nt):
    """HLLC flux (Toro's three-wave approximate Riemann solver: the HLL
    fan split at the contact) from the two face states. Each side is a dict
    with rho, un, ut (list), p, E, c and U, F in pencil order. Wave-speed
    bounds S_L = min(un_L - c_L, un_R - c_R), S_R = max(un_L + c_L, un_R + c_R);
    contact speed S* = (p_R - p_L + a_L un_L - a_R un_R) / (a_L - a_R) with
    a_K = rho_K (S_K - un_K); star state U*_K = f_K (1, S*, ut_K, E_K / rho_K +
    (S* - un_K)(S* + p_K / a_K)), f_K = a_K / (S_K - S*); flux F_L if S_L >= 0,
    else F_L + S_L (U*_L - U_L) if S* >= 0, else F_R + S_R (U*_R - U_R) if
    S_R > 0, else F_R."""
    L, R = left, right
    sL = np.minimum(L['un'] - L['c'], R['un'] - R['c'])
    sR = np.maximum(L['un'] + L['c'], R['un'] + R['c'])
    aL = L['rho'] * (sL - L['un'])
    aR = R['rho'] * (sR - R['un'])
    sM = (R['p'] - L['p'] + aL * L['un'] - aR * R['un']) / (aL - aR)

    def star_flux(K, a, s):
        f = a / (s - sM)
        Us = [f, f * sM] + [f * K['ut'][j] for j in range(nt)] + \
             [f * (K['E'] / K['rho'] + (sM - K['un']) * (sM + K['p'] / a))]
        return [K['F'][v] + s * (Us[v] - K['U'][v]) for v in range(nt + 3)]

    FsL = star_flux(L, aL, sL)
    FsR = star_flux(R, aR, sR)
    return [np.where(sL >= 0.0, L['F'][v],
                     np.where(sM >= 0.0, FsL[v], np.where(sR > 0.0, FsR[v], R['F'][v])))
            for v in range(nt + 3)]


def face_flux(P, dim, gamma, flux='rusanov'):
    """Rusanov flux at the face between pencil nodes 2 and 3 (Sec. 3.2, Eqs. 11-12).

    P is a list of 6 pencil nodes (i-2 .. i+3), each a tuple (p, un, ut, T) where
    un is the velocity normal to the face and ut is the list of tangential
    velocities in increasing dimension order. Arrays broadcast over faces.

    Steps:
      1. frozen state at the face: pbar, Tbar (arithmetic means of nodes i, i+1),
         rhobar = pbar / Tbar, cbar = sqrt(gamma Tbar), z = rhobar cbar,
         kappa = (gamma - 1) / (gamma rhobar);
      2. characteristic variables of the linearised primitive system in (p, u, T):
         w1 = p - z un (speed u - c), w2 = T - kappa p (speed u),
         w_t = ut (speed u), w5 = p + z un (speed u + c);
      3. left- and right-biased WENO5-JS interpolation of each field;
      4. back to p = (w1 + w5) / 2, un = (w5 - w1) / (2 z), T = w2 + kappa p,
         with a first-order fallback (nodes i, i+1) if p or T is not positive;
      5. conserved states and Euler fluxes at both sides, S = max(c + |un|) and
         F = (F^R + F^L)/2 - S (U^R - U^L)/2.
    With flux='hllc', step 5 uses the HLLC flux of `hllc` from the same states
    instead (an option the method leaves open; not in the paper).
    Returns the flux in pencil order (mass, normal momentum, tangential momenta,
    energy).
    """
    gm1 = gamma - 1.0
    nt = dim - 1
    p2, un2, ut2, T2 = P[2]
    p3, un3, ut3, T3 = P[3]
    z, kap = frozen_state(p2, T2, p3, T3, gamma)
    W = [char_forward(P[k], z, kap) for k in range(6)]
    nf = nt + 3
    wl = [weno5_left(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f]) for f in range(nf)]
    wr = [weno5_left(W[5][f], W[4][f], W[3][f], W[2][f], W[1][f]) for f in range(nf)]
    pL, unL, utL, TL = char_inverse(wl, z, kap)
    pR, unR, utR, TR = char_inverse(wr, z, kap)
    bad = np.logical_not((pL > 0.0) & (TL > 0.0) & (pR > 0.0) & (TR > 0.0))
    if np.any(bad):
        pL = np.where(bad, p2, pL)
        unL = np.where(bad, un2, unL)
        TL = np.where(bad, T2, TL)
        utL = [np.where(bad, ut2[j], utL[j]) for j in range(nt)]
        pR = np.where(bad, p3, pR)
        unR = np.where(bad, un3, unR)
        TR = np.where(bad, T3, TR)
        utR = [np.where(bad, ut3[j], utR[j]) for j in range(nt)]

    def side(p, un, ut, T):
        rho = p / T
        c = np.sqrt(gamma * T)
        usq = un * un
        for j in range(nt):
            usq = usq + ut[j] * ut[j]
        E = p / gm1 + 0.5 * rho * usq
        mn = rho * un
        U = [rho, mn] + [rho * ut[j] for j in range(nt)] + [E]
        F = [mn, mn * un + p] + [mn * ut[j] for j in range(nt)] + [(E + p) * un]
        s = c + np.abs(un)
        return U, F, s, dict(rho=rho, un=un, ut=ut, p=p, E=E, c=c, U=U, F=F)

    UL, FL, sL, left = side(pL, unL, utL, TL)
    UR, FR, sR, right = side(pR, unR, utR, TR)
    if flux == 'hllc':
        return hllc(left, right, nt)
    hS = 0.5 * np.maximum(sR, sL)
    return [0.5 * (FR[v] + FL[v]) - hS * (UR[v] - UL[v]) for v in range(dim + 2)]


def central_mid(a, b, c, d):
    """4th-order central mid-point value at x_{i+1/2} from nodes i-1 .. i+2
    (Sec. 3.2, Eq. 8, read with the node and edge roles the other way round:
    the printed form gives a node value from edge values):
    (9 (phi_i + phi_{i+1}) - (phi_{i-1} + phi_{i+2})) / 16, exact for cubics."""
    return (9.0 * (b + c) - (a + d)) * 0.0625


def central_face_flux(P, dim, gamma):
    """Shock-free face flux (Sec. 3.2: central mid-point interpolation of the
    primitive set p, T, u_j, then the flux assembled at the edge point).

    P is a list of 4 pencil nodes (i-1 .. i+2), each a tuple (p, un, ut, T) as
    in `face_flux`. Each of p, un, ut, T is interpolated with `central_mid`; if
    p or T is not positive there, the face takes the mean of nodes i and i+1
    (a guard the paper leaves open). The flux is the Euler flux of that single
    edge state: no upwinding and no dissipation. Returns it in pencil order.
    """
    gm1 = gamma - 1.0
    nt = dim - 1
    p = central_mid(P[0][0], P[1][0], P[2][0], P[3][0])
    un = central_mid(P[0][1], P[1][1], P[2][1], P[3][1])
    ut = [central_mid(P[0][2][j], P[1][2][j], P[2][2][j], P[3][2][j]) for j in range(nt)]
    T = central_mid(P[0][3], P[1][3], P[2][3], P[3][3])
    bad = np.logical_not((p > 0.0) & (T > 0.0))
    if np.any(bad):
        p = np.where(bad, 0.5 * (P[1][0] + P[2][0]), p)
        un = np.where(bad, 0.5 * (P[1][1] + P[2][1]), un)
        ut = [np.where(bad, 0.5 * (P[1][2][j] + P[2][2][j]), ut[j]) for j in range(nt)]
        T = np.where(bad, 0.5 * (P[1][3] + P[2][3]), T)
    rho = p / T
    usq = un * un
    for j in range(nt):
        usq = usq + ut[j] * ut[j]
    E = p / gm1 + 0.5 * rho * usq
    mn = rho * un
    return [mn, mn * un + p] + [mn * ut[j] for j in range(nt)] + [(E + p) * un]


def hybrid_face_flux(P, dim, gamma, theta):
    """Per-face choice between the shock-free central scheme and the
    shock-capturing one (Sec. 3.2: the central schemes are for flows without
    shocks, characteristic WENO5 with the Rusanov flux for flows with them; the
    switch between them face by face is this build's extension).

    P is the 6-node pencil i-2 .. i+3 of `face_flux`. Shock sensor: the
    relative jump of the refinement criterion, |phi_{k+1} - phi_{k-1}| >
    theta (phi_{k+1} + 2 phi_k + phi_{k-1}) for phi in (rho = p / T, p),
    tested along the pencil at the four nodes k = i-1 .. i+2 whose neighbours
    lie in the pencil. Where no node trips it, the face takes the central
    scheme's conservative face value G_{i+1/2} = (26 F_{i+1/2} - F_{i-1/2} -
    F_{i+3/2}) / 24 of Eq. 9 (the central face fluxes from nodes i-1..i+2,
    i-2..i+1 and i..i+3); elsewhere the WENO5 + Rusanov flux of `face_flux`.
    Either way the face carries one value, so the divergence stays a difference
    of face values (conservative), and both need only nodes i-2 .. i+3.
    Returns the face value in pencil order and the boolean `smooth` mask.
    """
    rho = [P[k][0] / P[k][3] for k in range(6)]
    shock = None
    for phi in (rho, [P[k][0] for k in range(6)]):
        for k in range(1, 5):
            s = np.abs(phi[k + 1] - phi[k - 1]) > theta * (phi[k + 1] + 2.0 * phi[k] + phi[k - 1])
            shock = s if shock is None else (shock | s)
    smooth = np.logical_not(shock)
    Fm = central_face_flux(P[1:5], dim, gamma)
    Fl = central_face_flux(P[0:4], dim, gamma)
    Fh = central_face_flux(P[2:6], dim, gamma)
    Gc = [(26.0 * Fm[v] - Fl[v] - Fh[v]) / 24.0 for v in range(dim + 2)]
    Fw = face_flux(P, dim, gamma, 'rusanov')
    return [np.where(smooth, Gc[v], Fw[v]) for v in range(dim + 2)], smooth


def pencil_to_global(F, dim, d):
    """Map a flux in pencil order (mass, normal, tangentials, energy) back to
    the global order (mass, m_0 .. m_{d-1}, energy) for a face normal to d."""
    tdims = [e for e in range(dim) if e != d]
    out = [None] * (dim + 2)
    out[0] = F[0]
    out[1 + d] = F[1]
    for j, e in enumerate(tdims):
        out[1 + e] = F[2 + j]
    out[dim + 1] = F[dim + 1]
    return out


def patch_rhs(A, dim, N, g, dx, gamma, flux='rusanov', theta_switch=0.05):
    """Right-hand side R = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d on a patch interior
    (Sec. 3.2, Eq. 10: divergence of the Riemann fluxes; dims in order x, y, z).

    With flux='central' (the shock-free schemes of Sec. 3.2) the face fluxes
    come from `central_face_flux` at faces i-3/2 .. N+1/2 and the divergence is
    the 4th-order staggered difference of Eq. 9,
    (27 (F_{i+1/2} - F_{i-1/2}) - (F_{i+3/2} - F_{i-3/2})) / (24 dx), evaluated
    in its conservative form: the difference of the face values
    G_{i+1/2} = (26 F_{i+1/2} - F_{i-1/2} - F_{i+3/2}) / 24, so that sums over
    patches telescope and the coarse-fine correction acts on G.

    With flux='hybrid' every face i+1/2 (i = -1 .. N-1) takes the value of
    `hybrid_face_flux` with threshold theta_switch: the central G where the
    shock sensor is quiet, the WENO5 + Rusanov flux elsewhere.

    A: slot array (nv, Z, Y, X) with g ghost layers in every active dimension
    (array axis 3 - d holds dimension d). Returns (R, faces) where R has the
    interior shape (nv, [N]*dim reversed) and faces[d] = (F_low, F_high): the
    fluxes on the low (index 0) and high (index N) boundary faces of dimension d,
    in global variable order, each of shape (nv, interior transverse shape).
    """
    rho, u, p, T = primitives(A, dim, gamma)
    nv = dim + 2
    inner = [slice(None)] * 4
    for d in range(dim):
        inner[3 - d] = slice(g, g + N)
    R = None
    faces = {}
    for d in range(dim):
        ax = 3 - d
        tdims = [e for e in range(dim) if e != d]
        P = []
        if flux == 'central':
            for k in range(4):
                sl = list(inner)
                sl[ax] = slice(k, k + N + 3)   # faces i+1/2, i = -2..N (nodes i-1..i+2)
                sl = tuple(sl[1:])
                P.append((p[sl], u[d][sl], [u[e][sl] for e in tdims], T[sl]))
            Fc = np.stack(pencil_to_global(central_face_flux(P, dim, gamma), dim, d))
            mid = [slice(None)] * 4
            below = [slice(None)] * 4
            above = [slice(None)] * 4
            mid[ax] = slice(1, N + 2)
            below[ax] = slice(0, N + 1)
            above[ax] = slice(2, N + 3)
            F = (26.0 * Fc[tuple(mid)] - Fc[tuple(below)] - Fc[tuple(above)]) / 24.0
        else:
            for k in range(6):
                sl = list(inner)
                sl[ax] = slice(k, k + N + 1)   # faces i+1/2, i = -1..N-1
                sl = tuple(sl[1:])
                P.append((p[sl], u[d][sl], [u[e][sl] for e in tdims], T[sl]))
            if flux == 'hybrid':
                Fp, _ = hybrid_face_flux(P, dim, gamma, theta_switch)
            else:
                Fp = face_flux(P, dim, gamma, flux)
            F = pencil_to_global(Fp, dim, d)
            F = np.stack(F)                      # (nv, ..., N+1 along ax)
        hi = [slice(None)] * 4
        lo = [slice(None)] * 4
        hi[ax] = slice(1, N + 1)
        lo[ax] = slice(0, N)
        div = (F[tuple(hi)] - F[tuple(lo)]) / dx[d]
        R = -div if R is None else R - div
        f_lo = [slice(None)] * 4
        f_hi = [slice(None)] * 4
        f_lo[ax] = 0
        f_hi[ax] = N
        faces[d] = (F[tuple(f_lo)].copy(), F[tuple(f_hi)].copy())
    assert R.shape[0] == nv
    return R, faces
