"""One segregated time step of the VOF evaporating-droplet method (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The stage order is the paper's (Sec. 3.1, Fig. Scheme):
  S0 thermodynamics at T^n: saturation (Sec. 2.5), liquid pinned to Y_eq,
     gas density (Eq. densitygas)
  S1 evaporation flux: interface cells, adjacent gas cell along the normal,
     total flux j = j_d + j_c (Eqs. 9-13), m_raw = -j . grad(alpha) (Eq. massflux),
     K normalisation and f(alpha) = sqrt(alpha(1-alpha)) (Eq. alphafunction)
  S2 alpha source (Eq. alphasource), constant rho_L
  S3 alpha advection (Eq. advection): upwind + compressive high-order flux with
     a Zalesak (FCT) limiter, replacing isoAdvector
  S4 mixture properties (Sec. 2.7)
  S5 energy (Eq. Teqn), S6 species (Eq. speciesequation)
  S7 momentum predictor with the centripetal force (Eq. NavierStokesModified)
  S8-S10 pressure equation with the Stefan source (Eq. pequation), velocity
     correction
  S11 diagnostics
Linear systems are assembled as sparse matrices and solved with a direct
factorisation.

Parity unpinned: the interface-cell threshold on |grad(alpha)| and the adjacent
gas-cell threshold ALPHA_GAS (the paper gives neither number), and the coupled
dynamics of the 3D forced-convection case with an evaporating Peng-Robinson droplet
beyond its invariants (its thermodynamics, its flow without a droplet and its
conservation properties have pins); these rest on the comparison with the CUDA path
alone.  Every other stage has a pin in the tests.  Discrete readings of points the paper leaves open are listed in
the repository's design notes; the code states each where it is used.
"""
import math
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid, AXIS, WALL, OPEN, FORCED
from . import plic
from . import thermo as th

PHYS_EVAP, PHYS_ENERGY, PHYS_SPECIES, PHYS_FLOW = 1, 2, 4, 8
FLAG_NO_INTERFACE, FLAG_MDOT_CAPPED, FLAG_ALPHA_CLIPPED, FLAG_ADJ_NOT_FOUND, FLAG_BOILING = 1, 2, 4, 8, 16
ALPHA_GAS = 1e-3          # adjacent gas cell threshold (reading R11)
W = 2                     # ghost layers used by the padded views


# ============================================================ padded views

def _pad(G, core):
    pw = [(W, W) if a in G.act else (0, 0) for a in range(3)]
    return np.pad(core, pw)


def _view(G, P, core_shape, shifts=None):
    """View of padded array P with the given core shape, offset by shifts[a]."""
    shifts = shifts or {}
    sl = []
    for a in range(3):
        if a in G.act:
            o = W + shifts.get(a, 0)
            sl.append(slice(o, o + core_shape[a]))
        else:
            sl.append(slice(0, core_shape[a]))
    return P[tuple(sl)]


def _slab(G, core_shape, a, pidx):
    """Index tuple: padded index pidx along a, the core range along other axes."""
    sl = []
    for b in range(3):
        if b == a:
            sl.append(slice(pidx, pidx + 1))
        elif b in G.act:
            sl.append(slice(W, W + core_shape[b]))
        else:
            sl.append(slice(0, core_shape[b]))
    return tuple(sl)


def _face_slab(arr, a, idx):
    sl = [slice(None)] * 3
    sl[a] = slice(idx, idx + 1)
    return arr[tuple(sl)]


def _outward_vel(G, u, a, side):
    """Outward normal velocity on the boundary faces of side 0 (low) or 1 (high)."""
    if side == 0:
        return -_face_slab(u[a], a, 0)
    return _face_slab(u[a], a, G.n[a])


def pad_scalar(G, phi, rule, u=None, amb=0.0):
    """Cell field with two ghost layers filled by the boundary rule.

    rule 'alpha': mirror at the axis, alpha = 0 outside every other boundary.
    rule 'zg'   : zero gradient everywhere (mirror at the axis).
    rule 'TO'   : temperature / species (Table tableboundary): axis mirror,
                  wall zero gradient, forced inlet fixed value amb, open
                  boundary inletOutlet (fixed amb where the boundary face
                  velocity points into the domain, zero gradient otherwise).
    A fixed face value amb gives the ghost 2 amb - phi_b; both ghost layers get
    the same value (the second layer only feeds boundary faces, whose
    high-order values are never used).
    """
    n = G.n
    P = _pad(G, phi)
    for a in G.act:
        for side in (0, 1):
            kind = G.bc[a][side]
            bidx = W if side == 0 else W + n[a] - 1
            inner = P[_slab(G, n, a, bidx)]
            if rule == "alpha":
                g = inner.copy() if kind == AXIS else np.zeros_like(inner)
            elif rule == "zg":
                g = inner.copy()
            else:
                if kind in (AXIS, WALL):
                    g = inner.copy()
                elif kind == FORCED:
                    g = 2.0 * amb - inner
                else:
                    vout = _outward_vel(G, u, a, side)
                    g = np.where(vout < 0.0, 2.0 * amb - inner, inner)
            for layer in (1, 2):
                pidx = bidx - layer if side == 0 else bidx + layer
                P[_slab(G, n, a, pidx)] = g
    return P


def pad_velocity(G, u, c, u_in):
    """Face velocity u_c with two ghost layers on every active axis.

    Along its own axis (beyond the boundary face, value u_b):
      axis / wall / forced inlet: u(-k) = 2 u_b - u(k)   (odd about the face)
      open boundary:              u(-k) = u_b             (zero gradient)
    Along a tangential axis (beyond the boundary cells):
      wall / forced inlet (no slip / fixed zero tangential velocity): u(-k) = -u(k-1)
      axis (u_z is even about r = 0):                                  u(-k) = u(k-1)
      open boundary:                                                   u(-k) = u(0)
    """
    shp = list(G.n)
    shp[c] += 1
    P = _pad(G, u)
    for a in G.act:
        m = shp[a]
        for side in (0, 1):
            kind = G.bc[a][side]
            for k in (1, 2):
                if a == c:
                    if side == 0:
                        ub = P[_slab(G, shp, a, W)]
                        uk = P[_slab(G, shp, a, W + k)]
                        val = ub.copy() if kind == OPEN else 2.0 * ub - uk
                        P[_slab(G, shp, a, W - k)] = val
                    else:
                        ub = P[_slab(G, shp, a, W + m - 1)]
                        uk = P[_slab(G, shp, a, W + m - 1 - k)]
                        val = ub.copy() if kind == OPEN else 2.0 * ub - uk
                        P[_slab(G, shp, a, W + m - 1 + k)] = val
                else:
                    if side == 0:
                        src = P[_slab(G, shp, a, W + k - 1)]
                        first = P[_slab(G, shp, a, W)]
                        if kind in (WALL, FORCED):
                            val = -src
                        elif kind == AXIS:
                            val = src.copy()
                        else:
                            val = first.copy()
                        P[_slab(G, shp, a, W - k)] = val
                    else:
                        src = P[_slab(G, shp, a, W + m - k)]
                        last = P[_slab(G, shp, a, W + m - 1)]
                        if kind in (WALL, FORCED):
                            val = -src
                        elif kind == AXIS:
                            val = src.copy()
                        else:
                            val = last.copy()
                        P[_slab(G, shp, a, W + m - 1 + k)] = val
    return P


def fshape(G, a):
    """Shape of a face array of direction a (n_a + 1 faces along a)."""
    s = list(G.n)
    s[a] += 1
    return tuple(s)


# ============================================================ small formulas

def minmod(x, y):
    """minmod(x, y): the smaller magnitude when x and y share a sign, else 0."""
    return np.where(x * y > 0.0, np.sign(x) * np.minimum(np.abs(x), np.abs(y)), 0.0)


def lim_upwind(uu, u, d):
    """Linear-upwind face value limited by minmod (TVD): u + 1/2 minmod(u-uu, d-u)."""
    return u + 0.5 * minmod(u - uu, d - u)


def van_leer(uu, u, d):
    """Van Leer limited upwind face value u + dU dD/(dU + dD) when dU dD > 0."""
    dU = u - uu
    dD = d - u
    prod = dU * dD
    with np.errstate(divide="ignore", invalid="ignore"):
        corr = np.where(prod > 0.0, prod / (dU + dD), 0.0)
    return u + corr


def props(cfg, alpha, rhoG, omega, T, solid=None):
    """Mixture properties chi = alpha chi_L + (1 - alpha) chi_G (Sec. 2.7), the liquid
    density at the cell's temperature (rho_L(T), reading R31).  The fibre's cells
    conduct and diffuse nothing (k = D = 0: no flux of T or omega across the sphere,
    reading R32)."""
    a = alpha
    rho = a * th.rho_liquid(cfg, T) + (1.0 - a) * rhoG
    mu = a * cfg["mu_l"] + (1.0 - a) * cfg["mu_g"]
    k = a * cfg["k_l"] + (1.0 - a) * cfg["k_g"]
    cpG = omega * cfg["cp_v"] + (1.0 - omega) * cfg["cp_g"]
    cp = a * cfg["cp_l"] + (1.0 - a) * cpG
    D = a * cfg["D_l"] + (1.0 - a) * th.D_gas(cfg)
    if solid is not None:
        k = np.where(solid, 0.0, k)
        D = np.where(solid, 0.0, D)
    return dict(rho=rho, mu=mu, k=k, cp=cp, D=D)


def xi_field(cfg, G):
    """Centripetal potential xi = xi0 D_f / (2 r) (Eq. magneticpotential), r the
    distance to the fibre centre, capped below at D_f (reading R2)."""
    X = np.meshgrid(G.xc[0], G.xc[1], G.xc[2], indexing="ij")
    d2 = np.zeros(G.n)
    for a in G.act:
        d2 = d2 + (X[a] - cfg["xc"][a]) ** 2
    r = np.sqrt(d2)
    Df = cfg["fiber_radius"]
    return cfg["xi0"] * Df / (2.0 * np.maximum(r, Df))


# ============================================================ linear systems

def solve_box(shape, diag, coup, rhs):
    """Solve the SPD system  diag_P x_P + sum_pairs c (x_P - x_Q) = rhs  exactly.

    coup[a] has shape with shape[a] - 1 entries along a: the coupling between
    unknowns m and m + e_a.  Direct sparse factorisation (scipy SuperLU).
    """
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape, order="F")
    rows, cols, vals = [], [], []
    dtot = diag.astype(np.float64).copy()
    for a, c in coup.items():
        if c is None or shape[a] < 2:
            continue
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[a] = slice(0, shape[a] - 1)
        sl_hi[a] = slice(1, shape[a])
        i0 = idx[tuple(sl_lo)].ravel(order="F")
        i1 = idx[tuple(sl_hi)].ravel(order="F")
        cv = c.ravel(order="F")
        dtot[tuple(sl_lo)] += c
        dtot[tuple(sl_hi)] += c
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-cv, -cv]
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(dtot.ravel(order="F"))
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    x = spla.spsolve(A, rhs.ravel(order="F"))
    return x.reshape(shape, order="F")


def box_apply(shape, diag, coup, x):
    """The same operator applied to x (used by tests and diagnostics)."""
    y = diag * x
    for a, c in coup.items():
        if c is None or shape[a] < 2:
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        lo, hi = tuple(lo), tuple(hi)
        d = x[lo] - x[hi]
        y[lo] += c * d
        y[hi] -= c * d
    return y


# ============================================================ initial state

def init_state(cfg):
    """Initial fields (Sec. 3.3, Fig. initialconditions), reading R3:
    alpha = fraction of S^d sub-cell sample points inside the sphere of
    diameter D0 (S = 16 in 2D, 8 in 3D); T from the steady spherical conduction
    profile around the droplet (conduction_profile); omega = Y_eq(T) where
    alpha >= 1/2, else the quasi-steady spherical Stefan profile from
    Y_s = Y_eq(T_drop) at r_s to 0 at R (stefan_profile; R = 2 D0, or 4 mm in
    the constant-property check); u = 0, p_rgh = 0."""
    G = Grid(cfg)
    S = 16 if G.axisym else 8
    R2 = (0.5 * cfg["D0"]) * (0.5 * cfg["D0"])
    frac = (np.arange(S) + 0.5) / S
    count = np.zeros(G.n)
    # sample coordinates (i + frac) * h, squared distance summed axis by axis
    subs = []
    for a in range(3):
        if a in G.act:
            pos = (np.arange(G.n[a])[:, None] + frac[None, :]) * G.h[a]      # [n_a, S]
            subs.append((pos - cfg["xc"][a]) ** 2)
        else:
            subs.append(None)
    if G.axisym:
        d2 = subs[0][:, None, :, None] + subs[1][None, :, None, :]          # [n0, n1, S, S]
        count[:, :, 0] = (d2 <= R2).sum(axis=(2, 3))
        alpha = count / (S * S)
    else:
        for k in range(G.n[2]):
            d2 = (subs[0][:, None, :, None, None] + subs[1][None, :, None, :, None]) + subs[2][k][None, None, None, None, :]
            count[:, :, k] = (d2 <= R2).sum(axis=(2, 3, 4))
        alpha = count / (S ** 3)
    if cfg["const_props_check"]:
        T = np.full(G.n, cfg["T_drop"])
    else:
        T = conduction_profile(cfg, G)
    if cfg["T_perturb"] != 0.0:
        T = T * (1.0 + cfg["T_perturb"] * perturbation(cfg, G))
    yeq = th.Y_eq(cfg, T)
    Ys = float(th.Y_eq(cfg, np.array([cfg["T_drop"]]))[0])
    R_inf = 4e-3 if cfg["const_props_check"] else 2.0 * cfg["D0"]
    omega = np.where(alpha >= 0.5, yeq, stefan_profile(cfg, G, Ys, R_inf))
    solid = solid_mask(cfg, G)
    if solid is not None:        # the fibre: no liquid, the liquid's initial temperature, no vapour
        alpha = np.where(solid, 0.0, alpha)
        T = np.where(solid, cfg["T_drop"], T)
        omega = np.where(solid, 0.0, omega)
    u = [np.zeros(fshape(G, a)) if a in G.act else None for a in range(3)]
    if G.bc[G.s][0] == FORCED:
        _face_slab(u[G.s], G.s, 0)[...] = cfg["u_inflow"]
    st = dict(alpha=alpha, T=T, omega=omega, p=np.zeros(G.n), u=u,
              t=0.0, step=0, vap_out_cum=0.0, clip_mass=0.0, flags=0)
    st["dt"] = courant_dt(cfg, G, u)
    st["rhoG"] = th.rho_gas(cfg, T, omega)
    return st


def _dist_centre(cfg, G):
    X = np.meshgrid(G.xc[0], G.xc[1], G.xc[2], indexing="ij")
    d2 = np.zeros(G.n)
    for a in G.act:
        d2 = d2 + (X[a] - cfg["xc"][a]) ** 2
    return np.sqrt(d2)


def solid_mask(cfg, G):
    """The spherical fibre's cells (Sec. 3.1.1 and Table tableboundary, "sphere" row;
    reading R32): with cfg["fiber"] = 1, every cell whose centre lies closer than D_f
    (cfg["fiber_radius"]) to the droplet centre is solid (a staircase sphere); None
    without a fibre."""
    if not cfg.get("fiber", 0):
        return None
    return _dist_centre(cfg, G) < cfg["fiber_radius"]


def conduction_profile(cfg, G):
    """Initial temperature: T_drop inside the sphere r <= r_s = D0/2, the steady
    spherical conduction profile T_amb + (T_drop - T_amb)(1/r - 1/R)/(1/r_s - 1/R)
    for r_s < r < R = 2 D0, T_amb beyond (cell-centre distance r)."""
    r = _dist_centre(cfg, G)
    rs = 0.5 * cfg["D0"]
    Rf = 2.0 * cfg["D0"]
    w = (1.0 / np.maximum(r, rs) - 1.0 / Rf) / (1.0 / rs - 1.0 / Rf)
    w = np.clip(w, 0.0, 1.0)
    return cfg["T_amb"] + (cfg["T_drop"] - cfg["T_amb"]) * w


def perturbation(cfg, G):
    """u_i in [-1, 1): 2 (splitmix64(seed xor i) >> 11) 2^-53 - 1, i the linear cell index."""
    m = (1 << 64) - 1
    out = np.empty(G.ncell())
    seed = int(cfg["seed"]) & m
    for i in range(G.ncell()):
        z = ((seed ^ i) + 0x9E3779B97F4A7C15) & m
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        z = z ^ (z >> 31)
        out[i] = 2.0 * ((z >> 11) * (1.0 / (1 << 53))) - 1.0
    return out.reshape(G.n, order="F")


def stefan_profile(cfg, G, Ys, R_inf):
    """Quasi-steady spherical Stefan profile of the vapour mass fraction:
    ln(1-Y) = ln(1-Ys) (1/r - 1/R_inf)/(1/r_s - 1/R_inf) for r_s < r < R_inf,
    Y = Ys for r <= r_s, 0 beyond R_inf (cell-centre distance r)."""
    r = _dist_centre(cfg, G)
    rs = 0.5 * cfg["D0"]
    with np.errstate(divide="ignore"):
        w = (1.0 / np.maximum(r, rs) - 1.0 / R_inf) / (1.0 / rs - 1.0 / R_inf)
    Y = 1.0 - np.exp(np.log(1.0 - Ys) * np.clip(w, 0.0, 1.0))
    return np.where(r >= R_inf, 0.0, Y)


# ============================================================ stages

def thermo_pin(cfg, G, alpha, T, omega):
    """S0: saturation value written into the liquid (alpha >= 1/2), gas density."""
    yeq = th.Y_eq(cfg, T)
    omega = np.where(alpha >= 0.5, yeq, omega)
    rhoG = th.rho_gas(cfg, T, omega)
    return omega, rhoG


def grad_central(G, P, core=None, solid=None):
    """Central-difference gradient of a padded cell field (inactive axes: 0).  With a
    solid mask, a neighbour inside the fibre takes the cell's own value (zero gradient
    across the sphere, reading R32)."""
    n = G.n
    if solid is not None:
        Ps = _pad(G, solid)
        c0 = _view(G, P, n)
    g = []
    for a in range(3):
        if a in G.act:
            hi = _view(G, P, n, {a: 1})
            lo = _view(G, P, n, {a: -1})
            if solid is not None:
                hi = np.where(_view(G, Ps, n, {a: 1}), c0, hi)
                lo = np.where(_view(G, Ps, n, {a: -1}), c0, lo)
            g.append((hi - lo) / (2.0 * G.h[a]))
        else:
            g.append(np.zeros(n))
    return g


def cell_velocity(G, u):
    """Cell-centred velocity: average of the two faces along each axis."""
    out = []
    for a in range(3):
        if a in G.act:
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[a] = slice(0, G.n[a])
            hi[a] = slice(1, G.n[a] + 1)
            out.append(0.5 * (u[a][tuple(lo)] + u[a][tuple(hi)]))
        else:
            out.append(np.zeros(G.n))
    return out


def evaporation_flux(cfg, G, alpha, omega, rhoG, u, T):
    """S1: Eqs. (9)-(17).

    grad(alpha) by central differences; interface cells |grad alpha| > 1e-8/h_min
    (reading R10); n = -grad(alpha)/|grad(alpha)| points out of the liquid; the
    adjacent gas cell is the first cell hit at distances h_min, 2 h_min, 3 h_min
    along n with alpha < 1e-3 (reading R11; r mirrored at the axis, the march
    stops at the domain edge).  j = -rho D grad(omega) + rho omega v at that
    cell; m_raw = -j . grad(alpha) (reading R12); K = sum(m_raw V)/sum(f m_raw V),
    m = K f(alpha) m_raw with f = sqrt(alpha (1 - alpha)).
    Returns (mdot, mdot_raw, adj, K, flags).
    """
    n = G.n
    flags = 0
    solid = solid_mask(cfg, G)
    Pa = pad_scalar(G, alpha, "alpha")
    g = grad_central(G, Pa, solid=solid)
    gm = np.sqrt(sum(g[a] * g[a] for a in G.act))
    iface = gm > 1e-8 / G.hmin
    if solid is not None:
        iface &= ~solid
    # total flux j at every cell (only gathered at adjacent cells)
    pr = props(cfg, alpha, rhoG, omega, T, solid)
    Pw = pad_scalar(G, omega, "TO", u=u, amb=0.0)
    gw = grad_central(G, Pw, solid=solid)
    vc = cell_velocity(G, u)
    j = [(-pr["rho"] * pr["D"] * gw[a] + pr["rho"] * omega * vc[a]) if a in G.act else None for a in range(3)]
    mraw = np.zeros(n)
    adj = np.full(n, -1, dtype=np.int64)
    I = np.argwhere(iface)
    for (i0, i1, i2) in I:
        idx = (i0, i1, i2)
        nh = [-g[a][idx] / gm[idx] if a in G.act else 0.0 for a in range(3)]
        found = None
        for s in (1, 2, 3):
            q = [0, 0, 0]
            inside = True
            for a in G.act:
                xi = (idx[a] + 0.5) + (s * (G.hmin / G.h[a])) * nh[a]
                if G.axisym and a == 0:
                    xi = abs(xi)
                qa = math.floor(xi)
                if qa < 0 or qa >= n[a]:
                    inside = False
                    break
                q[a] = qa
            if not inside:
                break
            q = tuple(q)
            if solid is not None and solid[q]:
                continue                  # the march passes over the fibre's cells
            if alpha[q] < ALPHA_GAS:
                found = q
                break
        if found is None:
            flags |= FLAG_ADJ_NOT_FOUND
            continue
        adj[idx] = G.lin(*found)
        mraw[idx] = -sum(j[a][found] * g[a][idx] for a in G.act)
    f = np.sqrt(alpha * (1.0 - alpha))
    s1 = float(np.sum(mraw * G.V))
    s2 = float(np.sum(f * mraw * G.V))
    if abs(s2) < 1e-300:
        K = 0.0
        flags |= FLAG_NO_INTERFACE
        mdot = np.zeros(n)
    else:
        K = s1 / s2
        mdot = K * f * mraw
    return mdot, mraw, adj, K, flags


def alpha_source(cfg, alpha, mdot, dt, rhoL=None, expand=None):
    """S2: Eq. (alphasource), d(alpha)/dt = -mdot/rho_L - (alpha/rho_L) D(rho_L)/Dt, mdot
    capped at rho_L alpha/dt.  rhoL: the liquid density at T^n (default the constant
    one); expand: the term (alpha/rho_L) D(rho_L)/Dt of the previous step's continuity
    source, which the divergence of the advecting velocity u^n carries (reading R31), so
    that the two cancel in the liquid."""
    rhoL = cfg["rho_l"] if rhoL is None else rhoL
    cap = rhoL * alpha / dt
    capped = mdot > cap
    mdot = np.where(capped, cap, mdot)
    alpha_star = alpha - dt * mdot / rhoL
    if expand is not None:
        alpha_star = alpha_star - dt * expand
    return alpha_star, mdot, int(capped.sum())


def face_flux(G, u, dt):
    """phi_f = u_f A_f dt per face (volume crossing the face in one step)."""
    return [u[a] * G.A[a] * dt if a in G.act else None for a in range(3)]


def divergence_sum(G, F):
    """Net outflow sum over the faces of each cell of a face quantity F[a]."""
    out = np.zeros(G.n)
    for a in G.act:
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, G.n[a])
        hi[a] = slice(1, G.n[a] + 1)
        out += F[a][tuple(hi)] - F[a][tuple(lo)]
    return out


def _interior_mask(G, a):
    m = np.zeros(fshape(G, a), dtype=bool)
    sl = [slice(None)] * 3
    sl[a] = slice(1, G.n[a])
    m[tuple(sl)] = True
    return m


def alpha_advection(cfg, G, alpha_star, u, dt):
    """S3: Eq. (advection) by flux-corrected transport (Zalesak limiter).

    Low order: upwind.  High order: van Leer limited upwind value plus the
    compressive flux C_alpha |phi| (n_f . e) a_c (1 - a_c), n_f the normalised sum
    of the two cell gradients (pointing into the liquid), a_c the central face
    value.  Antidiffusive fluxes only on interior faces.  Bounds: the min / max
    of alpha* and alpha^L over the cell and its face neighbours, clipped to
    [0, 1].  A residual excursion out of [0, 1] is clipped and its volume
    accounted (reading R14).
    Returns (alpha_new, clip_volume, n_clipped).
    """
    n = G.n
    solid = solid_mask(cfg, G)
    phi = face_flux(G, u, dt)
    Pa = pad_scalar(G, alpha_star, "alpha")
    g = grad_central(G, Pa, solid=solid)
    Pg = [_pad(G, g[a]) if a in G.act else None for a in range(3)]
    FL = [None] * 3
    AF = [None] * 3
    for a in G.act:
        fs = fshape(G, a)
        L = _view(G, Pa, fs, {a: -1})
        R = _view(G, Pa, fs, {a: 0})
        LL = _view(G, Pa, fs, {a: -2})
        RR = _view(G, Pa, fs, {a: 1})
        pos = phi[a] >= 0.0
        up = np.where(pos, L, R)
        FL[a] = phi[a] * up
        aVL = np.where(pos, van_leer(LL, L, R), van_leer(RR, R, L))
        # face normal from the two adjacent cell gradients
        gf = [(_view(G, Pg[b], fs, {a: -1}) + _view(G, Pg[b], fs, {a: 0})) if b in G.act else None for b in range(3)]
        gfm = np.sqrt(sum(gf[b] * gf[b] for b in G.act))
        with np.errstate(divide="ignore", invalid="ignore"):
            ne = np.where(gfm > 1e-8 / G.hmin, gf[a] / gfm, 0.0)
        ac = 0.5 * (L + R)
        FH = phi[a] * aVL + cfg["C_alpha"] * np.abs(phi[a]) * ne * ac * (1.0 - ac)
        AF[a] = np.where(_interior_mask(G, a), FH - FL[a], 0.0)
    alphaL = alpha_star - divergence_sum(G, FL) / G.V
    # local bounds over the cell and its face neighbours (inside the domain)
    hi_v = np.maximum(alpha_star, alphaL)
    lo_v = np.minimum(alpha_star, alphaL)
    amax = hi_v.copy()
    amin = lo_v.copy()
    Ps = _pad(G, solid) if solid is not None else None
    for a in G.act:
        for sh in (-1, 1):
            # neighbours outside the domain do not take part: pad with the cell's own value
            Ph = pad_scalar(G, hi_v, "zg")
            Pl = pad_scalar(G, lo_v, "zg")
            nh = _view(G, Ph, n, {a: sh})
            nl = _view(G, Pl, n, {a: sh})
            if Ps is not None:       # nor do the fibre's cells
                ns = _view(G, Ps, n, {a: sh})
                nh = np.where(ns, hi_v, nh)
                nl = np.where(ns, lo_v, nl)
            amax = np.maximum(amax, nh)
            amin = np.minimum(amin, nl)
    amax = np.minimum(amax, 1.0)
    amin = np.maximum(amin, 0.0)
    Pp = np.zeros(n)
    Pm = np.zeros(n)
    for a in G.act:
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, n[a])
        hi[a] = slice(1, n[a] + 1)
        A_lo = AF[a][tuple(lo)]     # flux through the low face, into the cell when > 0
        A_hi = AF[a][tuple(hi)]     # flux through the high face, out of the cell when > 0
        Pp += np.maximum(0.0, A_lo) + np.maximum(0.0, -A_hi)
        Pm += np.maximum(0.0, -A_lo) + np.maximum(0.0, A_hi)
    Qp = (amax - alphaL) * G.V
    Qm = (alphaL - amin) * G.V
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        Rp = np.where(Pp > 0.0, np.minimum(1.0, np.maximum(0.0, Qp / Pp)), 0.0)
        Rm = np.where(Pm > 0.0, np.minimum(1.0, np.maximum(0.0, Qm / Pm)), 0.0)
    CA = [None] * 3
    for a in G.act:
        fs = fshape(G, a)
        PRp = pad_scalar(G, Rp, "zg")
        PRm = pad_scalar(G, Rm, "zg")
        RpL = _view(G, PRp, fs, {a: -1})
        RpR = _view(G, PRp, fs, {a: 0})
        RmL = _view(G, PRm, fs, {a: -1})
        RmR = _view(G, PRm, fs, {a: 0})
        C = np.where(AF[a] >= 0.0, np.minimum(RpR, RmL), np.minimum(RpL, RmR))
        CA[a] = C * AF[a]
    anew = alphaL - divergence_sum(G, CA) / G.V
    clipped = np.clip(anew, 0.0, 1.0)
    clip_vol = float(np.sum((anew - clipped) * G.V))
    nclip = int(np.count_nonzero(anew != clipped))
    return clipped, clip_vol, nclip, alphaL


def youngs_normal(G, a):
    """Interface normal of every cell in box-scaled coordinates (component a times h_a),
    pointing out of the liquid: minus the gradient of alpha by Youngs' weighting, each
    difference alpha(+1) - alpha(-1) along an axis summed over the neighbouring rows with
    weights (1, 2, 1) per other axis (the mean of the gradients at the cell's corners;
    the cell size cancels in box coordinates).  Ghosts: mirror at the axis, 0 outside."""
    P = pad_scalar(G, a, "alpha")
    w = (1.0, 2.0, 1.0)
    out = []
    for ax in range(3):
        if ax not in G.act:
            out.append(None)
            continue
        others = [b for b in G.act if b != ax]
        acc = np.zeros(G.n)
        if len(others) == 1:
            for ib, sb in enumerate((-1, 0, 1)):
                acc += w[ib] * (_view(G, P, G.n, {ax: 1, others[0]: sb}) - _view(G, P, G.n, {ax: -1, others[0]: sb}))
        else:
            for ib, sb in enumerate((-1, 0, 1)):
                for ic, sc in enumerate((-1, 0, 1)):
                    sh_p = {ax: 1, others[0]: sb, others[1]: sc}
                    sh_m = {ax: -1, others[0]: sb, others[1]: sc}
                    acc += w[ib] * w[ic] * (_view(G, P, G.n, sh_p) - _view(G, P, G.n, sh_m))
        out.append(-acc)
    return out


def alpha_advection_geometric(cfg, G, alpha_star, u, dt):
    """S3 by geometric advection (Sec. 2.1, Eq. advection: the paper's isoAdvector
    transports a planar interface through the faces geometrically), on the uniform grid
    (reading R30): one sweep per axis in the order 0, 1 (, 2).  In each sweep every
    cell with 0 < alpha < 1 holds a plane (PLIC: Youngs' normal, the constant that cuts
    its alpha), and the liquid a face passes is the flux phi_f = u_f A_f dt times the
    fraction of the donor cell's swept slab (width |u_f| dt / h) on the liquid side of
    the donor's plane (full and empty donors pass phi_f and 0, a donor whose Youngs
    normal vanishes -- no direction to the interface -- its own fraction; nothing enters
    from outside the domain).  The update of sweep k is
        alpha <- alpha - (F_hi - F_lo)/V + a_c (dphi_k - dphi / D)/V,
    a_c = 1 where alpha* > 1/2 (Weymouth & Yue's term, which keeps a solenoidal flow's
    sweeps bounded), with the cell's mean divergence dphi / D taken out of each sweep so
    that the terms cancel over the sweeps and the scheme conserves the liquid volume
    exactly whatever the divergence (the Stefan flow has div u = S).  A residual
    excursion out of [0, 1] is clipped and its volume accounted (reading R14).
    Returns (alpha_new, clip_volume, n_clipped, alpha_before_clipping)."""
    n = G.n
    phi = face_flux(G, u, dt)
    ac = (alpha_star > 0.5).astype(np.float64)
    dphi = {}
    for k in G.act:
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[k] = slice(0, n[k])
        hi[k] = slice(1, n[k] + 1)
        dphi[k] = phi[k][tuple(hi)] - phi[k][tuple(lo)]
    div = sum(dphi[k] for k in G.act)
    D = float(len(G.act))
    a = alpha_star.copy()
    for k in G.act:
        ac_k = np.clip(a, 0.0, 1.0)
        N = youngs_normal(G, ac_k)
        mixed = (ac_k > 0.0) & (ac_k < 1.0)
        Nm = np.stack([N[b][mixed] for b in G.act], axis=1)
        beta = np.zeros(n)
        beta[mixed] = plic.plane_constant(Nm, ac_k[mixed])
        # fraction of the swept slab: donor L through its high face (phi >= 0), donor R
        # through its low face (phi < 0); ghosts outside the domain are empty
        fs = fshape(G, k)
        Pa = _pad(G, ac_k)
        aL = _view(G, Pa, fs, {k: -1})
        aR = _view(G, Pa, fs, {k: 0})
        pos = phi[k] >= 0.0
        donor_a = np.where(pos, aL, aR)
        frac = np.where(donor_a >= 1.0, 1.0, 0.0)
        width = np.minimum(np.abs(u[k]) * dt / G.h[k], 1.0)
        kk = G.act.index(k)
        for side_pos in (True, False):
            sel_f = (pos == side_pos) & (donor_a > 0.0) & (donor_a < 1.0)
            if not sel_f.any():
                continue
            # donor cell index of each selected face
            idx_f = np.argwhere(sel_f)
            if side_pos:
                idx_f[:, k] -= 1
            cells = tuple(idx_f[:, b] for b in range(3))
            Nd = np.stack([N[b][cells] for b in G.act], axis=1)
            bd = beta[cells]
            c = width[sel_f]
            Ns = Nd.copy()
            Ns[:, kk] = c * Nd[:, kk]
            bs = bd - Nd[:, kk] * (1.0 - c) if side_pos else bd
            flat = np.all(Nd == 0.0, axis=1)
            frac[sel_f] = np.where(flat, ac_k[cells], plic.cut_fraction(Ns, bs))
        F = phi[k] * frac
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[k] = slice(0, n[k])
        hi[k] = slice(1, n[k] + 1)
        a = a - (F[tuple(hi)] - F[tuple(lo)]) / G.V + ac * (dphi[k] - div / D) / G.V
    clipped = np.clip(a, 0.0, 1.0)
    clip_vol = float(np.sum((a - clipped) * G.V))
    nclip = int(np.count_nonzero(a != clipped))
    return clipped, clip_vol, nclip, a


def scalar_transport(cfg, G, phi_n, coef_t, gamma, src, u, dt, amb, pin_mask=None, pin_val=None, solid=None,
                     src_int=None):
    """S5 / S6: backward-Euler diffusion, explicit limited-linear-upwind convection.

    coef_t V (phi - phi^n)/dt + coef_t [sum_f F_f phi_f - phi_P sum_f F_f]
        = sum_f gamma_f A_f (phi_N - phi_P)/h + src V
    F_f = u_f A_f outward; phi_f = minmod limited linear upwind (reading R15);
    gamma_f the harmonic face mean 2 gL gR/(gL + gR) (series resistance across
    the face; with the paper's mixture rule for k and rho D an arithmetic mean
    lets the liquid-side values leak one cell into the gas).  Dirichlet faces (forced inlet, inflowing open
    faces) use gamma_P A_b/(h/2) towards amb.  Rows in pin_mask are fixed at
    pin_val and eliminated symmetrically.  With a fibre (solid mask, reading R32) the
    solid cells carry gamma = 0, so the harmonic mean closes every face of the sphere
    (two zeros give 0), the faces of the sphere carry no velocity, and a far upwind
    value inside the fibre is replaced by the near one (zero gradient).  src_int, when
    given, is a source already integrated over each cell, added to the right-hand side.
    """
    n = G.n
    P = pad_scalar(G, phi_n, "TO", u=u, amb=amb)
    flux = [None] * 3
    coup = {}
    diag = coef_t * G.V / dt
    rhs = coef_t * G.V * phi_n / dt + src * G.V
    if src_int is not None:
        rhs = rhs + src_int
    Pg = pad_scalar(G, gamma, "zg")
    for a in G.act:
        fs = fshape(G, a)
        L = _view(G, P, fs, {a: -1})
        R = _view(G, P, fs, {a: 0})
        LL = _view(G, P, fs, {a: -2})
        RR = _view(G, P, fs, {a: 1})
        if solid is not None:
            Ps = _pad(G, solid)
            LL = np.where(_view(G, Ps, fs, {a: -2}), L, LL)
            RR = np.where(_view(G, Ps, fs, {a: 1}), R, RR)
        F = u[a] * G.A[a]
        pos = F >= 0.0
        val = np.where(pos, lim_upwind(LL, L, R), lim_upwind(RR, R, L))
        # boundary faces: upwind value (ghost = amb-side value on inflow)
        for side in (0, 1):
            fidx = 0 if side == 0 else n[a]
            kind = G.bc[a][side]
            vf = _face_slab(val, a, fidx)
            Fb = _face_slab(F, a, fidx)
            inner = _face_slab(R if side == 0 else L, a, fidx)
            inflow = (Fb > 0.0) if side == 0 else (Fb < 0.0)
            if kind in (OPEN, FORCED):
                vf[...] = np.where(inflow, amb, inner)
            else:
                vf[...] = inner
        flux[a] = F * val
        gL = _view(G, Pg, fs, {a: -1})
        gR = _view(G, Pg, fs, {a: 0})
        with np.errstate(divide="ignore", invalid="ignore"):
            cf = np.where(gL + gR > 0.0, 2.0 * gL * gR / (gL + gR), 0.0) * G.A[a] / G.h[a]
        sl = [slice(None)] * 3
        sl[a] = slice(1, n[a])
        coup[a] = cf[tuple(sl)]
        # Dirichlet boundary faces
        for side in (0, 1):
            kind = G.bc[a][side]
            fidx = 0 if side == 0 else n[a]
            cidx = 0 if side == 0 else n[a] - 1
            Ab = _face_slab(G.A[a], a, fidx)
            gP = _face_slab(gamma, a, cidx)
            if kind == FORCED:
                isdir = np.ones_like(Ab, dtype=bool)
            elif kind == OPEN:
                isdir = _outward_vel(G, u, a, side) < 0.0
            else:
                continue
            cb = np.where(isdir, gP * Ab / (0.5 * G.h[a]), 0.0)
            _face_slab(diag, a, cidx)[...] += cb
            _face_slab(rhs, a, cidx)[...] += cb * amb
    net = divergence_sum(G, flux)
    Fsum = divergence_sum(G, [u[a] * G.A[a] if a in G.act else None for a in range(3)])
    rhs = rhs - coef_t * (net - phi_n * Fsum)
    if pin_mask is not None and pin_mask.any():
        for a in G.act:
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[a] = slice(0, n[a] - 1)
            hi[a] = slice(1, n[a])
            lo, hi = tuple(lo), tuple(hi)
            c = coup[a]
            pl, ph = pin_mask[lo], pin_mask[hi]
            # unpinned neighbour of a pinned cell: known value to the rhs, coupling kept on its diagonal
            m_lo = ~pl & ph
            m_hi = pl & ~ph
            rhs[lo] += np.where(m_lo, c * pin_val[hi], 0.0)
            diag[lo] += np.where(m_lo, c, 0.0)
            rhs[hi] += np.where(m_hi, c * pin_val[lo], 0.0)
            diag[hi] += np.where(m_hi, c, 0.0)
            coup[a] = np.where(pl | ph, 0.0, c)
        # pinned rows keep the scale of the other rows (coef V/dt), so that a
        # relative residual measures the free rows too
        dpin = coef_t * G.V / dt
        diag = np.where(pin_mask, dpin, diag)
        rhs = np.where(pin_mask, dpin * pin_val, rhs)
    return solve_box(n, diag, coup, rhs)


def enthalpy_diffusion(cfg, G, omega, T, gamma):
    """The species-diffusion enthalpy term of Eq. (Teqn), -sum_i j_d,i C_p,i . grad T, for
    the binary gas (vapour v, inert g): with Fick's fluxes j_v = -rho D grad(omega) and
    j_g = -j_v it is (C_p,v - C_p,g) rho D grad(omega) . grad(T).  Reading R33: integrated
    over each cell as half the sum, over the cell's interior faces f, of
    gamma_f (A_f / h_f) (omega_N - omega_P)(T_N - T_P), gamma_f the harmonic face mean of
    rho D of the species equation (S6); boundary faces carry none.  Each face's product is
    shared equally by its two cells.  Evaluated at omega^n and T^n (explicit)."""
    dcp = cfg["cp_v"] - cfg["cp_g"]
    Q = np.zeros(G.n)
    if dcp == 0.0:
        return Q
    for a in G.act:
        if G.n[a] < 2:
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, G.n[a] - 1)
        hi[a] = slice(1, G.n[a])
        lo, hi = tuple(lo), tuple(hi)
        gL, gR = gamma[lo], gamma[hi]
        with np.errstate(divide="ignore", invalid="ignore"):
            gf = np.where(gL + gR > 0.0, 2.0 * gL * gR / (gL + gR), 0.0)
        sl = [slice(None)] * 3
        sl[a] = slice(1, G.n[a])
        Af = G.A[a][tuple(sl)]                  # the interior faces' areas
        prod = gf * Af / G.h[a] * (omega[hi] - omega[lo]) * (T[hi] - T[lo])
        Q[lo] += 0.5 * prod
        Q[hi] += 0.5 * prod
    return dcp * Q


def momentum_predictor(cfg, G, st, pr, alpha, dt, parts=None):
    """S7: Eq. (NavierStokesModified) on the staggered (MAC) faces, p_rgh form.

    For face f of direction c (cells L, R), multiplied by the face control
    volume V_f:
      rho_f V_f (u* - u^n)/dt = -rho_f V_f sum_a ubar_a (u^{+a} - u^{-a})/h_a   (advective form)
          + sum_a [A'_a mu d_a u*_c]^{+a}_{-a}   (implicit)  - 2 mu_f V_f u*_r / r_f^2 (axisym, c = r)
          + sum_a [A'_a mu d_c u_a^n]^{+a}_{-a}  (explicit transpose part)
          - A_f (p_R - p_L) - A_f (g . x_f)(rho_R - rho_L) + A_f (rho alpha)_f (xi_R - xi_L)
    A'_a is the area of the control-volume face normal to a, mu at cell
    centres (a = c) or at edges (mean of the four cells around the edge).
    Boundary faces: wall / axis 0, forced inlet u_in, open boundary zero
    gradient (copied from the adjacent interior face after the solve).
    """
    n = G.n
    u = st["u"]
    solid = solid_mask(cfg, G)
    rho, mu = pr["rho"], pr["mu"]
    xi = xi_field(cfg, G)
    Prho = pad_scalar(G, rho, "zg")
    Pmu = pad_scalar(G, mu, "zg")
    Pp = pad_scalar(G, st["p"], "zg")
    Pxi = pad_scalar(G, xi, "zg")
    Pra = pad_scalar(G, rho * alpha, "zg")
    Pu = [pad_velocity(G, u[a], a, cfg["u_inflow"]) if a in G.act else None for a in range(3)]
    ustar = [None if x is None else x.copy() for x in u]
    g = cfg["g"]
    for c in G.act:
        fs = fshape(G, c)
        rhoL = _view(G, Prho, fs, {c: -1})
        rhoR = _view(G, Prho, fs, {c: 0})
        muL = _view(G, Pmu, fs, {c: -1})
        muR = _view(G, Pmu, fs, {c: 0})
        rho_f = 0.5 * (rhoL + rhoR)
        mu_f = 0.5 * (muL + muR)
        # coordinates of the face centres
        X = [Grid.along(G.xf[a], a) if a == c else Grid.along(G.xc[a], a) for a in range(3)]
        if G.axisym:
            r_f = np.broadcast_to(X[0], fs)
            V_f = r_f * G.h[0] * G.h[1]
        else:
            r_f = None
            V_f = np.full(fs, G.h[0] * G.h[1] * G.h[2])
        A_f = V_f / G.h[c]
        diag = rho_f * V_f / dt
        rhs = rho_f * V_f * u[c] / dt
        coup = {}
        U = Pu[c]
        t_adv = np.zeros(fs)
        t_vT = np.zeros(fs)
        d_visc = np.zeros(fs)
        for a in G.act:
            # ---- advection (explicit, advective form)
            if a == c:
                ubar = u[c]
            else:
                ubar = np.zeros(fs)
                for (cell_sh, face_sh) in ((-1, 0), (-1, 1), (0, 0), (0, 1)):
                    ubar = ubar + _view(G, _pad(G, u[a]), fs, {c: cell_sh, a: face_sh})
                ubar = 0.25 * ubar
            um2 = _view(G, U, fs, {a: -2})
            um1 = _view(G, U, fs, {a: -1})
            u0 = _view(G, U, fs, {a: 0})
            up1 = _view(G, U, fs, {a: 1})
            up2 = _view(G, U, fs, {a: 2})
            pos = ubar >= 0.0
            uplus = np.where(pos, lim_upwind(um1, u0, up1), lim_upwind(up2, up1, u0))
            uminus = np.where(pos, lim_upwind(um2, um1, u0), lim_upwind(up1, u0, um1))
            t_adv = t_adv - rho_f * V_f * ubar * (uplus - uminus) / G.h[a]
            # ---- viscous terms
            if a == c:
                # control-volume faces at the cell centres L (minus) and R (plus)
                if G.axisym and c == 0:
                    rL = np.broadcast_to(Grid.along(np.concatenate(([0.0], G.xc[0])), 0), fs)
                    rR = np.broadcast_to(Grid.along(np.concatenate((G.xc[0], [0.0])), 0), fs)
                    ApL = G.area_normal(0, rL)
                    ApR = G.area_normal(0, rR)
                elif G.axisym:
                    ApL = ApR = G.area_normal(1, r_f)
                else:
                    ApL = ApR = np.full(fs, G.area_normal(c, None))
                kR = muR * ApR / G.h[c]           # coupling f <-> f + e_c
                kL = muL * ApL / G.h[c]           # coupling f - e_c <-> f
                # explicit transpose part (a = c): d_c u_c at the cell centres
                dR = (_view(G, U, fs, {c: 1}) - u0) / G.h[c]
                dL = (u0 - _view(G, U, fs, {c: -1})) / G.h[c]
                t_vT = t_vT + muR * ApR * dR - muL * ApL * dL
                # implicit couplings between interior faces; known boundary faces to the rhs
                cc = kR.copy()
                sl = [slice(None)] * 3
                sl[c] = slice(1, n[c] - 1)
                coup[c] = cc[tuple(sl)]
                for side in (0, 1):
                    kind = G.bc[c][side]
                    if kind == OPEN:
                        continue
                    if side == 0:
                        f1 = 1
                        kb = _face_slab(kL, c, f1)
                        ub = _face_slab(u[c], c, 0)
                    else:
                        f1 = n[c] - 1
                        kb = _face_slab(kR, c, f1)
                        ub = _face_slab(u[c], c, n[c])
                    _face_slab(d_visc, c, f1)[...] += kb
                    _face_slab(rhs, c, f1)[...] += kb * ub
            else:
                # edges at f +- e_a/2; mu = mean of the 4 cells around the edge
                def mu_edge(sh):
                    # viscosity on the edge between this face and its neighbour at
                    # offset sh along a: the mean of the four cells around the edge
                    s = _view(G, Pmu, fs, {c: -1}) + _view(G, Pmu, fs, {c: 0}) \
                        + _view(G, Pmu, fs, {c: -1, a: sh}) + _view(G, Pmu, fs, {c: 0, a: sh})
                    return 0.25 * s
                if G.axisym and a == 0:
                    r_ep = np.broadcast_to(Grid.along(G.xf[0][1:], 0), fs)
                    r_em = np.broadcast_to(Grid.along(G.xf[0][:-1], 0), fs)
                    App = G.area_normal(0, r_ep)
                    Apm = G.area_normal(0, r_em)
                elif G.axisym:
                    App = Apm = G.area_normal(1, r_f)
                else:
                    App = Apm = np.full(fs, G.area_normal(a, None))
                mup = mu_edge(1)
                mum = mu_edge(-1)
                kp = mup * App / G.h[a]
                # explicit transpose: d_c u_a at the edges from the a-faces of cells L and R
                Pua = _pad(G, u[a])
                uaR_hi = _view(G, Pua, fs, {c: 0, a: 1})
                uaL_hi = _view(G, Pua, fs, {c: -1, a: 1})
                uaR_lo = _view(G, Pua, fs, {c: 0, a: 0})
                uaL_lo = _view(G, Pua, fs, {c: -1, a: 0})
                t_vT = t_vT + mup * App * (uaR_hi - uaL_hi) / G.h[c] - mum * Apm * (uaR_lo - uaL_lo) / G.h[c]
                sl = [slice(None)] * 3
                sl[a] = slice(0, n[a] - 1)
                coup[a] = kp[tuple(sl)]
                # ghost neighbours beyond the tangential boundary
                for side in (0, 1):
                    kind = G.bc[a][side]
                    if kind in (WALL, FORCED):
                        if side == 0:
                            kb = _face_slab(mum * Apm / G.h[a], a, 0)
                            _face_slab(d_visc, a, 0)[...] += 2.0 * kb
                        else:
                            kb = _face_slab(kp, a, n[a] - 1)
                            _face_slab(d_visc, a, n[a] - 1)[...] += 2.0 * kb
        if G.axisym and c == 0:
            with np.errstate(divide="ignore", invalid="ignore"):
                hoop = np.where(r_f > 0.0, 2.0 * mu_f * V_f / (r_f * r_f), 0.0)
            d_visc = d_visc + hoop
        # pressure, buoyancy (p_rgh form) and centripetal force, balanced face form
        gx = np.zeros(fs)
        for a in G.act:
            gx = gx + g[a] * np.broadcast_to(X[a], fs)
        pL = _view(G, Pp, fs, {c: -1})
        pR = _view(G, Pp, fs, {c: 0})
        xiL = _view(G, Pxi, fs, {c: -1})
        xiR = _view(G, Pxi, fs, {c: 0})
        raL = _view(G, Pra, fs, {c: -1})
        raR = _view(G, Pra, fs, {c: 0})
        t_force = -A_f * (pR - pL) - A_f * gx * (rhoR - rhoL) + A_f * 0.5 * (raL + raR) * (xiR - xiL)
        diag = diag + d_visc
        rhs = rhs + t_adv + t_vT + t_force
        # solve on the interior faces
        sl = [slice(None)] * 3
        sl[c] = slice(1, n[c])
        sl = tuple(sl)
        ms = list(fs)
        ms[c] = n[c] - 1
        cpl = {}
        for a in G.act:
            cc = coup[a]
            if a != c:
                cc = cc[sl]
            cpl[a] = cc
        if parts is not None:
            parts[c] = dict(sl=sl, shape=tuple(ms), d_visc=d_visc[sl], coup=cpl, adv=t_adv[sl],
                            visc_T=t_vT[sl], force=t_force[sl], V_f=V_f[sl])
        dsol, rsol = diag[sl], rhs[sl]
        if solid is not None:
            # faces of the sphere (a fibre cell on either side, reading R32): no slip and no
            # penetration, u* = 0; a neighbour's coupling to one of them goes into that
            # neighbour's diagonal (the known value 0)
            Ps = _pad(G, solid)
            B = (_view(G, Ps, fs, {c: -1}) | _view(G, Ps, fs, {c: 0}))[sl]
            dsol, rsol = dsol.copy(), np.where(B, 0.0, rsol)
            for a in G.act:
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[a] = slice(0, ms[a] - 1)
                hi[a] = slice(1, ms[a])
                lo, hi = tuple(lo), tuple(hi)
                cc = cpl[a]
                dsol[lo] += np.where(~B[lo] & B[hi], cc, 0.0)
                dsol[hi] += np.where(B[lo] & ~B[hi], cc, 0.0)
                cpl[a] = np.where(B[lo] | B[hi], 0.0, cc)
        x = solve_box(tuple(ms), dsol, cpl, rsol)
        us = ustar[c]
        us[sl] = x
        for side in (0, 1):
            kind = G.bc[c][side]
            if kind == OPEN:
                if side == 0:
                    _face_slab(us, c, 0)[...] = _face_slab(us, c, 1)
                else:
                    _face_slab(us, c, n[c])[...] = _face_slab(us, c, n[c] - 1)
    return ustar


def projection(cfg, G, st, ustar, pr, mdot, alpha, rhoG_old, rhoG_new, dt, rhoL_old=None, rhoL_new=None):
    """S8-S10: Eq. (pequation),
        div u = S = mdot (1/rho_G - 1/rho_L) - (1 - alpha)/rho_G (D rho_G/Dt)
                    - alpha/rho_L (D rho_L/Dt),
    D rho/Dt = (rho^{n+1} - rho^n)/dt + vbar^n . grad rho^{n+1} for both densities (the
    liquid one rho_L(T), reading R31; its term vanishes for a constant density).
    Pressure increment:  sum_f beta_f (dp_P - dp_N) + sum_open beta_b dp_P
                        = (S_P V_P - sum_f u*_f A_f)/dt,
    beta_f = A_f/(rho_f h), beta_b = A_b/(rho_P h/2) on open (p_rgh = p_ext) faces.
    Then u = u* - dt (grad dp)_f / rho_f, p_rgh += dp (one corrector, reading R19).
    Returns (u_new, p_new, dp, S).
    """
    n = G.n
    rho = pr["rho"]
    solid = solid_mask(cfg, G)
    vc = cell_velocity(G, st["u"])
    gr = grad_central(G, pad_scalar(G, rhoG_new, "zg"), solid=solid)
    adv = sum(vc[a] * gr[a] for a in G.act)
    rL1 = cfg["rho_l"] if rhoL_new is None else rhoL_new
    S = mdot * (1.0 / rhoG_new - 1.0 / rL1) - (1.0 - alpha) / rhoG_new * ((rhoG_new - rhoG_old) / dt + adv)
    expand = np.zeros(n)
    if rhoL_new is not None and cfg.get("drho_l_dT", 0.0) != 0.0:
        grl = grad_central(G, pad_scalar(G, rhoL_new, "zg"))
        advl = sum(vc[a] * grl[a] for a in G.act)
        expand = alpha / rhoL_new * ((rhoL_new - rhoL_old) / dt + advl)
        S = S - expand
    if solid is not None:
        S = np.where(solid, 0.0, S)      # the fibre holds no fluid: no continuity source
    diag, coup, beta = pressure_system(G, rho, solid, cfg["rho_l"])
    div_star = divergence_sum(G, [ustar[a] * G.A[a] if a in G.act else None for a in range(3)])
    rhs = (S * G.V - div_star) / dt
    dp = solve_box(n, diag, coup, rhs)
    Pdp = _pad(G, dp)       # ghost 0 = the Dirichlet value on open faces
    unew = [None] * 3
    for a in G.act:
        # beta_f (dR - dL)/A_f = (grad dp)_f/rho_f, with the half-cell distance on open faces
        dL = _view(G, Pdp, fshape(G, a), {a: -1})
        dR = _view(G, Pdp, fshape(G, a), {a: 0})
        with np.errstate(divide="ignore", invalid="ignore"):
            corr = np.where(G.A[a] > 0.0, dt * beta[a] * (dR - dL) / G.A[a], 0.0)
        unew[a] = ustar[a] - corr
    return unew, st["p"] + dp, dp, S, (diag, coup, rhs), expand


def pressure_system(G, rho, solid=None, rho_l=None):
    """Variable-density pressure operator of Eq. (pequation):
    (L x)_P = sum_f beta_f (x_P - x_N) + sum_open beta_b x_P,
    beta_f = A_f/(rho_f h) with rho_f the arithmetic face mean, beta_b =
    A_b/(rho_P h/2) on open (p_rgh = p_ext) faces, zero on walls, the axis and
    a forced inlet.  With a fibre (reading R32) beta vanishes on the faces of the
    sphere (zero normal gradient) and each solid cell's row is decoupled with the
    diagonal 2 d V_P / (h_min^2 rho_L) (d the active axes; the value does not change the
    solution), so that its increment is 0.  Returns (diag, couplings, beta per face)."""
    n = G.n
    Prho = pad_scalar(G, rho, "zg")
    diag = np.zeros(n)
    coup = {}
    beta = [None] * 3
    Ps = _pad(G, solid) if solid is not None else None
    for a in G.act:
        fs = fshape(G, a)
        rho_f = 0.5 * (_view(G, Prho, fs, {a: -1}) + _view(G, Prho, fs, {a: 0}))
        b = G.A[a] / (rho_f * G.h[a])
        if Ps is not None:
            b = np.where(_view(G, Ps, fs, {a: -1}) | _view(G, Ps, fs, {a: 0}), 0.0, b)
        for side in (0, 1):
            fidx = 0 if side == 0 else n[a]
            cidx = 0 if side == 0 else n[a] - 1
            if G.bc[a][side] == OPEN:
                bb = _face_slab(G.A[a], a, fidx) / (_face_slab(rho, a, cidx) * 0.5 * G.h[a])
                _face_slab(b, a, fidx)[...] = bb
                _face_slab(diag, a, cidx)[...] += bb
            else:
                _face_slab(b, a, fidx)[...] = 0.0
        beta[a] = b
        sl = [slice(None)] * 3
        sl[a] = slice(1, n[a])
        coup[a] = b[tuple(sl)]
    if solid is not None:
        diag = np.where(solid, 2.0 * len(G.act) * G.V / (G.hmin * G.hmin * rho_l), diag)
    return diag, coup, beta


def boundary_vapour_outflow(cfg, G, u, omega, rhoG):
    """Vapour mass leaving through the open boundaries per unit time (per radian
    in 2D): sum rho_G omega_b u_out A_b, omega_b upwind (0 on inflow)."""
    tot = 0.0
    for a in G.act:
        for side in (0, 1):
            if G.bc[a][side] not in (OPEN, FORCED):
                continue
            fidx = 0 if side == 0 else G.n[a]
            cidx = 0 if side == 0 else G.n[a] - 1
            vout = _outward_vel(G, u, a, side)
            Ab = _face_slab(G.A[a], a, fidx)
            wP = _face_slab(omega, a, cidx)
            rP = _face_slab(rhoG, a, cidx)
            tot += float(np.sum(np.where(vout > 0.0, rP * wP * vout * Ab, 0.0)))
    return tot


def courant_dt(cfg, G, u, dt_prev=None):
    """Time step from the threshold Courant number (Sec. 3.1: the step is computed
    automatically from a Courant threshold; the paper gives neither the threshold nor
    the growth rule, reading R29).  With co_max > 0:
        dt = min(dt_max, co_max h_min / max|u|, 1.2 dt_prev)
    over every face velocity u, dt_max the configured dt (no velocity limit while u = 0,
    no growth limit for the first step); with co_max = 0 the configured dt."""
    co = cfg.get("co_max", 0.0)
    if not co > 0.0:
        return cfg["dt"]
    umax = max(float(np.max(np.abs(u[a]))) for a in G.act)
    d = cfg["dt"]
    if umax > 0.0:
        d = min(d, (co * G.hmin) / umax)
    if dt_prev is not None:
        d = min(d, 1.2 * dt_prev)
    return d


def step(cfg, st, keep=False):
    """Advance the state by one time step dt (the state's, from the Courant rule, or
    the configured one).  Returns the new state; with keep=True the intermediate fields
    of every stage are attached under 'aux'."""
    G = Grid(cfg)
    dt = st.get("dt", cfg["dt"])
    mask = cfg["physics_mask"]
    const = bool(cfg["const_props_check"])
    alpha, T, omega, u = st["alpha"], st["T"], st["omega"], st["u"]
    flags = 0
    # S0
    omega, rhoG_old = thermo_pin(cfg, G, alpha, T, omega)
    # S1, S2
    if mask & PHYS_EVAP:
        mdot, mraw, adj, K, f1 = evaporation_flux(cfg, G, alpha, omega, rhoG_old, u, T)
        flags |= f1
    else:
        mdot, mraw, adj, K = np.zeros(G.n), np.zeros(G.n), np.full(G.n, -1), 0.0
    rhoL_old = th.rho_liquid(cfg, T)
    alpha_star, mdot, ncap = alpha_source(cfg, alpha, mdot, dt, rhoL_old, st.get("expand"))
    if ncap:
        flags |= FLAG_MDOT_CAPPED
    # S3
    if (mask & PHYS_FLOW) and cfg.get("adv_scheme", 0) == 1:
        alpha_new, clip_vol, nclip, alphaL = alpha_advection_geometric(cfg, G, alpha_star, u, dt)
    elif mask & PHYS_FLOW:
        alpha_new, clip_vol, nclip, alphaL = alpha_advection(cfg, G, alpha_star, u, dt)
    else:
        alpha_new, clip_vol, nclip, alphaL = np.clip(alpha_star, 0.0, 1.0), 0.0, 0, alpha_star
        clip_vol = float(np.sum((alpha_star - alpha_new) * G.V))
        nclip = int(np.count_nonzero(alpha_star != alpha_new))
    if nclip:
        flags |= FLAG_ALPHA_CLIPPED
    # S4
    solid = solid_mask(cfg, G)
    pr = props(cfg, alpha_new, rhoG_old, omega, T, solid)
    # S5
    if (mask & PHYS_ENERGY) and not const:
        hd = None
        if cfg["cp_v"] != cfg["cp_g"]:
            hd = enthalpy_diffusion(cfg, G, omega, T, pr["rho"] * pr["D"])
        T_new = scalar_transport(cfg, G, T, pr["rho"] * pr["cp"], pr["k"], -mdot * cfg["Lv"], u, dt, cfg["T_amb"],
                                 solid=solid, src_int=hd)
    else:
        T_new = T.copy()
    # S6
    yeq_new = th.Y_eq(cfg, T_new)
    pin = alpha_new >= 0.5
    if mask & PHYS_SPECIES:
        omega_new = scalar_transport(cfg, G, omega, pr["rho"], pr["rho"] * pr["D"], np.zeros(G.n), u, dt, 0.0,
                                     pin_mask=pin, pin_val=yeq_new, solid=solid)
    else:
        omega_new = np.where(pin, yeq_new, omega)
    rhoG_new = th.rho_gas(cfg, T_new, omega_new)
    # S7 - S10
    if mask & PHYS_FLOW:
        ustar = momentum_predictor(cfg, G, st, pr, alpha_new, dt)
        u_new, p_new, dp, S, psys, expand = projection(cfg, G, st, ustar, pr, mdot, alpha_new, rhoG_old, rhoG_new,
                                                       dt, rhoL_old, th.rho_liquid(cfg, T_new))
    else:
        ustar, u_new, p_new, dp, S, psys = u, u, st["p"], np.zeros(G.n), np.zeros(G.n), None
        expand = np.zeros(G.n)      # no flow to carry an expansion
    out = dict(alpha=alpha_new, T=T_new, omega=omega_new, p=p_new, u=u_new, rhoG=rhoG_new,
               t=st["t"] + dt, step=st["step"] + 1,
               clip_mass=st["clip_mass"] + clip_vol,
               flags=flags, K=K, mdot=mdot, ncap=ncap, nclip=nclip)
    out["vap_out_cum"] = st["vap_out_cum"] + dt * boundary_vapour_outflow(cfg, G, u_new, omega_new, rhoG_new)
    out["dt"] = courant_dt(cfg, G, u_new, dt)
    out["expand"] = expand
    if keep:
        out["aux"] = dict(omega_pinned=omega, rhoG_old=rhoG_old, mraw=mraw, adj=adj, mdot=mdot,
                          alpha_star=alpha_star, alphaL=alphaL, ustar=ustar, dp=dp, S=S, psys=psys,
                          props=pr, yeq_new=yeq_new)
    return out


def diagnostics(cfg, st):
    """S11: droplet volume, equivalent diameter, evaporation rate, mean surface
    temperature, liquid and vapour masses, velocity and alpha extrema."""
    G = Grid(cfg)
    w = 2.0 * math.pi if G.axisym else 1.0
    alpha = st["alpha"]
    V_l = w * float(np.sum(alpha * G.V))
    d_eq = (6.0 * V_l / math.pi) ** (1.0 / 3.0)
    solid = solid_mask(cfg, G)
    g = grad_central(G, pad_scalar(G, alpha, "alpha"), solid=solid)
    gm = np.sqrt(sum(g[a] * g[a] for a in G.act))
    if solid is not None:
        gm = np.where(solid, 0.0, gm)     # the fibre's cells are not part of the surface
    sw = float(np.sum(gm * G.V))
    Ts = float(np.sum(st["T"] * gm * G.V)) / sw if sw > 0.0 else 0.0
    mdot = st.get("mdot", np.zeros(G.n))
    return dict(
        t=st["t"], step=st["step"], V_l=V_l, d_eq=d_eq, d2=d_eq * d_eq,
        mdot_tot=w * float(np.sum(mdot * G.V)), K_norm=st.get("K", 0.0), T_s_mean=Ts,
        M_liq=w * float(np.sum(th.rho_liquid(cfg, st["T"]) * alpha * G.V)),
        M_vap=w * float(np.sum((1.0 - alpha) * st["rhoG"] * st["omega"] * G.V)),
        vap_out_cum=w * st["vap_out_cum"],
        max_u=max(float(np.max(np.abs(st["u"][a]))) for a in G.act),
        alpha_min=float(alpha.min()), alpha_max=float(alpha.max()),
        clip_mass=w * st["clip_mass"], flags=st["flags"])


def run(cfg, nsteps, st=None):
    """nsteps time steps from the initial state of cfg (or from st)."""
    st = init_state(cfg) if st is None else st
    for _ in range(nsteps):
        st = step(cfg, st)
    return st
