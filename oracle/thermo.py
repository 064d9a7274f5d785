"""Oracle thermodynamics (plain FP64, scalar/numpy), Sec. 2.5 and Sec. 2.7.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Contents
  psat            Clausius-Clapeyron vapour pressure anchored at the normal
                  boiling point (the reading used in place of the paper's Yaws
                  correlations, which are not available).
  y_raoult        Eq. (equilibirumyi) with phi = phi_hat = 1 and no Poynting
                  factor: the ideal Raoult limit.
  pr_pure / pr_mix / pr_Z / pr_lnphi
                  Peng-Robinson (1976) a, b, mixing rule, largest real root of
                  the cubic in Z (Cardano), and mixture fugacity coefficients.
  y_pr            Eq. (equilibirumyi) with Peng-Robinson fugacities and the
                  Poynting factor exp(v_L (p - p0)/(R T)), v_L = M/rho_L
                  (Sec. 2.5, last equation), solved by fixed point in y.
  Y_eq            saturation mass fraction from the mole fraction.
  rho_gas         Eq. (densitygas): rho_G = p M_w / (Z R T).
"""
import math
import numpy as np

R_GAS = 8.314462618
P_ATM = 101325.0
SQRT2 = math.sqrt(2.0)

# status bits mirrored by the diagnostics (boiling clamp of the mole fraction)
Y_CLAMP = 1.0 - 1e-6


def psat(cfg, T):
    """Clausius-Clapeyron vapour pressure, p0(Tb) = 1 atm exactly."""
    return P_ATM * np.exp((cfg["Lv"] * cfg["M_l"] / R_GAS) * (1.0 / cfg["Tb"] - 1.0 / np.asarray(T, dtype=np.float64)))


def y_raoult(cfg, T):
    """Ideal equilibrium mole fraction y = p0(T)/p, clamped below 1 (boiling)."""
    y = psat(cfg, T) / cfg["P"]
    return np.minimum(y, Y_CLAMP)


def Y_from_y(cfg, y):
    """Mass fraction of the fuel vapour from its mole fraction (binary gas)."""
    ml, mg = cfg["M_l"], cfg["M_g"]
    return y * ml / (y * ml + (1.0 - y) * mg)


def y_from_Y(cfg, Y):
    """Mole fraction of the fuel vapour from its mass fraction (binary gas)."""
    ml, mg = cfg["M_l"], cfg["M_g"]
    return (Y / ml) / (Y / ml + (1.0 - Y) / mg)


# ---------------------------------------------------------------- Peng-Robinson

def pr_pure(T, Tc, Pc, om):
    """Pure-component PR parameters a(T), b (Peng & Robinson 1976)."""
    kappa = 0.37464 + 1.54226 * om - 0.26992 * om * om
    sq = 1.0 + kappa * (1.0 - math.sqrt(T / Tc))
    a = 0.45724 * R_GAS * R_GAS * Tc * Tc / Pc * sq * sq
    b = 0.07780 * R_GAS * Tc / Pc
    return a, b


def cubic_largest_root(c2, c1, c0):
    """Largest real root of z^3 + c2 z^2 + c1 z + c0 = 0 by Cardano's formula.

    Depressed cubic t^3 + p t + q = 0 with z = t - c2/3.  One real root
    (discriminant > 0): t = u - p/(3u), u = cbrt(-q/2 + sign(-q/2) sqrt(D)),
    which avoids cancellation.  Three real roots: trigonometric form, k = 0
    branch (the largest).
    """
    p = c1 - c2 * c2 / 3.0
    q = 2.0 * c2 * c2 * c2 / 27.0 - c2 * c1 / 3.0 + c0
    disc = 0.25 * q * q + p * p * p / 27.0
    if disc > 0.0:
        h = -0.5 * q
        u = math.copysign(abs(h + math.copysign(math.sqrt(disc), h)) ** (1.0 / 3.0),
                          h + math.copysign(math.sqrt(disc), h))
        t = u - p / (3.0 * u) if u != 0.0 else 0.0
    else:
        if p == 0.0:
            t = 0.0
        else:
            m = 2.0 * math.sqrt(-p / 3.0)
            arg = 3.0 * q / (p * m)
            arg = min(1.0, max(-1.0, arg))
            t = m * math.cos(math.acos(arg) / 3.0)
    return t - c2 / 3.0


def pr_mix(T, P, ys, crit, kij):
    """Mixture A, B and the pure a_i, b_i and a_ij for mole fractions ys.

    crit = [(Tc, Pc, omega), ...]; van der Waals one-fluid mixing rules
    a_m = sum_ij y_i y_j sqrt(a_i a_j)(1 - k_ij), b_m = sum_i y_i b_i.
    """
    ab = [pr_pure(T, *c) for c in crit]
    n = len(ys)
    aij = [[math.sqrt(ab[i][0] * ab[j][0]) * (1.0 - (kij if i != j else 0.0)) for j in range(n)] for i in range(n)]
    am = sum(ys[i] * ys[j] * aij[i][j] for i in range(n) for j in range(n))
    bm = sum(ys[i] * ab[i][1] for i in range(n))
    A = am * P / (R_GAS * T) ** 2
    B = bm * P / (R_GAS * T)
    return A, B, am, bm, ab, aij


def pr_Z(A, B):
    """Vapour compressibility: largest real root of the PR cubic
    Z^3 - (1-B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0."""
    return cubic_largest_root(-(1.0 - B), A - 3.0 * B * B - 2.0 * B, -(A * B - B * B - B * B * B))


def pr_lnphi(T, P, ys, crit, kij):
    """ln of the mixture fugacity coefficients phi_hat_i and Z (vapour root)."""
    A, B, am, bm, ab, aij = pr_mix(T, P, ys, crit, kij)
    Z = pr_Z(A, B)
    logterm = math.log((Z + (1.0 + SQRT2) * B) / (Z + (1.0 - SQRT2) * B))
    out = []
    for i in range(len(ys)):
        bi = ab[i][1]
        sa = sum(ys[j] * aij[i][j] for j in range(len(ys)))
        out.append(bi / bm * (Z - 1.0) - math.log(Z - B)
                   - A / (2.0 * SQRT2 * B) * (2.0 * sa / am - bi / bm) * logterm)
    return out, Z


def pr_lnphi_mixture(T, P, ys, crit, kij):
    """ln of the mixture fugacity coefficient, ln phi = Z - 1 - ln(Z-B) - A/(2 sqrt2 B) ln(...).

    Used only to pin pr_lnphi: ln phi_hat_i is the n_i-derivative of n ln phi.
    """
    A, B, am, bm, ab, aij = pr_mix(T, P, ys, crit, kij)
    Z = pr_Z(A, B)
    return Z - 1.0 - math.log(Z - B) - A / (2.0 * SQRT2 * B) * math.log((Z + (1.0 + SQRT2) * B) / (Z + (1.0 - SQRT2) * B))


def _crit(cfg):
    return [(cfg["Tc"], cfg["Pc"], cfg["omega_ac"]), (cfg["Tc_g"], cfg["Pc_g"], cfg["omega_g"])]


def rho_liquid(cfg, T):
    """Liquid density rho_L(T) = rho_l + (d rho_L / dT)(T - T_drop): the paper takes it from
    property correlations (Sec. 2.7) and lets it change the volume (Eqs. alphasource,
    pequation); here a linear law through the configured density at the initial liquid
    temperature stands in for them (reading R31; drho_l_dT = 0: constant density)."""
    return cfg["rho_l"] + cfg.get("drho_l_dT", 0.0) * (np.asarray(T, dtype=np.float64) - cfg["T_drop"])


def y_pr_scalar(cfg, T):
    """Eq. (equilibirumyi) for one cell: x = 1 (pure liquid fuel), fixed point in y.

    y <- p0 phi_pure(T, p0) exp(v_L (p - p0)/(R T)) / (p phi_hat_fuel(T, p, y)),
    started from the Raoult value, at most 50 iterations, stop when |dy| < 1e-13.
    """
    P = cfg["P"]
    crit = _crit(cfg)
    kij = cfg["kij"]
    p0 = float(psat(cfg, T))
    vL = cfg["M_l"] / float(rho_liquid(cfg, T))
    lnphi_pure, _ = pr_lnphi(T, p0, [1.0, 0.0], crit, kij)
    num = p0 * math.exp(lnphi_pure[0]) * math.exp(vL * (P - p0) / (R_GAS * T))
    y = min(p0 / P, Y_CLAMP)
    for _ in range(50):
        lnphi, _ = pr_lnphi(T, P, [y, 1.0 - y], crit, kij)
        y_new = min(num / (P * math.exp(lnphi[0])), Y_CLAMP)
        dy = abs(y_new - y)
        y = y_new
        if dy < 1e-13:
            break
    return y


def Z_gas_scalar(cfg, T, Y):
    """PR compressibility of the local gas mixture (fuel mass fraction Y)."""
    y = float(y_from_Y(cfg, Y))
    A, B, *_ = pr_mix(T, cfg["P"], [y, 1.0 - y], _crit(cfg), cfg["kij"])
    return pr_Z(A, B)


def Y_eq(cfg, T):
    """Saturation vapour mass fraction at temperature T (array), Sec. 2.5."""
    T = np.asarray(T, dtype=np.float64)
    if cfg["eq_model"] == 0:
        y = y_raoult(cfg, T)
    else:
        y = np.vectorize(lambda t: y_pr_scalar(cfg, float(t)), otypes=[np.float64])(T)
    return Y_from_y(cfg, y)


def rho_gas(cfg, T, Y):
    """Eq. (densitygas): rho_G = p M_w / (Z R T); Z = 1 for the Raoult model."""
    T = np.asarray(T, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if cfg["const_props_check"]:
        return np.full(T.shape, cfg["P"] * cfg["M_g"] / (R_GAS * cfg["T_amb"]))
    inv_m = Y / cfg["M_l"] + (1.0 - Y) / cfg["M_g"]
    if cfg["eq_model"] == 0:
        Z = np.ones_like(T)
    else:
        Z = np.vectorize(lambda t, yy: Z_gas_scalar(cfg, float(t), float(yy)), otypes=[np.float64])(T, Y)
    return cfg["P"] / (Z * R_GAS * T * inv_m)


def D_gas(cfg):
    """Binary diffusivity at the operating pressure: D_g given at 1 bar, scaled 1/p."""
    return cfg["D_g"] * (1.0e5 / cfg["P"])
