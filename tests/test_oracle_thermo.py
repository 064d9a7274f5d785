"""Pins of the oracle's thermodynamics (Sec. 2.5, Eqs. equilibrium, equilibirumyi, densitygas)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import thermo as th
from paper_2005_02867_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "heptane_thermo.json")))


def test_psat_anchored_at_boiling_point():
    cfg = W.make()
    assert float(th.psat(cfg, cfg["Tb"])) == pytest.approx(101325.0, rel=1e-15)
    assert float(th.psat(cfg, 300.0)) == pytest.approx(GOLD["psat_300K_Pa"], rel=2e-4)


def test_saturation_and_d2_constants():
    cfg = W.make()
    Ys = float(th.Y_eq(cfg, np.array([300.0]))[0])
    assert Ys == pytest.approx(GOLD["Y_s_300K_1bar"], abs=1e-5)
    B = Ys / (1.0 - Ys)
    assert B == pytest.approx(GOLD["B_Y"], abs=1e-5)
    assert math.log(1.0 + B) == pytest.approx(GOLD["ln_1pB"], abs=1e-5)
    cfg1 = W.cfg1_d2law()
    rg = float(th.rho_gas(cfg1, np.array([300.0]), np.array([0.1]))[0])
    assert rg == pytest.approx(GOLD["rho_g_773K_1bar"], abs=1e-5)
    K = 8.0 * rg * cfg1["D_g"] * math.log(1.0 + B) / cfg1["rho_l"]
    assert K == pytest.approx(GOLD["K_d2_m2_per_s"], rel=2e-4)


def test_mole_mass_fraction_roundtrip():
    cfg = W.make()
    Y = np.linspace(0.0, 1.0, 11)
    assert np.allclose(th.Y_from_y(cfg, th.y_from_Y(cfg, Y)), Y, atol=1e-15)


@pytest.mark.parametrize("roots", [(-1.0, 0.5, 2.0), (0.01, 0.02, 0.9), (1.0, 1.0 + 1e-3, 1.0 + 2e-3)])
def test_cardano_three_real_roots(roots):
    r1, r2, r3 = roots
    c2 = -(r1 + r2 + r3)
    c1 = r1 * r2 + r1 * r3 + r2 * r3
    c0 = -r1 * r2 * r3
    assert th.cubic_largest_root(c2, c1, c0) == pytest.approx(max(roots), rel=1e-7)


@pytest.mark.parametrize("r,re,im", [(0.95, 0.1, 0.2), (0.3, -1.0, 2.0), (5.0, 0.0, 1e-3)])
def test_cardano_one_real_root(r, re, im):
    # (z - r)(z^2 - 2 re z + re^2 + im^2)
    s = re * re + im * im
    c2 = -(r + 2 * re)
    c1 = s + 2 * r * re
    c0 = -r * s
    assert th.cubic_largest_root(c2, c1, c0) == pytest.approx(r, rel=1e-12)


def _crit(cfg):
    return [(cfg["Tc"], cfg["Pc"], cfg["omega_ac"]), (cfg["Tc_g"], cfg["Pc_g"], cfg["omega_g"])]


def test_pr_root_reproduces_pressure():
    """The vapour root put back into the PR equation p = RT/(v-b) - a/(v^2+2bv-b^2)."""
    cfg = W.cfg3_cart3d(nc=8)
    for T, P, y in [(500.0, 20e5, 0.2), (773.0, 20e5, 0.05), (400.0, 1e5, 0.5)]:
        ys = [y, 1 - y]
        A, B, am, bm, *_ = th.pr_mix(T, P, ys, _crit(cfg), 0.0)
        Z = th.pr_Z(A, B)
        v = Z * th.R_GAS * T / P
        p_back = th.R_GAS * T / (v - bm) - am / (v * v + 2 * bm * v - bm * bm)
        assert p_back == pytest.approx(P, rel=1e-10)


def test_pr_ideal_gas_limit():
    cfg = W.cfg3_cart3d(nc=8)
    lnphi, Z = th.pr_lnphi(600.0, 1.0, [0.3, 0.7], _crit(cfg), 0.0)
    assert abs(Z - 1.0) < 1e-6 and max(abs(x) for x in lnphi) < 1e-6


def test_pr_partial_molar_and_gibbs_duhem():
    """ln phi_hat_i = d(n ln phi)/dn_i (central FD) and sum_i y_i d ln phi_hat_i = 0."""
    cfg = W.cfg3_cart3d(nc=8)
    crit = _crit(cfg)
    T, P = 650.0, 20e5
    n = np.array([0.3, 0.7])
    lnphi, _ = th.pr_lnphi(T, P, list(n / n.sum()), crit, 0.0)
    h = 1e-6
    for i in range(2):
        npl, nmi = n.copy(), n.copy()
        npl[i] += h
        nmi[i] -= h
        fp = npl.sum() * th.pr_lnphi_mixture(T, P, list(npl / npl.sum()), crit, 0.0)
        fm = nmi.sum() * th.pr_lnphi_mixture(T, P, list(nmi / nmi.sum()), crit, 0.0)
        assert (fp - fm) / (2 * h) == pytest.approx(lnphi[i], abs=1e-7)
    y = 0.3
    dy = 1e-6
    lp, _ = th.pr_lnphi(T, P, [y + dy, 1 - y - dy], crit, 0.0)
    lm, _ = th.pr_lnphi(T, P, [y - dy, 1 - y + dy], crit, 0.0)
    gd = y * (lp[0] - lm[0]) + (1 - y) * (lp[1] - lm[1])
    assert abs(gd / (2 * dy)) < 1e-7


def test_pr_equilibrium_fixed_point():
    cfg = W.cfg3_cart3d(nc=8)
    crit = _crit(cfg)
    for T in (300.0, 400.0, 500.0):
        y = th.y_pr_scalar(cfg, T)
        p0 = float(th.psat(cfg, T))
        lpure, _ = th.pr_lnphi(T, p0, [1.0, 0.0], crit, 0.0)
        lmix, _ = th.pr_lnphi(T, cfg["P"], [y, 1 - y], crit, 0.0)
        vL = cfg["M_l"] / cfg["rho_l"]
        lhs = p0 * math.exp(lpure[0]) * math.exp(vL * (cfg["P"] - p0) / (th.R_GAS * T))
        rhs = cfg["P"] * y * math.exp(lmix[0])
        assert lhs == pytest.approx(rhs, rel=1e-11)


def test_pr_reduces_to_raoult_at_low_pressure():
    cfg = W.cfg3_cart3d(nc=8, P=5000.0)
    T = 250.0
    y_pr = th.y_pr_scalar(cfg, T)
    y_id = float(th.y_raoult(cfg, T))
    assert y_pr == pytest.approx(y_id, rel=1e-2)
    # at 20 bar the non-ideality is large: the PR value differs from Raoult
    cfg20 = W.cfg3_cart3d(nc=8)
    assert abs(th.y_pr_scalar(cfg20, 450.0) / float(th.y_raoult(cfg20, 450.0)) - 1.0) > 0.05
