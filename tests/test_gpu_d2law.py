"""The d2 law on the GPU (Sec. 1 and Sec. 4: once the initial transient is over the
squared diameter of an isolated droplet falls linearly, K = 8 rho_g D ln(1 + B_Y) /
rho_l): the constant-property microgravity case run for 25 ms (five times r_s^2/D),
the slope fitted over the second half, as in the oracle's pin.

- FP64 on 64 x 128 against the oracle's run of the same case: the same slope.
- Mixed precision against FP64 at the accuracy the spec asks of it: d2 slope
  within 1e-3, droplet volume within 1e-5 -- at the benchmark's solver tolerances
  (1e-8) as well as at tight ones.
- Refinement 64 x 128 -> 128 x 256 -> 256 x 512 at a fixed Courant number (dt
  halved with h: 1e-4, 5e-5, 2.5e-5 s; the Stefan velocity stays near 0.03 m/s, a
  Courant number below 0.1): the method reads the flux one to two cells outside the
  surface, where the spherical flux density is lower by (r_s / r)^2, so the rate rises
  under refinement at first order (each increment at least a third smaller than the
  one before: 0.771 -> 0.869 -> 0.892 K) towards K times the finite-domain factor, and
  lies within [1.0, 1.143] K +- 15 % from 128 x 256 on.  At a Courant number
  near 0.2 (256 x 512 with dt 1e-4 s) the compressive scheme lets the interface
  widen by a few cells over the run and some interface cells find no gas cell
  within three cells: the runs check that this flag stays clear.
"""
import math

import numpy as np
import pytest

from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 250


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_02867_gb300 import _build, droplet
    _build.build_library()
    droplet.load_library()
    torch.cuda.set_device(0)
    return droplet


def slope(t, d2):
    t, d2 = np.asarray(t), np.asarray(d2)
    h = len(t) // 2
    return -float(np.polyfit(t[h:], d2[h:], 1)[0])


def run(D, n=64, precision=0, rtol=1e-10):
    """25 ms of the check case on n x 2n cells, dt = 1e-4 s x 64 / n."""
    cfg = W.cfg1_d2law(n=(n, 2 * n, 1), dt=1e-4 * 64 / n, precision=precision, cg_rtol=rtol, helm_rtol=rtol)
    sim = D.Droplet(cfg)
    t, d2 = [], []
    flags = 0
    for _ in range(STEPS * n // 64):
        assert sim.step(1) == 0
        d = sim.diag()
        flags |= d["flags"]
        t.append(d["t"])
        d2.append(d["d2"])
    V = d["V_l"]
    sim.close()
    assert not flags & D.FLAG_ADJ_NOT_FOUND, (n, flags)
    return slope(t, d2), V, cfg


def d2_constant(cfg):
    """K from the thermodynamics of the configuration: Raoult with Clausius-Clapeyron
    at T_drop, ideal-gas rho_g at T_amb (frozen in the check mode)."""
    R = 8.314462618
    p0 = 101325.0 * math.exp(cfg["Lv"] * cfg["M_l"] / R * (1.0 / cfg["Tb"] - 1.0 / cfg["T_drop"]))
    y = p0 / cfg["P"]
    Ys = y * cfg["M_l"] / (y * cfg["M_l"] + (1.0 - y) * cfg["M_g"])
    rg = cfg["P"] * cfg["M_g"] / (R * cfg["T_amb"])
    return 8.0 * rg * cfg["D_g"] * math.log(1.0 + Ys / (1.0 - Ys)) / cfg["rho_l"]


@pytest.fixture(scope="module")
def oracle_slope():
    """The oracle's d2 slope and final volume of the 64 x 128 case."""
    from oracle import step as O
    cfg = W.cfg1_d2law()
    st = O.init_state(cfg)
    t, d2 = [], []
    for _ in range(STEPS):
        st = O.step(cfg, st)
        d = O.diagnostics(cfg, st)
        t.append(d["t"])
        d2.append(d["d2"])
    return slope(t, d2), d["V_l"]


def test_d2_slope_fp64_matches_oracle(D, oracle_slope):
    ko, vo = oracle_slope
    k64, v64, _ = run(D, 64, 0, rtol=1e-12)
    assert abs(k64 - ko) <= 1e-6 * ko, (k64, ko)
    assert abs(v64 - vo) <= 1e-10 * vo, (v64, vo)


def test_d2_slope_mixed_matches_oracle(D, oracle_slope):
    """Mixed precision at the benchmark's solver tolerances against the FP64 oracle."""
    ko, vo = oracle_slope
    k32, v32, _ = run(D, 64, 1, rtol=1e-8)
    assert abs(k32 - ko) <= 1e-3 * ko, (k32, ko)
    assert abs(v32 - vo) <= 1e-5 * vo, (v32, vo)


@pytest.mark.parametrize("rtol", [1e-10, 1e-8])
def test_d2_slope_mixed_vs_fp64(D, rtol):
    k64, v64, _ = run(D, 64, 0, rtol)
    k32, v32, _ = run(D, 64, 1, rtol)
    assert k64 > 0.0
    assert abs(k32 - k64) <= 1e-3 * k64, (k32, k64)
    assert abs(v32 - v64) <= 1e-5 * v64, (v32, v64)


def test_d2_slope_converges_to_K(D):
    K = d2_constant(W.cfg1_d2law())
    r = {n: run(D, n, 0)[0] / K for n in (64, 128, 256)}
    inc = (r[128] - r[64], r[256] - r[128])
    assert inc[0] > 0.0 and abs(inc[1]) < 0.67 * inc[0], r
    assert 0.85 <= r[128] <= 1.31 and 0.85 <= r[256] <= 1.31, r
