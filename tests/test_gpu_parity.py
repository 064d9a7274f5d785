"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Parity mode solves every linear system to a relative residual of 1e-16, so
that one step from an identical state agrees to 1e-10 relative in every field
(the pressure system's kappa * eps floor is far below that at these
tolerances).  Multi-step runs compare trajectories; the full-size 3D case is
checked on sampled cells and through invariants that hold at any size.
"""
import math

import numpy as np
import pytest

from oracle import step as O
from oracle.grid import Grid
from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAR = dict(cg_rtol=1e-16, helm_rtol=1e-16, cg_maxit=300, helm_maxit=600)
TOL = 1e-10


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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def set_state(sim, G, st, cfg=None):
    for nm in ("alpha", "T", "omega", "p", "rhoG"):
        sim.set(nm, st[nm].ravel(order="F"))
    for a in G.act:
        sim.set("u%d" % a, st["u"][a].ravel(order="F"))
    if cfg is not None and cfg.get("drho_l_dT", 0.0) != 0.0 and "expand" in st:
        sim.set("expand", st["expand"].ravel(order="F"))   # the previous step's expansion term


def compare_state(sim, G, st, tol, extra_aux=None):
    errs = {}
    for nm in ("alpha", "T", "omega", "rhoG", "p"):
        errs[nm] = rel(sim.get(nm), st[nm].ravel(order="F"))
    for a in G.act:
        errs["u%d" % a] = rel(sim.get("u%d" % a), st["u"][a].ravel(order="F"))
    if extra_aux is not None:
        for nm in ("mdot", "mraw", "alpha_star", "dp", "S", "rhoG_old"):
            errs[nm] = rel(sim.get(nm), extra_aux[nm].ravel(order="F"))
        for a in G.act:
            errs["ustar%d" % a] = rel(sim.get("ustar%d" % a), extra_aux["ustar"][a].ravel(order="F"))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    return errs


SMALL = dict(n=(32, 64, 1), L=(2e-3, 4e-3, 0.0), xc=(0.0, 2e-3, 0.0))
CASES = {
    "axisym-natural": (W.cfg1_axisym_64x128(**SMALL, **PAR), 3),
    "axisym-gravity": (W.cfg5_axisym_128x256(**SMALL, **PAR), 3),
    "axisym-ragged-24x40": (W.cfg5_axisym_128x256(n=(24, 40, 1), L=(1.5e-3, 2.5e-3, 0.0), xc=(0.0, 1.25e-3, 0.0),
                                                  D0=0.8e-3, **PAR), 2),
    "axisym-d2law": (W.cfg1_d2law(**SMALL, **PAR), 3),
    "axisym-forced-inlet": (W.cfg5_axisym_128x256(**SMALL, bc_mode=1, u_inflow=0.3, **PAR), 2),
    "cart3d-natural-16": (W.make(geom=1, n=(16, 16, 16), L=(1.6e-3,) * 3, xc=(0.8e-3,) * 3, D0=0.8e-3,
                                 g=(0, 0, -9.81), **PAR), 2),
    "cart3d-pr-forced-16": (W.cfg3_cart3d(nc=16, L=(1.6e-3,) * 3, xc=(0.8e-3,) * 3, precision=0, **PAR), 1),
    "cart3d-ragged-12x10x14": (W.make(geom=1, n=(12, 10, 14), L=(1.2e-3, 1.0e-3, 1.4e-3), xc=(0.6e-3, 0.5e-3, 0.7e-3),
                                      D0=0.6e-3, g=(0, 0, -9.81), **PAR), 1),
}


# The launched (multi-kernel) solvers that grids beyond 2^22 cells use -- the
# multigrid-preconditioned CG with its one-block coarse tail, and the FP64 Jacobi-PCG
# -- selected at small sizes (solver_select = 1), so that the path of the 256^3 grid
# is held to the same element-wise parity.
LAUNCHED = {name + "-launched": (dict(cfg, solver_select=1), pre)
            for name, (cfg, pre) in CASES.items()
            if name in ("axisym-natural", "axisym-gravity", "axisym-ragged-24x40", "cart3d-natural-16",
                        "cart3d-pr-forced-16", "cart3d-ragged-12x10x14")}
CASES.update(LAUNCHED)
# Geometric interface advection (adv_scheme = 1): a plane per partly filled cell and one
# sweep per axis, FP64 in both precisions
GEOMETRIC = {name + "-geometric": (dict(cfg, adv_scheme=1), pre)
             for name, (cfg, pre) in list(CASES.items())
             if name in ("axisym-gravity", "axisym-ragged-24x40", "axisym-d2law", "axisym-forced-inlet",
                         "cart3d-natural-16", "cart3d-pr-forced-16", "cart3d-ragged-12x10x14")}
CASES.update(GEOMETRIC)
# A temperature-dependent liquid density (drho_l_dT, n-heptane's ~ -0.9 kg m^-3 K^-1): the
# mixture density, the evaporation flux, the alpha source and the continuity source's
# expansion term, on both advection schemes and both solver paths
EXPANDING = {name + "-expanding": (dict(cfg, drho_l_dT=-0.9), pre)
             for name, (cfg, pre) in list(CASES.items())
             if name in ("axisym-gravity", "axisym-natural", "cart3d-natural-16", "axisym-gravity-launched",
                         "axisym-gravity-geometric", "cart3d-ragged-12x10x14-geometric")}
CASES.update(EXPANDING)
# The spherical fibre inside the droplet (fiber = 1, Table tableboundary "sphere" row): 8 solid
# cells in 2D (radius 0.15 mm at h = 62.5 um), 56 in 3D (0.22 mm at h = 0.1 mm), on both
# solver paths, with natural convection, gravity and a forced flow past it
FIBRE = {name + "-fibre": (dict(cfg, fiber=1, fiber_radius=1.5e-4 if cfg["geom"] == 0 else 2.2e-4), pre)
         for name, (cfg, pre) in list(CASES.items())
         if name in ("axisym-gravity", "axisym-gravity-launched", "axisym-forced-inlet", "cart3d-natural-16",
                     "cart3d-natural-16-launched", "cart3d-pr-forced-16")}
CASES.update(FIBRE)
# Vapour and inert gas of different heat capacities (c_p,v = 2400 against c_p,g = 1100 J/kg/K):
# the species-diffusion enthalpy term of Eq. Teqn in the energy rows (reading R33), on both
# solver paths, with the fibre and on a ragged 3D grid
HEATCAP = {name + "-heatcap": (dict(cfg, cp_v=2400.0), pre)
           for name, (cfg, pre) in list(CASES.items())
           if name in ("axisym-natural", "axisym-gravity-launched", "axisym-gravity-fibre", "cart3d-natural-16",
                       "cart3d-pr-forced-16", "cart3d-ragged-12x10x14")}
CASES.update(HEATCAP)


@pytest.mark.parametrize("name", list(CASES))
def test_init_parity(D, name):
    cfg, _ = CASES[name]
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    st = O.init_state(cfg)
    assert np.array_equal(sim.get("alpha"), st["alpha"].ravel(order="F"))   # integer sample counts: exact
    for nm in ("T", "omega", "rhoG"):
        assert rel(sim.get(nm), st[nm].ravel(order="F")) < 1e-14, nm
    for a in G.act:
        assert np.array_equal(sim.get("u%d" % a), st["u"][a].ravel(order="F"))
    sim.close()


@pytest.mark.parametrize("name", list(CASES))
def test_single_step_parity_from_identical_state(D, name):
    cfg, pre = CASES[name]
    G = Grid(cfg)
    st = O.init_state(cfg)
    for _ in range(pre):
        st = O.step(cfg, st)
    sim = D.Droplet(cfg)
    set_state(sim, G, st, cfg)
    rc = sim.step(1)
    assert rc == 0
    st1 = O.step(cfg, st, keep=True)
    compare_state(sim, G, st1, TOL, extra_aux=st1["aux"])
    if cfg.get("drho_l_dT", 0.0) != 0.0:
        assert np.abs(st1["expand"]).max() > 0.0
        assert rel(sim.get("expand"), st1["expand"].ravel(order="F")) <= TOL
    d = sim.diag()
    od = O.diagnostics(cfg, st1)
    for k in ("mdot_tot", "K_norm", "T_s_mean", "M_vap", "max_u", "M_liq"):
        assert abs(d[k] - od[k]) <= TOL * max(abs(od[k]), 1e-30), (k, d[k], od[k])
    # the liquid volume is bookkept exactly step to step: compare with the oracle's diagnostic directly
    assert abs(d["V_l"] - od["V_l"]) <= 1e-13 * od["V_l"]
    sim.close()


def test_trajectory_parity_config1(D):
    """Config 1 as specified (64 x 128, zero gravity, Raoult, 773 K, 1 bar, FP64,
    dt 1e-5 s, 200 steps): the two trajectories from the same initial state, every
    field and the diagnostics.  Each system is solved to 1e-16 on both sides and one
    step agrees to 1e-12 ... 1e-15; along the run the differences add up: alpha, T,
    omega, p_rgh and rho_G stay within 1e-10 (measured ~1e-11), the velocities, which
    follow the pressure increment of a system with condition number ~1e7, within 5e-10
    (measured 2.2e-10), and so does the evaporation rate, which carries the convective
    flux (measured 2.3e-10); the other diagnostics within 1e-10."""
    cfg = W.cfg1_axisym_64x128(**PAR)
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    st = O.init_state(cfg)
    for _ in range(200):
        assert sim.step(1) == 0
        st = O.step(cfg, st)
    errs = compare_state(sim, G, st, 5e-10)
    assert max(errs[k] for k in ("alpha", "T", "omega", "rhoG", "p")) <= TOL, errs
    print("config 1, 200 steps:", {k: float("%.2g" % v) for k, v in errs.items()})
    d, od = sim.diag(), O.diagnostics(cfg, st)
    for k in ("V_l", "d2", "T_s_mean", "M_vap", "vap_out_cum"):
        assert abs(d[k] - od[k]) <= TOL * max(abs(od[k]), 1e-30), (k, d[k], od[k], errs)
    # the evaporation rate carries the convective flux rho omega v at the adjacent cells
    assert abs(d["mdot_tot"] - od["mdot_tot"]) <= 5e-10 * abs(od["mdot_tot"]), (d["mdot_tot"], od["mdot_tot"])
    sim.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_thermal_expansion_trajectory_parity(D, scheme):
    """The heated, expanding droplet of the oracle's thermal-expansion pin (32 x 64, no
    evaporation, drho_l_dT = -0.9, 10 ms): 100 steps on both sides from the same initial
    state, every field, the expansion term, and the volume and liquid mass they move."""
    cfg = W.make(n=(32, 64, 1), L=(2e-3, 4e-3, 0.0), xc=(0.0, 2e-3, 0.0), D0=1e-3, T_amb=500.0,
                 physics_mask=W.PHYS_ENERGY | W.PHYS_FLOW, dt=1e-4, drho_l_dT=-0.9, adv_scheme=scheme, **PAR)
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    st = O.init_state(cfg)
    for _ in range(100):
        assert sim.step(1) == 0
        st = O.step(cfg, st)
    errs = compare_state(sim, G, st, 5e-10)
    assert rel(sim.get("expand"), st["expand"].ravel(order="F")) <= 5e-10
    print("thermal expansion, 100 steps:", {k: float("%.2g" % v) for k, v in errs.items()})
    d, od = sim.diag(), O.diagnostics(cfg, st)
    d0 = O.diagnostics(cfg, O.init_state(cfg))
    assert od["V_l"] > d0["V_l"] * (1 + 1e-3)             # the volume grew
    for k in ("V_l", "M_liq"):
        assert abs(d[k] - od[k]) <= TOL * od[k], (k, d[k], od[k])
    sim.close()


@pytest.mark.parametrize("solver_select", [0, 1])
def test_courant_adaptive_step_parity(D, solver_select):
    """Courant-adaptive time step (co_max > 0): the device forms each next dt from the
    face velocities it has just reduced, with the oracle's rule and operations, so the
    clocks agree step by step to the velocities' rounding differences (each dt is
    co h / max|u|: the clock inherits the velocities' relative differences, measured
    2e-12 ... 4.4e-12), and after eight steps in which the Courant limit binds the
    fields agree to 1e-10 and the velocities, still small as they start from rest and
    so larger in relative terms, to 1e-9 (measured 2.3e-10 ... 4.1e-10)."""
    cfg = W.cfg5_axisym_128x256(**SMALL, dt=4e-5, co_max=0.01, solver_select=solver_select, **PAR)
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    st = O.init_state(cfg)
    for _ in range(8):
        assert sim.step(1) == 0
        st = O.step(cfg, st)
        assert sim.diag()["t"] == pytest.approx(st["t"], rel=TOL, abs=0.0)
    assert st["dt"] < cfg["dt"]                  # the limit binds
    errs = compare_state(sim, G, st, 1e-9)
    assert max(errs[k] for k in ("alpha", "T", "omega", "rhoG", "p")) <= TOL, errs
    sim.close()


def test_mixed_precision_matches_fp64(D):
    """FP32 multigrid preconditioner inside the FP64 CG: same discrete answer."""
    cfg64 = W.cfg5_axisym_128x256(**SMALL, cg_rtol=1e-12, helm_rtol=1e-12)
    cfg32 = dict(cfg64, precision=1)
    a, b = D.Droplet(cfg64), D.Droplet(cfg32)
    for _ in range(10):
        a.step(1)
        b.step(1)
    da, db = a.diag(), b.diag()
    assert abs(da["V_l"] - db["V_l"]) <= 1e-5 * da["V_l"]
    assert rel(b.get("alpha"), a.get("alpha")) < 1e-6
    assert rel(b.get("T"), a.get("T")) < 1e-6
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["axisym-gravity-fibre", "cart3d-pr-forced-16-fibre"])
def test_fibre_in_mixed_precision(D, name):
    """The fibre in mixed precision (binary32 assembly increments, FP32 solves): over ten
    steps (2D; three in 3D) it follows the FP64 path of the same case (droplet volume 1e-5,
    alpha and T 1e-5, solver tolerances 1e-10), and its sphere stays closed: no liquid in
    the solid cells, their temperature kept (1e-9), zero velocity on every sphere face."""
    cfg64 = dict(CASES[name][0], cg_rtol=1e-10, helm_rtol=1e-10)
    cfg32 = dict(cfg64, precision=1)
    G = Grid(cfg64)
    solid = O.solid_mask(cfg64, G).ravel(order="F")
    a, b = D.Droplet(cfg64), D.Droplet(cfg32)
    T0 = b.get("T")[solid].copy()
    for _ in range(10 if G.axisym else 3):
        assert a.step(1) == 0 and b.step(1) == 0
    da, db = a.diag(), b.diag()
    assert abs(da["V_l"] - db["V_l"]) <= 1e-5 * da["V_l"]
    assert rel(b.get("alpha"), a.get("alpha")) < 1e-5
    assert rel(b.get("T"), a.get("T")) < 1e-5
    assert b.get("alpha")[solid].max() == 0.0
    assert np.abs(b.get("T")[solid] - T0).max() <= 1e-9 * T0.max()
    Ps = O._pad(G, O.solid_mask(cfg64, G))
    for c in G.act:
        fs = O.fshape(G, c)
        sph = (O._view(G, Ps, fs, {c: -1}) | O._view(G, Ps, fs, {c: 0})).ravel(order="F")
        assert np.abs(b.get("u%d" % c)[sph]).max() == 0.0
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["axisym-natural-heatcap", "cart3d-pr-forced-16-heatcap"])
def test_heat_capacities_in_mixed_precision(D, name):
    """The enthalpy term of different heat capacities in mixed precision (formed in binary32
    from the copies of rho D, omega and T): over ten steps (2D; three in 3D) the run follows
    the FP64 path of the same case (droplet volume 1e-5, alpha and T 1e-5, solver tolerances
    1e-10), ten times closer than the FP64 run with equal heat capacities is."""
    cfg64 = dict(CASES[name][0], cg_rtol=1e-10, helm_rtol=1e-10)
    cfg32 = dict(cfg64, precision=1)
    G = Grid(cfg64)
    a, b, c = D.Droplet(cfg64), D.Droplet(cfg32), D.Droplet(dict(cfg64, cp_v=cfg64["cp_g"]))
    for _ in range(10 if G.axisym else 3):
        assert a.step(1) == 0 and b.step(1) == 0 and c.step(1) == 0
    da, db = a.diag(), b.diag()
    assert abs(da["V_l"] - db["V_l"]) <= 1e-5 * da["V_l"]
    assert rel(b.get("alpha"), a.get("alpha")) < 1e-5
    assert rel(b.get("T"), a.get("T")) < 1e-5
    assert rel(c.get("T"), a.get("T")) > 10.0 * rel(b.get("T"), a.get("T"))
    a.close()
    b.close()
    c.close()


@pytest.mark.parametrize("shape", [(128, 96, 1), (32, 24, 20), (176, 176, 176)])
def test_launched_binary32_multigrid(D, shape):
    """The launched V-cycle of a binary32 hierarchy (the path of the large mixed grids): the
    prolongation folded into the first post-smoothing half sweep of every level above the
    one-block coarse solve (one such level on 128 x 96 and 32 x 24 x 20, four at 176^3), and on
    the levels of 2^20 or more updated cells (176^3) the half sweeps at two cells a thread.  Over a few steps the mixed run follows the FP64 run of the same case (both on the
    launched solvers): droplet volume 1e-5, alpha and T 1e-5."""
    if shape[2] == 1:
        cfg64 = W.cfg5_axisym_128x256(n=shape, L=(shape[0] * 6.25e-5, shape[1] * 6.25e-5, 0.0),
                                      xc=(0.0, shape[1] * 3.125e-5, 0.0), D0=0.8e-3)
    else:
        h = 1.0e-4 if shape[0] < 64 else 2.0e-5
        Lx = tuple(m * h for m in shape)
        cfg64 = W.make(geom=1, n=shape, L=Lx, xc=tuple(0.5 * x for x in Lx), D0=0.5 * min(Lx),
                       g=(0, 0, -9.81), dt=2e-6)
    cfg64 = dict(cfg64, solver_select=1, cg_rtol=1e-10, helm_rtol=1e-10)
    cfg32 = dict(cfg64, precision=1)
    a, b = D.Droplet(cfg64), D.Droplet(cfg32)
    for _ in range(4 if shape[0] < 64 else 2):
        assert a.step(1) == 0 and b.step(1) == 0
    da, db = a.diag(), b.diag()
    assert abs(da["V_l"] - db["V_l"]) <= 1e-5 * da["V_l"]
    assert rel(b.get("alpha"), a.get("alpha")) < 1e-5
    assert rel(b.get("T"), a.get("T")) < 1e-5
    a.close()
    b.close()


def test_fibre_finer_than_the_grid_is_no_fibre(D):
    """A fibre radius below every cell-centre distance leaves no solid cell: the run is the
    run without a fibre (the same radius D_f of the potential xi), bit for bit (the fibre's
    tests are then off altogether)."""
    cfg = dict(CASES["axisym-gravity"][0], fiber_radius=1e-7)
    a, b = D.Droplet(cfg), D.Droplet(dict(cfg, fiber=1))
    for _ in range(2):
        assert a.step(1) == 0 and b.step(1) == 0
    for f in ("alpha", "T", "omega", "p", "u0", "u1"):
        assert np.array_equal(a.get(f), b.get(f)), f
    a.close()
    b.close()


def test_not_converged_is_reported_and_state_advances(D):
    cfg = W.cfg1_axisym_64x128(**SMALL, cg_maxit=1, cg_rtol=1e-16)
    sim = D.Droplet(cfg)
    rc = sim.step(1)
    assert rc == D.ERR_NOT_CONVERGED
    d = sim.diag()
    assert d["step"] == 1 and d["its_p"] == 1
    sim.close()


def test_field_size_mismatch(D):
    cfg = W.cfg1_axisym_64x128(**SMALL)
    sim = D.Droplet(cfg)
    with pytest.raises(D.DropletError) as e:
        sim.set("alpha", np.zeros(10))
    assert e.value.status == -5
    sim.close()


def test_config2_full_size_one_step(D):
    """Config 2 grid (256 x 512, gravity, centripetal force): one step from the
    initial state, every field against the oracle."""
    cfg = W.cfg2_axisym_256x512(precision=0, **PAR)
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    st = O.init_state(cfg)
    assert sim.step(1) == 0
    st1 = O.step(cfg, st)
    compare_state(sim, G, st1, TOL)
    sim.close()


def _alpha_bruteforce(cfg, G, cell):
    """Sample count of one 3D cell by the plain definition (8^3 points)."""
    S = 8
    R2 = (0.5 * cfg["D0"]) ** 2
    cnt = 0
    for m0 in range(S):
        for m1 in range(S):
            for m2 in range(S):
                d2 = 0.0
                for a, m in zip(range(3), (m0, m1, m2)):
                    x = (cell[a] + (m + 0.5) / S) * G.h[a]
                    d2 = d2 + (x - cfg["xc"][a]) ** 2
                cnt += d2 <= R2
    return cnt / S ** 3


def test_config3_full_size_sampled_and_invariants(D):
    """Config 3 at its full 256^3 size in the benchmark's settings: initial
    alpha on sampled cells by brute force, then after two steps alpha in
    [0, 1], exact liquid-volume bookkeeping, and div u = S to the solver
    tolerance."""
    cfg = W.cfg3_cart3d()
    G = Grid(cfg)
    sim = D.Droplet(cfg)
    a0 = sim.get("alpha").reshape(G.n, order="F")
    rng = np.random.default_rng(7)
    c = (np.array(cfg["xc"]) / np.array(G.h)).astype(int)
    samples = [tuple(c + rng.integers(-14, 15, 3)) for _ in range(24)] + [tuple(rng.integers(0, 256, 3)) for _ in range(8)]
    for cell in samples:
        assert a0[cell] == _alpha_bruteforce(cfg, G, cell), cell
    V = G.V
    vol0 = float(np.sum(a0 * V))
    assert vol0 == pytest.approx(math.pi / 6 * cfg["D0"] ** 3, rel=2e-3)
    d0 = sim.diag()
    sim.step(1)
    a1 = sim.get("alpha").reshape(G.n, order="F")
    d1 = sim.diag()
    mdot = sim.get("mdot").reshape(G.n, order="F")
    assert a1.min() >= 0.0 and a1.max() <= 1.0
    lhs = float(np.sum(a1 * V)) - vol0
    rhs = -cfg["dt"] * float(np.sum(mdot * V)) / cfg["rho_l"] - (d1["clip_mass"] - d0["clip_mass"])
    assert abs(lhs - rhs) <= 1e-12 * vol0
    # projection: discrete divergence of u^{n+1} against S V (relative to the largest face flux)
    u = [sim.get("u%d" % a).reshape(O.fshape(G, a), order="F") for a in range(3)]
    S = sim.get("S").reshape(G.n, order="F")
    div = O.divergence_sum(G, [u[a] * G.A[a] for a in range(3)])
    scale = max(float(np.abs(u[a] * G.A[a]).max()) for a in range(3))
    assert float(np.abs(div - S * V).max()) <= 1e-6 * scale
    sim.close()


def test_graph_step_equals_direct_step(D):
    """The captured step (solver loops as conditional graph nodes) and the directly
    launched step run the same kernels on the same data: identical trajectories."""
    cfg = W.cfg5_axisym_128x256(**SMALL, cg_rtol=1e-12, helm_rtol=1e-12)
    a, b = D.Droplet(cfg), D.Droplet(cfg)
    D.droplet_profile(b.h, 1)          # profiling forces direct launches
    for _ in range(5):
        assert a.step(1) == 0
        assert b.step(1) == 0
    for nm in ("alpha", "T", "omega", "p", "u0", "u1"):
        assert np.array_equal(a.get(nm), b.get(nm)), nm
    da, db = a.diag(), b.diag()
    assert da["its_p"] == db["its_p"] and da["its_u"] == db["its_u"] and da["step"] == db["step"] == 5
    a.close()
    b.close()


def test_checkpoint_resume_is_bit_identical(D, tmp_path):
    cfg = W.cfg5_axisym_128x256(**SMALL, cg_rtol=1e-12, helm_rtol=1e-12)
    a = D.Droplet(cfg)
    a.step(4)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(3)
    b = D.Droplet(cfg)
    b.load(path)
    assert b.diag()["step"] == 4
    b.step(3)
    for nm in ("alpha", "T", "omega", "p", "rhoG", "u0", "u1"):
        assert np.array_equal(a.get(nm), b.get(nm)), nm
    da, db = a.diag(), b.diag()
    assert da["step"] == db["step"] == 7 and da["clip_mass"] == db["clip_mass"]
    other = D.Droplet(dict(cfg, T_amb=700.0))
    with pytest.raises(D.DropletError) as e:
        other.load(path)
    assert e.value.status == -1
    with pytest.raises(D.DropletError) as e:
        other.load(str(tmp_path / "missing.bin"))
    assert e.value.status == -7
    for s in (a, b, other):
        s.close()
