"""Mixed precision (precision = 1: FP32 multigrid and Helmholtz solves, FP32 stencil
increments, FP64 state, thermodynamics, CG residuals of the pressure and mass
bookkeeping) against the plain FP64 oracle, at the benchmark's solver tolerances
(cg_rtol = helm_rtol = 1e-8), on the physics of the benchmarked configurations at
sizes the oracle finishes in seconds:

- config 2 (axisymmetric, gravity, centripetal force, 773 K, 1 bar, dt 5e-6 s) on
  64 x 128, 20 steps;
- config 3 (3D, forced inflow 1 m/s, 20 bar, Peng-Robinson, 1 % perturbation,
  dt 2e-6 s) on 24^3 with the cell size of a 96^3 grid, 2 steps;
- config 4 (a batch of uneven droplets): the 64 x 128 droplets of the seed-drawn
  batch stepped together as a batch, each against its own oracle run, 10 steps.

The benchmark spec asks for the droplet volume within 1e-5 relative (the d2 slope within
1e-3 is checked in test_gpu_d2law.py); the fields are held to 1e-3 relative (max-norm
over max-norm; p_rgh is gauge-fixed by the open boundaries).  Each case also runs the
GPU's plain FP64 path at the same solver tolerances: the part of the error that the
tolerance 1e-8 itself causes (the velocities follow the pressure increment, whose
system has a condition number near 1e7) is the FP64 column, and mixed precision must
not add more than ten times that, or 1e-6 where it is smaller.  The measured errors
are printed, and written as JSON to the path in DROPLET_ERROR_TABLE when set.
"""
import json
import os

import numpy as np
import pytest

from oracle import step as O
from oracle.grid import Grid
from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BENCH_TOL = dict(cg_rtol=1e-8, helm_rtol=1e-8)
TABLE = {}


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_02867_gb300 import _build, droplet
    _build.build_library()
    droplet.load_library()
    torch.cuda.set_device(0)
    yield droplet
    path = os.environ.get("DROPLET_ERROR_TABLE")
    if path:
        with open(path, "w") as fh:
            json.dump(TABLE, fh, indent=1)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def errors(sim, cfg, st, droplet=0):
    G = Grid(cfg)
    e = {nm: rel(sim.get(nm, droplet=droplet), st[nm].ravel(order="F")) for nm in ("alpha", "T", "omega", "p", "rhoG")}
    for a in G.act:
        e["u%d" % a] = rel(sim.get("u%d" % a, droplet=droplet), st["u"][a].ravel(order="F"))
    d, od = sim.diag(droplet), O.diagnostics(cfg, st)
    e["V_l"] = abs(d["V_l"] - od["V_l"]) / od["V_l"]
    e["mdot_tot"] = abs(d["mdot_tot"] - od["mdot_tot"]) / max(abs(od["mdot_tot"]), 1e-300)
    return e


def check(name, e, e64, field_tol=1e-3):
    TABLE[name] = {"mixed": e, "fp64_same_tolerance": e64}
    print(name, "mixed", json.dumps({k: float("%.3g" % v) for k, v in e.items()}))
    print(name, "fp64 ", json.dumps({k: float("%.3g" % v) for k, v in e64.items()}))
    assert e["V_l"] <= 1e-5, (name, e)
    bad = {k: v for k, v in e.items() if k not in ("V_l", "mdot_tot") and not v <= field_tol}
    assert not bad, (name, bad)
    added = {k: (v, e64[k]) for k, v in e.items() if not v <= max(10.0 * e64[k], 1e-6)}
    assert not added, (name, added)


def oracle_run(cfg, steps):
    st = O.init_state(cfg)
    for _ in range(steps):
        st = O.step(cfg, st)
    return st


def gpu_errors(D, cfgs, steps, oracle_states):
    """Errors of the GPU run of cfgs (one droplet, or a batch) against the oracle."""
    sim = D.Droplet(cfgs if len(cfgs) > 1 else cfgs[0])
    for _ in range(steps):
        assert sim.step(1) == 0
    out = [errors(sim, c, st, droplet=i) for i, (c, st) in enumerate(zip(cfgs, oracle_states))]
    sim.close()
    return out


def run_case(D, name, cfgs, steps):
    sts = [oracle_run(c, steps) for c in cfgs]
    mixed = gpu_errors(D, cfgs, steps, sts)
    fp64 = gpu_errors(D, [dict(c, precision=0) for c in cfgs], steps, sts)
    for i, c in enumerate(cfgs):
        label = name if len(cfgs) == 1 else (f"{name}, droplet {i} (64x128, D0 {c['D0'] * 1e3:.2f} mm, "
                                             f"{c['T_amb']:.0f} K, {c['P'] / 1e5:.1f} bar)")
        check(label, mixed[i], fp64[i])


def test_config2_physics_mixed_vs_oracle(D):
    run_case(D, "cfg2 physics, 64x128, 20 steps", [W.cfg2_axisym_256x512(n=(64, 128, 1), **BENCH_TOL)], 20)


def test_config3_physics_mixed_vs_oracle(D):
    nc, h = 24, 4e-3 / 96
    L = nc * h
    cfg = W.cfg3_cart3d(nc=nc, L=(L,) * 3, xc=(0.5 * L,) * 3, D0=0.4 * L, **BENCH_TOL)
    run_case(D, "cfg3 physics, 24^3 (h of 96^3), 2 steps", [cfg], 2)


def test_config4_batch_mixed_vs_oracle(D):
    drops = [c for c in W.cfg4_batch() if c["n"][0] == 64][:3]
    assert len(drops) >= 2
    run_case(D, "cfg4 batch, 10 steps", drops, 10)
