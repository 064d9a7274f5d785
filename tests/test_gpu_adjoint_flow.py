"""Hand-written adjoint of the step WITH flow (evaporation flux with its convective part,
FCT advection, energy and species with convection, momentum predictor with buoyancy and
the centripetal force, Stefan source, pressure projection), checked in three layers:

1. the stage formulas the adjoint differentiates reproduce the forward kernels' values
   (droplet_adjoint_check), so that it differentiates the step that runs;
2. one step: the derivative of the step's evaporation rate with respect to each state
   field in turn, against central differences;
3. whole runs: dJ/dT_amb, dJ/dD_g and directional dJ/dT0 of J = mean evaporation rate
   against central finite differences of the GPU forward (h = 1e-4 relative, see H_FD)
   and of the oracle (h = 1e-6, direct solves), and config 5 as specified (gravity,
   flow, 500 steps, checkpoints every 50).
"""
import numpy as np
import pytest

from oracle import step as O
from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAR = dict(cg_rtol=1e-16, helm_rtol=1e-16, cg_maxit=300, helm_maxit=600)


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


def small(**over):
    """Config 5's physics (gravity, centripetal force, natural convection, 773 K, 1 bar)
    on a 32 x 64 grid of the 2 x 4 mm domain."""
    base = dict(n=(32, 64, 1), L=(2e-3, 4e-3, 0.0), xc=(0.0, 2e-3, 0.0), **PAR)
    base.update(over)
    return W.cfg5_axisym_128x256(**base)


def small3d(**over):
    base = dict(geom=1, n=(12, 12, 14), L=(1.2e-3, 1.2e-3, 1.4e-3), xc=(0.6e-3, 0.6e-3, 0.7e-3), D0=0.6e-3,
                g=(0.0, 0.0, -9.81), **PAR)
    base.update(over)
    return W.make(**base)


def fields(sim):
    names = ["alpha", "T", "omega", "p"] + ["u%d" % a for a in range(3) if _has(sim, "u%d" % a)]
    return names


def _has(sim, name):
    try:
        sim.get(name)
        return True
    except Exception:
        return False


def pack(sim):
    return np.concatenate([sim.get(nm) for nm in fields(sim)])


def unpack(sim, v):
    out, o = {}, 0
    for nm in fields(sim):
        n = sim.get(nm).size
        out[nm] = v[o:o + n]
        o += n
    return out


def step_from(sim, v):
    for nm, x in unpack(sim, v).items():
        sim.set(nm, x)
    assert sim.step(1) in (0, -3)        # (-3: a parity-tolerance solve stopped at its cap)
    return pack(sim), sim.diag()["mdot_tot"]


@pytest.mark.parametrize("make", [small, small3d], ids=["axisym", "cart3d"])
def test_adjoint_formulas_match_the_forward_kernels(D, make):
    sim = D.Droplet(make())
    for _ in range(4):
        sim.step(1)
    rel = D.droplet_adjoint_check(sim.h)
    sim.close()
    bad = {k: v for k, v in rel.items() if not v <= 1e-12}
    assert not bad, rel


def _state_after(D, make, steps=4):
    sim = D.Droplet(make())
    for _ in range(steps):
        sim.step(1)
    return sim, pack(sim)


@pytest.mark.parametrize("make", [small, small3d], ids=["axisym", "cart3d"])
def test_one_step_rate_vjp_against_central_differences(D, make):
    """The step's evaporation rate as a function of the state before it (S0 - S2: the
    pinned saturation values, the gas density, the flux at the adjacent cells with its
    convective part, the K normalisation, the cap), one state field at a time: alpha in
    the interface band, T, omega in the gas and the interior face velocities."""
    sim, s0 = _state_after(D, make)
    parts = unpack(sim, s0)
    lam_prev, _ = D.droplet_adjoint_vjp(sim.h, np.zeros_like(s0), 1.0)
    rng = np.random.default_rng(3)
    a = parts["alpha"]
    errs = {}
    for nm in fields(sim):
        if nm == "p":
            continue                            # the rate does not depend on p_rgh
        d = {k: np.zeros_like(v) for k, v in parts.items()}
        x = parts[nm]
        if nm == "alpha":
            band = (a > 1e-3) & (a < 1 - 1e-3)
            d[nm][band] = rng.uniform(-1, 1, band.sum()) * np.minimum(a[band], 1 - a[band])
        elif nm == "omega":
            d[nm][:] = rng.uniform(-1, 1, x.size) * x * (a < 0.5)
        elif nm.startswith("u"):
            d[nm][:] = rng.uniform(-1, 1, x.size) * np.abs(x)
        else:
            d[nm][:] = rng.uniform(-1, 1, x.size) * x
        dv = np.concatenate([d[k] for k in fields(sim)])
        eps = 1e-6
        _, mp = step_from(sim, s0 + eps * dv)
        _, mm = step_from(sim, s0 - eps * dv)
        fd = (mp - mm) / (2 * eps)
        ad = lam_prev @ dv
        errs[nm] = (ad, fd, abs(ad - fd) / max(abs(fd), 1e-300))
    sim.close()
    bad = {k: v for k, v in errs.items() if not v[2] <= 1e-6}
    assert not bad, errs


@pytest.mark.parametrize("make", [small, small3d], ids=["axisym", "cart3d"])
def test_one_step_dot_product(D, make):
    """The dot-product test of one whole step s' = F(s) with flow: for a random cotangent
    lam on every output field (alpha, T, omega, p_rgh, the face velocities; scaled by each
    field's size) and a direction ds in the state, <(dF/ds)^T lam, ds> from the adjoint
    equals <lam, (F(s + e ds) - F(s - e ds)) / 2e>.  The directions keep the flat parts of
    the state flat (alpha (1 - alpha) in the interface band, T - T_amb, omega in the gas,
    the velocities themselves), where the minmod- and upwind-limited stencils have one-sided
    derivatives."""
    sim, s0 = _state_after(D, make)
    parts = unpack(sim, s0)
    cfg = make()
    rng = np.random.default_rng(11)
    lam = {nm: rng.standard_normal(x.size) / max(np.abs(x).max(), 1e-30) for nm, x in parts.items()}
    lam_v = np.concatenate([lam[nm] for nm in fields(sim)])
    lam_prev, _ = D.droplet_adjoint_vjp(sim.h, lam_v, 0.0)
    a = parts["alpha"]
    d = {"alpha": a * (1.0 - a), "T": parts["T"] - cfg["T_amb"], "omega": parts["omega"] * (a < 0.5),
         "p": parts["p"]}
    for nm in fields(sim):
        if nm.startswith("u"):
            d[nm] = parts[nm]
    dv = np.concatenate([d[k] for k in fields(sim)])
    eps = 1e-6
    sp, _ = step_from(sim, s0 + eps * dv)
    sm, _ = step_from(sim, s0 - eps * dv)
    fd = lam_v @ ((sp - sm) / (2 * eps))
    ad = lam_prev @ dv
    sim.close()
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


def J_gpu(D, cfg, steps, dT0=None):
    sim = D.Droplet(cfg)
    if dT0 is not None:
        sim.set("T", sim.get("T") + dT0)
    J = D.droplet_adjoint(sim.h, steps, 10, gradients=False)
    sim.close()
    return J


# Central differences of J need h ~ 1e-4 relative with flow: the forward solves reach the
# pressure system's attainable accuracy (condition number ~1e7 times the rounding unit), so
# a difference of J over h carries noise ~1e-11 / h, while the truncation error falls as
# h^2.  Measured on the 32 x 64 case (30 steps), central difference against the adjoint:
# h = 1e-7: 1.2e-4, 1e-6: 1.1e-5, 1e-5: 7e-7, 1e-4: 1.4e-7 (T_amb); 5e-6, 8e-6, 3e-7,
# 4e-8 (D_g).
H_FD = 1e-4


def _smooth_directions(T0, T_amb, T_drop, alpha, gT0):
    """Perturbations of the initial temperature that keep its flat regions flat (the
    ambient gas, the uniform liquid): minmod-limited convection is not differentiable
    where neighbouring values are equal, so a direction that makes them unequal has a
    direction-dependent one-sided derivative.  The profile itself and its square, and
    single cells next to the interface whose face neighbours all differ from them."""
    w = (T0 - T_amb) / (T_drop - T_amb)
    dirs = [T0 - T_amb, (T_drop - T_amb) * w * w]
    return dirs


def test_flow_adjoint_scalars_and_directions_against_central_fd(D):
    cfg = small()
    steps = 30
    sim = D.Droplet(cfg)
    T0 = sim.get("T")
    alpha = sim.get("alpha")
    J, gTa, gDg, gT0 = D.droplet_adjoint(sim.h, steps, 10)
    sim.close()
    assert J > 0
    for key, g in (("T_amb", gTa), ("D_g", gDg)):
        h = H_FD * cfg[key]
        fd = (J_gpu(D, dict(cfg, **{key: cfg[key] + h}), steps) - J_gpu(D, dict(cfg, **{key: cfg[key] - h}), steps)) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-5), (key, g, fd)
    n0, n1 = cfg["n"][0], cfg["n"][1]
    Tg = T0.reshape((n0, n1), order="F")
    dirs = _smooth_directions(T0, cfg["T_amb"], cfg["T_drop"], alpha, gT0)
    # single gas cells next to the interface, every face neighbour at a different temperature
    cand = np.flatnonzero((alpha < 1e-3) & (np.abs(gT0) > 1e-3 * np.abs(gT0).max()))
    picked = 0
    for c in cand:
        i, j = c % n0, c // n0
        nb = [Tg[q] for q in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)) if 0 <= q[0] < n0 and 0 <= q[1] < n1]
        if all(abs(v - Tg[i, j]) > 1e-6 * Tg[i, j] for v in nb):
            v = np.zeros_like(T0)
            v[c] = T0[c]
            dirs.append(v)
            picked += 1
        if picked == 3:
            break
    assert picked == 3
    for v in dirs:
        fd = (J_gpu(D, cfg, steps, H_FD * v) - J_gpu(D, cfg, steps, -H_FD * v)) / (2 * H_FD)
        ad = float(gT0 @ v)
        assert ad == pytest.approx(fd, rel=1e-4, abs=1e-6 * abs(J)), (ad, fd)


def J_oracle(cfg, steps):
    st = O.init_state(cfg)
    acc = 0.0
    for _ in range(steps):
        st = O.step(cfg, st)
        acc += O.diagnostics(cfg, st)["mdot_tot"]
    return acc / steps


def test_flow_adjoint_against_oracle_fd(D):
    """The oracle's central-difference gradient (plain FP64, direct solves) with flow."""
    cfg = small(n=(24, 48, 1), L=(1.5e-3, 3e-3, 0.0), xc=(0.0, 1.5e-3, 0.0), D0=0.8e-3)
    steps = 12
    sim = D.Droplet(cfg)
    J, gTa, gDg, _ = D.droplet_adjoint(sim.h, steps, 5)
    sim.close()
    assert J == pytest.approx(J_oracle(cfg, steps), rel=1e-9)
    for key, g in (("T_amb", gTa), ("D_g", gDg)):
        h = 1e-6 * cfg[key]
        fd = (J_oracle(dict(cfg, **{key: cfg[key] + h}), steps) -
              J_oracle(dict(cfg, **{key: cfg[key] - h}), steps)) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-4), (key, g, fd)


def test_config5_flow_adjoint_500_steps(D):
    """Config 5 as specified: 128 x 256 over 4 x 8 mm, D0 = 1 mm, 773 K, 1 bar, gravity and
    the centripetal force, natural convection, FP64, 500 steps of 1e-5 s with checkpoints
    every 50: the scalar gradients against central differences.  Over 500 steps the
    discrete decisions at the interface (the adjacent gas cell along the normal) start to
    flip within +-h from h ~ 1e-4 (measured D_g: 1.4e-4 at h = 1e-4, 1e-2 at 3e-4), while
    the solver noise floor stays near 1e-11 / h, so h = 1e-5 (measured 1.9e-5 for D_g,
    4.2e-6 for T_amb; at 250 steps 1.7e-7 and 1.6e-6)."""
    cfg = W.cfg5_axisym_128x256(cg_rtol=1e-14, helm_rtol=1e-15, cg_maxit=400, helm_maxit=2000)
    sim = D.Droplet(cfg)
    J, gTa, gDg, gT0 = D.droplet_adjoint(sim.h, 500, 50)
    sim.close()
    assert J > 0 and np.all(np.isfinite(gT0))
    for key, g in (("T_amb", gTa), ("D_g", gDg)):
        h = 1e-5 * cfg[key]
        Jp = J_gpu(D, dict(cfg, **{key: cfg[key] + h}), 500)
        Jm = J_gpu(D, dict(cfg, **{key: cfg[key] - h}), 500)
        fd = (Jp - Jm) / (2 * h)
        print("config 5 with flow:", key, g, fd, abs(g - fd) / abs(fd))
        assert g == pytest.approx(fd, rel=1e-4), (key, g, fd)


def test_autograd_function_with_flow(D):
    import torch
    F = D.evaporation_rate_function()
    cfg = small()
    Ta = torch.tensor(cfg["T_amb"], dtype=torch.float64, requires_grad=True)
    Dg = torch.tensor(cfg["D_g"], dtype=torch.float64, requires_grad=True)
    dT0 = torch.zeros(32 * 64, dtype=torch.float64, requires_grad=True)
    J = F.apply(Ta, Dg, dT0, cfg, 10, 5)
    J.backward()
    sim = D.Droplet(cfg)
    J2, gTa, gDg, gT0 = D.droplet_adjoint(sim.h, 10, 5)
    sim.close()
    assert float(J.detach()) == pytest.approx(J2, rel=1e-14)
    # (the reverse sweep adds into the adjoints with atomics, so two runs agree to the
    # rounding of their summation orders)
    assert float(Ta.grad) == pytest.approx(gTa, rel=1e-10)
    assert float(Dg.grad) == pytest.approx(gDg, rel=1e-10)
    assert np.allclose(dT0.grad.numpy(), gT0, rtol=1e-9, atol=1e-9 * np.abs(gT0).max())


def test_flow_adjoint_rejects_unsupported_forms(D):
    for over in (dict(adv_scheme=1), dict(precision=1), dict(co_max=0.2), dict(cp_v=2400.0)):
        sim = D.Droplet(small(**over))
        with pytest.raises(D.DropletError):
            D.droplet_adjoint(sim.h, 5, 5)
        sim.close()
