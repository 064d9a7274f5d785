"""Hand-written adjoint of the step without flow against central finite
differences (h = 1e-6 relative) of the GPU forward and of the oracle.

J = mean evaporation rate over the run; parameters: ambient temperature (it
enters through the initial temperature profile), gas diffusivity, and the
initial temperature field (directional derivatives)."""
import numpy as np
import pytest

from oracle import step as O
from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NOFLOW = W.PHYS_EVAP | W.PHYS_ENERGY | W.PHYS_SPECIES


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
    base = dict(n=(32, 64, 1), L=(2e-3, 4e-3, 0.0), xc=(0.0, 2e-3, 0.0), physics_mask=NOFLOW,
                helm_rtol=1e-15, helm_maxit=2000)
    base.update(over)
    return W.cfg5_axisym_128x256(**base)


def J_gpu(D, cfg, steps, dT0=None):
    sim = D.Droplet(cfg)
    if dT0 is not None:
        sim.set("T", sim.get("T") + dT0)
    J = D.droplet_adjoint(sim.h, steps, 10, gradients=False)
    sim.close()
    return J


def test_adjoint_scalars_against_central_fd(D):
    cfg = small()
    steps = 30
    sim = D.Droplet(cfg)
    J, gTa, gDg, gT0 = D.droplet_adjoint(sim.h, steps, 10)
    sim.close()
    assert J > 0
    for key, g in (("T_amb", gTa), ("D_g", gDg)):
        h = 1e-6 * cfg[key]
        Jp = J_gpu(D, dict(cfg, **{key: cfg[key] + h}), steps)
        Jm = J_gpu(D, dict(cfg, **{key: cfg[key] - h}), steps)
        fd = (Jp - Jm) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-5), (key, g, fd)


def test_adjoint_directional_initial_temperature(D):
    cfg = small()
    steps = 20
    sim = D.Droplet(cfg)
    T0 = sim.get("T")
    alpha = sim.get("alpha")
    J, _, _, gT0 = D.droplet_adjoint(sim.h, steps, 7)
    sim.close()
    rng = np.random.default_rng(5)
    dirs = [rng.choice([-1.0, 1.0], size=T0.size) * T0 for _ in range(4)]
    # single cells in the gas next to the interface
    near = np.flatnonzero((alpha < 1e-3) & (np.abs(gT0) > 1e-3 * np.abs(gT0).max()))[:4]
    for c in near:
        v = np.zeros_like(T0)
        v[c] = T0[c]
        dirs.append(v)
    for v in dirs:
        eps = 1e-6
        fd = (J_gpu(D, cfg, steps, eps * v) - J_gpu(D, cfg, steps, -eps * v)) / (2 * eps)
        ad = float(gT0 @ v)
        assert ad == pytest.approx(fd, rel=1e-4, abs=1e-8 * abs(J)), (ad, fd)


def J_oracle(cfg, steps):
    st = O.init_state(cfg)
    G = None
    acc = 0.0
    for _ in range(steps):
        st = O.step(cfg, st)
        acc += O.diagnostics(cfg, st)["mdot_tot"]
    return acc / steps


def test_adjoint_against_oracle_fd(D):
    """The oracle's central-difference gradient (plain FP64, direct solves)."""
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


def test_autograd_function(D):
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
    assert float(Ta.grad) == pytest.approx(gTa, rel=1e-12)
    assert float(Dg.grad) == pytest.approx(gDg, rel=1e-12)
    assert np.allclose(dT0.grad.numpy(), gT0, rtol=1e-12, atol=0)


def test_config5_adjoint_500_steps(D):
    """Config 5 grid (128 x 256, 4 x 8 mm, D0 = 1 mm, 773 K, 1 bar), 500 FP64 steps
    with checkpoints every 50, without flow: scalar gradients against central
    differences with h = 1e-6 relative."""
    cfg = W.cfg5_axisym_128x256(physics_mask=NOFLOW, helm_rtol=1e-14, helm_maxit=2000)
    sim = D.Droplet(cfg)
    J, gTa, gDg, gT0 = D.droplet_adjoint(sim.h, 500, 50)
    sim.close()
    assert J > 0 and np.isfinite(gT0).all()
    for key, g in (("T_amb", gTa), ("D_g", gDg)):
        h = 1e-6 * cfg[key]
        fd = (J_gpu(D, dict(cfg, **{key: cfg[key] + h}), 500) - J_gpu(D, dict(cfg, **{key: cfg[key] - h}), 500)) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-5), (key, g, fd)
