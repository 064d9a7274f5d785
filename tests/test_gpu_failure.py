"""Failure detection on the GPU without faulting it.

- A bounded device wait that runs out: the persistent (cooperative) solvers wait at
  grid barriers; wait_limit = 1 makes the first wait of a block that is not the last
  to arrive give up after two polls, so the solve stops, the step reports
  DROPLET_ERR_TIMEOUT, every block leaves the launch (no hang) and a fresh context on
  the same device steps normally.
- A non-finite value put into the state from the host (droplet_set_field): the
  diagnostics at the end of the next step see it and droplet_diag returns
  DROPLET_ERR_NONFINITE.
- A solve capped at one iteration reports DROPLET_ERR_NOT_CONVERGED and the state
  still advances (test_gpu_parity.py).
"""
import numpy as np
import pytest

from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = dict(n=(32, 64, 1), L=(2e-3, 4e-3, 0.0), xc=(0.0, 2e-3, 0.0))
CUBE = dict(geom=1, n=(16, 16, 16), L=(1.6e-3,) * 3, xc=(0.8e-3,) * 3, D0=0.8e-3, g=(0, 0, -9.81))


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


@pytest.mark.parametrize("geo", [SMALL, CUBE], ids=["axisym-32x64", "cart3d-16"])
@pytest.mark.parametrize("precision", [0, 1])
def test_wait_limit_runs_out_as_timeout(D, geo, precision):
    cfg = W.cfg5_axisym_128x256(**geo, precision=precision, wait_limit=1)
    sim = D.Droplet(cfg)
    rc = sim.step(1)
    assert rc == D.ERR_TIMEOUT, rc
    sim.close()
    # the device and a fresh context are unaffected
    ok = D.Droplet(dict(cfg, wait_limit=0))
    assert ok.step(2) == 0
    d = ok.diag()
    assert d["step"] == 2 and np.isfinite(d["V_l"]) and d["its_p"] > 0
    ok.close()


def test_launched_solvers_have_no_wait_to_run_out(D):
    """The launched solvers (solver_select = 1) never wait on other blocks: the same
    wait limit leaves them untouched."""
    cfg = W.cfg5_axisym_128x256(**SMALL, wait_limit=1, solver_select=1)
    sim = D.Droplet(cfg)
    assert sim.step(2) == 0
    sim.close()


@pytest.mark.parametrize("field,value", [("T", np.nan), ("omega", np.inf), ("u1", -np.inf), ("alpha", np.nan)])
def test_nonfinite_state_is_reported(D, field, value):
    cfg = W.cfg5_axisym_128x256(**SMALL, helm_maxit=20, cg_maxit=20)
    sim = D.Droplet(cfg)
    assert sim.step(1) == 0
    x = sim.get(field)
    x[len(x) // 3] = value
    sim.set(field, x)
    sim.step(1)
    with pytest.raises(D.DropletError) as e:
        sim.diag()
    assert e.value.status == D.ERR_NONFINITE
    sim.close()


@pytest.mark.parametrize("solver_select", [0, 1], ids=["persistent", "launched"])
def test_vanishing_vapour_stays_finite_in_binary32_solves(D, solver_select):
    """After a droplet has evaporated, the vapour left in the domain decays towards zero
    and the species system's defect falls far below the binary32 range (|r0| ~ 1e-50
    here).  The binary32 Jacobi-PCG of mixed precision normalises that defect in FP64
    before rounding it (persistent form) or scales it by a power of two (launched form);
    rounded first, it flushed to zero and the normalisation turned it into NaN.  A state
    with no liquid, uniform ambient temperature and a vapour fraction of ~1e-40 must step
    with every field finite, on both solver forms."""
    cfg = W.cfg5_axisym_128x256(**SMALL, precision=1, cg_rtol=1e-8, helm_rtol=1e-8, solver_select=solver_select)
    sim = D.Droplet(cfg)
    assert sim.step(1) == 0
    rng = np.random.default_rng(7)
    n = len(sim.get("alpha"))
    sim.set("alpha", np.zeros(n))
    sim.set("T", np.full(n, cfg["T_amb"]))
    sim.set("omega", 1e-40 * (1.0 + 0.5 * rng.random(n)))
    for _ in range(3):
        sim.step(1)
        sim.diag()   # raises DROPLET_ERR_NONFINITE on any non-finite state value
    for f in ("T", "omega", "p", "rhoG", "u0", "u1"):
        assert np.isfinite(sim.get(f)).all(), f
    w = sim.get("omega")
    assert w.max() < 1e-39 and w.min() >= 0.0
    sim.close()
