"""The persistent Jacobi-PCG on a box larger than L2, where each CG iteration runs in
two passes (update, then w = A r) instead of the fused single pass of the smaller
boxes.  The oracle cannot solve 2^21 unknowns in seconds, but it can assemble the
system: one energy-only step on a 128^3 grid must leave a T^{n+1} that satisfies the
oracle's backward-Euler energy system (Eq. Teqn, Sec. 3.1) to the solve tolerance."""
import numpy as np
import pytest

from oracle import step as O
from oracle.grid import Grid
from paper_2005_02867_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _oracle_energy_system(cfg, G, alpha, T, omega):
    """diag, couplings and right-hand side of the energy system of one step from the
    given state (energy alone: no evaporation, no flow), as the oracle assembles them."""
    omega_p, rhoG_old = O.thermo_pin(cfg, G, alpha, T, omega)
    pr = O.props(cfg, alpha, rhoG_old, omega_p, T)
    u = [np.zeros(O.fshape(G, a)) for a in range(3)]
    captured = {}
    solve = O.solve_box

    def capture(shape, diag, coup, rhs):
        captured.update(shape=shape, diag=diag, coup=coup, rhs=rhs)
        return np.zeros(shape)
    O.solve_box = capture
    try:
        O.scalar_transport(cfg, G, T, pr["rho"] * pr["cp"], pr["k"], np.zeros(G.n), u, cfg["dt"], cfg["T_amb"])
    finally:
        O.solve_box = solve
    return captured


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-5)])
def test_two_pass_solve_satisfies_the_oracle_system(D, precision, rtol, tol):
    """128^3 = 2^21 cells, seeded 1 % temperature perturbation, a time step long enough
    (Fourier number ~10 in the gas) that the solve takes tens of iterations, starting
    from a defect of the order of the right-hand side.  FP64: the residual of the
    oracle's FP64 system at the solve tolerance.  Mixed: FP32 iterations on the
    defect (their attainable reduction is ~1e-6) and an FP32 assembly that rounds b
    and the couplings, hence the looser bound."""
    cfg = W.cfg3_cart3d(nc=128, precision=precision, eq_model=0, P=1e5, u_inflow=0.0, bc_mode=0,
                        g=(0.0, 0.0, 0.0), physics_mask=W.PHYS_ENERGY, dt=1e-4, helm_rtol=rtol, helm_maxit=500)
    G = Grid(cfg)
    assert int(np.prod(G.n)) == 1 << 21
    sim = D.Droplet(cfg)
    fields = {k: sim.get(k).reshape(G.n, order="F") for k in ("alpha", "T", "omega")}
    assert sim.step(1) == 0
    d = sim.diag()
    T1 = sim.get("T").reshape(G.n, order="F")
    sim.close()
    assert d["its_T"] >= 4                       # the two-pass iteration did run
    sysm = _oracle_energy_system(cfg, G, fields["alpha"], fields["T"], fields["omega"])
    res = sysm["rhs"] - O.box_apply(sysm["shape"], sysm["diag"], sysm["coup"], T1)
    rel = float(np.linalg.norm(res) / np.linalg.norm(sysm["rhs"]))
    assert rel <= tol, rel
    # and the step did change T beyond that tolerance (the check is not vacuous)
    assert float(np.abs(T1 - fields["T"]).max() / np.abs(fields["T"]).max()) > 100 * tol
