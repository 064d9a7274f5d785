"""Batched droplets (config 4 form): one context, one graph launch per step with
one branch per droplet.  Each droplet of a batch must follow the same
trajectory as when it is stepped alone, and match the oracle."""
import numpy as np
import pytest

from oracle import step as O
from oracle.grid import Grid
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


def small_batch(**over):
    """Three uneven droplets: grid, diameter, ambient temperature and pressure differ."""
    out = []
    for nr, d0, tamb, p in ((24, 0.6e-3, 600.0, 2e5), (32, 1.0e-3, 773.0, 1e5), (40, 0.8e-3, 900.0, 5e5)):
        L0 = 4 * d0
        out.append(W.make(n=(nr, 2 * nr, 1), L=(L0, 2 * L0, 0.0), xc=(0.0, L0, 0.0), D0=d0, T_amb=tamb, P=p,
                          g=(0.0, -9.81, 0.0), dt=1e-5 * (L0 / nr) / 62.5e-6, **over))
    return out


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_batch_equals_single_runs(D):
    cfgs = small_batch(cg_rtol=1e-12, helm_rtol=1e-12)
    batch = D.Droplet(cfgs)
    singles = [D.Droplet(c) for c in cfgs]
    for _ in range(5):
        assert batch.step(1) == 0
        for s in singles:
            assert s.step(1) == 0
    for i, s in enumerate(singles):
        for nm in ("alpha", "T", "omega", "p", "u0", "u1"):
            assert rel(batch.get(nm, droplet=i), s.get(nm)) <= 1e-11, (i, nm)
        db, ds = batch.diag(i), s.diag()
        assert db["step"] == ds["step"] == 5
        assert abs(db["V_l"] - ds["V_l"]) <= 1e-12 * ds["V_l"]
        s.close()
    batch.close()


def test_batch_droplet_matches_oracle(D):
    cfgs = small_batch(**PAR)
    batch = D.Droplet(cfgs)
    k = 2
    cfg = cfgs[k]
    G = Grid(cfg)
    st = O.init_state(cfg)
    for _ in range(3):
        batch.step(1)
        st = O.step(cfg, st)
    for nm in ("alpha", "T", "omega", "p"):
        assert rel(batch.get(nm, droplet=k), st[nm].ravel(order="F")) <= 1e-10, nm
    for a in G.act:
        assert rel(batch.get("u%d" % a, droplet=k), st["u"][a].ravel(order="F")) <= 1e-10
    batch.close()


def test_mixed_batch_volume_matches_fp64(D):
    b64 = D.Droplet(small_batch(cg_rtol=1e-10, helm_rtol=1e-10))
    b32 = D.Droplet(small_batch(cg_rtol=1e-8, helm_rtol=1e-8, precision=1))
    for _ in range(10):
        b64.step(1)
        b32.step(1)
    for i in range(3):
        v64, v32 = b64.diag(i)["V_l"], b32.diag(i)["V_l"]
        assert abs(v32 - v64) <= 1e-5 * v64
    with pytest.raises(D.DropletError):
        b64.diag(3)
    b64.close()
    b32.close()


def test_batched_mixed_matches_unbatched_fp64_d2_slope(D):
    """Config 4 as benchmarked: the 64 seed-drawn droplets in one mixed-precision batch
    (one graph launch per step) against the same droplets stepped one by one in plain
    FP64, both at the benchmark's solver tolerances.  Over steps 150-300 each droplet's
    d2 slope agrees within 1e-3 (the benchmark spec's accuracy for reduced precision) and its
    volume within 1e-5: the two forms are compared at matched d2-slope error, so the
    benchmark's ratio of their throughputs is the batching-and-precision speed-up."""
    cfgs = W.cfg4_batch()
    batch = D.Droplet(cfgs)
    singles = [D.Droplet(dict(c, precision=0)) for c in cfgs]
    steps, start = 300, 150
    tb = np.zeros((steps, len(cfgs)))
    db = np.zeros_like(tb)
    ts = np.zeros_like(tb)
    ds = np.zeros_like(tb)
    for n in range(steps):
        assert batch.step(1) == 0
        for i, s in enumerate(singles):
            assert s.step(1) == 0
            d = s.diag()
            ts[n, i], ds[n, i] = d["t"], d["d2"]
        for i in range(len(cfgs)):
            d = batch.diag(i)
            tb[n, i], db[n, i] = d["t"], d["d2"]
    worst = 0.0
    for i in range(len(cfgs)):
        kb = -np.polyfit(tb[start:, i], db[start:, i], 1)[0]
        ks = -np.polyfit(ts[start:, i], ds[start:, i], 1)[0]
        assert ks > 0.0, i
        worst = max(worst, abs(kb - ks) / ks)
        assert abs(db[-1, i] - ds[-1, i]) <= 1.5e-5 * ds[-1, i], i     # d2 ~ V^(2/3): volume within 1e-5
    print("worst relative d2-slope difference over 64 droplets:", worst)
    assert worst <= 1e-3
    batch.close()
    for s in singles:
        s.close()
