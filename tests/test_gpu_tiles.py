"""The temporal blocking of the persistent multigrid smoothing recomputes tile halos
instead of exchanging them; every owned cell must get exactly the value of the
level-wide red-black sweep, whatever the tile.  So the whole step (and the
trajectory) is bit-identical across tile shapes, including tiles that do not divide
the grid and tiles larger than the coarse levels."""
import numpy as np
import pytest

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


FIELDS = ("alpha", "T", "omega", "p", "rhoG", "u0", "u1")


def run(D, tile, precision):
    cfg = W.cfg5_axisym_128x256(precision=precision, mg_tile=tile, cg_rtol=1e-10, helm_rtol=1e-10)
    sim = D.Droplet(cfg)
    assert sim.step(4) == 0
    out = {nm: sim.get(nm) for nm in FIELDS}
    out["its_p"] = sim.diag()["its_p"]
    sim.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_shape_does_not_change_the_result(D, precision):
    ref = run(D, (32, 32), precision)
    for tile in ((64, 64), (128, 32), (24, 40), (8, 8)):
        got = run(D, tile, precision)
        assert got["its_p"] == ref["its_p"], tile
        for nm in FIELDS:
            assert np.array_equal(got[nm], ref[nm]), (tile, nm)
