"""droplet_box_solve against the oracle's direct solve of the same box system."""
import numpy as np
import pytest

from oracle import step as O

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


def random_box(m, seed, diag_scale=1e-2):
    """SPD box system: positive couplings (c_a[P] at the high cell, zero where P_a = 0)
    spanning four decades, a small positive D."""
    rng = np.random.default_rng(seed)
    Dg = diag_scale * rng.uniform(0.5, 1.5, m)
    cs = []
    for a in range(3):
        if m[a] < 2:
            cs.append(None)
            continue
        c = 10.0 ** rng.uniform(-2, 2, m)
        sl = [slice(None)] * 3
        sl[a] = 0
        c[tuple(sl)] = 0.0
        cs.append(c)
    b = rng.standard_normal(m)
    return Dg, cs, b


def oracle_solve(m, Dg, cs, b):
    coup = {}
    for a in range(3):
        if cs[a] is None:
            continue
        sl = [slice(None)] * 3
        sl[a] = slice(1, m[a])
        coup[a] = cs[a][tuple(sl)]
    return O.solve_box(m, Dg, coup, b)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).cuda()


@pytest.mark.parametrize("m", [(37, 23, 1), (16, 12, 9), (1, 50, 1)])
def test_box_solve_matches_direct_solve(D, m):
    import torch
    Dg, cs, b = random_box(m, seed=sum(m))
    ref = oracle_solve(m, Dg, cs, b)
    t = [to_dev(Dg)] + [to_dev(c) if c is not None else to_dev(np.zeros(m)) for c in cs] + [to_dev(b)]
    x = torch.zeros_like(t[-1])
    st = torch.cuda.current_stream().cuda_stream
    rc, its, rel = D.droplet_box_solve(m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(),
                                       t[3].data_ptr() if m[2] > 1 else 0, t[4].data_ptr(), x.data_ptr(),
                                       1e-15, 5000, st)
    assert rc == 0 and rel <= 1e-15
    got = x.cpu().numpy().reshape(m, order="F")
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_box_solve_cap_and_arguments(D):
    import torch
    m = (20, 20, 1)
    Dg, cs, b = random_box(m, seed=3)
    t = [to_dev(Dg), to_dev(cs[0]), to_dev(cs[1]), to_dev(b)]
    x = torch.zeros_like(t[-1])
    st = torch.cuda.current_stream().cuda_stream
    rc, its, rel = D.droplet_box_solve(m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), 0, t[3].data_ptr(),
                                       x.data_ptr(), 1e-15, 2, st)
    assert rc == D.ERR_NOT_CONVERGED and its == 2
    rc, _, _ = D.droplet_box_solve((20, 20, 4), t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), 0,
                                   t[3].data_ptr(), x.data_ptr(), 1e-15, 10, st)
    assert rc == -1
