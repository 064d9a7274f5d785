"""droplet_box_solve_noalloc: the box solve for callers that cannot allocate
device memory (their memory comes from a pool they own, or they must not call
cudaMalloc / cudaFree while other work runs).  Its work vectors live in a
static device array of the library.  Checked against droplet_box_solve, the
allocating entry point, on two calls in a row (the second on a different
system, so that nothing left in the shared array from the first call leaks
into the second), and for the rejection of boxes larger than the array."""
import numpy as np
import pytest

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


def _system(m, seed):
    import torch
    rng = np.random.default_rng(seed)
    arrs = [1e-2 * rng.uniform(0.5, 1.5, m)]
    for a in range(3):
        c = 10.0 ** rng.uniform(-2, 2, m) if m[a] > 1 else np.zeros(m)
        sl = [slice(None)] * 3
        sl[a] = 0
        c[tuple(sl)] = 0.0
        arrs.append(c)
    arrs.append(rng.standard_normal(m))
    return [torch.from_numpy(np.ascontiguousarray(x.ravel(order="F"))).cuda() for x in arrs]


def _solve(fn, m, t, rtol=1e-14):
    import torch
    x = torch.zeros_like(t[-1])
    st = torch.cuda.current_stream().cuda_stream
    rc, its, rel = fn(m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr() if m[2] > 1 else 0,
                      t[4].data_ptr(), x.data_ptr(), rtol, 4000, st)
    return rc, its, rel, x.cpu().numpy()


def test_noalloc_matches_allocating_solver_twice(D):
    for call, (m, seed) in enumerate((((48, 40, 1), 11), ((20, 18, 12), 12))):
        t = _system(m, seed)
        rc_a, its_a, rel_a, xa = _solve(D.droplet_box_solve, m, t)
        rc_n, its_n, rel_n, xn = _solve(D.droplet_box_solve_noalloc, m, t)
        assert rc_a == 0 and rc_n == 0, (call, rc_a, rc_n)
        assert rel_n <= 1e-14
        assert np.abs(xn - xa).max() <= 1e-10 * np.abs(xa).max(), call


def test_noalloc_leaves_device_memory_unchanged(D):
    """After a first call (which, under lazy module loading, places the static
    array on the device), further calls change the device's free memory by
    nothing."""
    import torch
    m = (40, 36, 1)
    t = _system(m, 13)
    x = torch.zeros_like(t[-1])
    st = torch.cuda.current_stream().cuda_stream
    args = (m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), 0, t[4].data_ptr(), x.data_ptr(), 1e-12, 4000, st)
    assert D.droplet_box_solve_noalloc(*args)[0] == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        x.zero_()
        assert D.droplet_box_solve_noalloc(*args)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversize_box(D):
    import torch
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = small.data_ptr()
    st = torch.cuda.current_stream().cuda_stream
    big = D.NOALLOC_MAX_UNKNOWNS + 1
    # too many unknowns; and dimensions whose product would wrap a 64-bit integer
    for m in ((big, 1, 1), (2, big, 1), (2**31 - 1, 2**31 - 1, 2**31 - 1)):
        rc, _, _ = D.droplet_box_solve_noalloc(m, p, p, p, p, p, p, 1e-10, 10, st)
        assert rc == -5, m


def test_noalloc_refuses_a_capturing_stream(D):
    """The call synchronises its stream, so inside a stream capture it must
    refuse (DROPLET_ERR_ARG) before it enqueues anything; the (empty) capture
    then ends cleanly and a plain call afterwards still solves."""
    import torch
    m = (16, 12, 1)
    t = _system(m, 14)
    x = torch.zeros_like(t[-1])
    s = torch.cuda.Stream()
    args = (m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), 0, t[4].data_ptr(), x.data_ptr(), 1e-12, 4000)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = D.droplet_box_solve_noalloc(*args, s.cuda_stream)[0]
    assert rc == -1
    torch.cuda.synchronize()
    assert D.droplet_box_solve_noalloc(*args, torch.cuda.current_stream().cuda_stream)[0] == 0
