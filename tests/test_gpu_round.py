"""The integer-pipe binary64 -> binary32 conversion of the mixed-precision kernels
against IEEE 754 round-to-nearest-even (numpy's float32 cast), bit for bit, and its
widening back to binary64 (exact)."""
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
    return droplet


def cases():
    rng = np.random.default_rng(7)
    f32 = np.finfo(np.float32)
    parts = [
        rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000),   # the normal range, both signs
        rng.uniform(-1e3, 1e3, 100000),
        np.array([0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -126, -(2.0 ** -126), float(f32.max), -float(f32.max),
                  float(f32.tiny), 3.4028235677973366e38, 3.4028236e38, 1e39, -1e39, 1e-39, 1e-45, 1e-50,
                  np.inf, -np.inf, 1e300, -1e-300]),
    ]
    # exact ties: a float32 value plus half an ulp (round to even both ways), and neighbours
    base = rng.uniform(1.0, 2.0, 50000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(base.astype(np.float32)).astype(np.float64)
    parts += [base + 0.5 * ulp, base - 0.5 * ulp, base + 0.5 * ulp * (1 + 2 ** -20), base + 0.5 * ulp * (1 - 2 ** -20)]
    # values whose rounding carries into the exponent
    parts.append(np.nextafter(np.float64(2.0), 0.0) * 2.0 ** rng.integers(-100, 100, 1000))
    return np.concatenate(parts)


def test_round_to_nearest_even_bitwise(D):
    x = cases()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    out, back = D.droplet_round_f32(x)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
    # the widening back is exact (NaN-free inputs here)
    assert np.array_equal(back, ref.astype(np.float64))


def test_nan_stays_nan(D):
    out, back = D.droplet_round_f32(np.array([np.nan, -np.nan]))
    assert np.isnan(out).all() and np.isnan(back).all()
