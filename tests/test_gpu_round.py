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


def test_reciprocal_within_one_ulp(D):
    """The binary64 reciprocal that stands in for divisions in the step kernels (a
    binary32 seed and two Newton-Raphson steps) against the correctly rounded 1 / x:
    at most one ulp apart over binary32's normal range, identical (a division) outside
    it, including zeros, infinities and NaN."""
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.standard_normal(300000) * 10.0 ** rng.uniform(-37, 37, 300000),
        rng.uniform(0.01, 2000.0, 100000),                          # densities, temperatures
        np.nextafter(2.0 ** rng.integers(-120, 120, 2000).astype(np.float64), np.inf),
        2.0 ** rng.integers(-120, 120, 2000).astype(np.float64),    # exact powers of two
    ])
    y = D.droplet_rcp_f64(x)
    ref = 1.0 / x
    ulps = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0, (ulps.max(), x[np.argmax(ulps)])
    assert np.array_equal(y[-2000:], ref[-2000:])                 # powers of two: exact
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, -1e-300, 1e300, 1e-39, 3e38, 1e39])
    ye = D.droplet_rcp_f64(edge)
    with np.errstate(divide="ignore"):
        re = 1.0 / edge
    assert np.array_equal(ye, re, equal_nan=True)
