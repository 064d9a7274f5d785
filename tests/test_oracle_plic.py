"""Pins of the plane geometry of the geometric advection (oracle/plic.py) against
constructions that share nothing with its inclusion-exclusion formulas:

- 2D: the area of the unit square clipped by the half-plane, by polygon clipping
  (Sutherland-Hodgman) and the shoelace formula;
- 3D: the volume as the integral over the third coordinate of the clipped area of
  each slice (the same polygon clipping): the slice area is piecewise quadratic
  between the heights where the slice line passes a square corner, so two-point
  Gauss-Legendre on each piece is exact;
- the inverse: the fraction of the plane constant it returns is the one asked for.
Random planes of every orientation, grid-aligned and nearly aligned ones included.
"""
import numpy as np
import pytest

from oracle import plic


def clip_area(n1, n2, c):
    """Area of {x in [0,1]^2 : n1 x + n2 y <= c} by polygon clipping."""
    poly = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    f = [n1 * x + n2 * y - c for x, y in poly]
    out = []
    for k in range(4):
        p, q = poly[k], poly[(k + 1) % 4]
        fp, fq = f[k], f[(k + 1) % 4]
        if fp <= 0.0:
            out.append(p)
        if (fp < 0.0 < fq) or (fq < 0.0 < fp):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    if len(out) < 3:
        return 0.0
    s = 0.0
    for k in range(len(out)):
        x0, y0 = out[k]
        x1, y1 = out[(k + 1) % len(out)]
        s += x0 * y1 - x1 * y0
    return abs(0.5 * s)


def clip_volume(n, beta):
    """Volume of {x in [0,1]^3 : n . x <= beta}: slice areas integrated over x3."""
    n1, n2, n3 = n
    cuts = [0.0, 1.0]
    if n3 != 0.0:
        for corner in (0.0, n1, n2, n1 + n2):
            z = (beta - corner) / n3
            if 0.0 < z < 1.0:
                cuts.append(z)
    cuts = sorted(cuts)
    g = 0.5 / np.sqrt(3.0)
    v = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        mid, half = 0.5 * (a + b), 0.5 * (b - a)
        for z in (mid - 2 * g * half, mid + 2 * g * half):
            v += half * clip_area(n1, n2, beta - n3 * z)
    return v


def random_planes(d, k, seed):
    rng = np.random.default_rng(seed)
    n = rng.standard_normal((k, d))
    # grid-aligned and nearly aligned normals
    n[: k // 8, 1:] = 0.0
    n[k // 8: k // 4, 0] *= 1e-9
    if d == 3:
        n[k // 4: 3 * k // 8, 1] = 0.0
    beta = rng.uniform(-0.2, 1.2, k) * np.sum(np.abs(n), axis=1) + np.sum(np.minimum(n, 0.0), axis=1)
    return n, beta


def test_cut_fraction_2d_against_polygon_clipping():
    n, beta = random_planes(2, 4000, 1)
    got = plic.cut_fraction(n, beta)
    ref = np.array([clip_area(a, b, c) for (a, b), c in zip(n, beta)])
    assert np.abs(got - ref).max() < 1e-13


def test_cut_fraction_3d_against_slice_integration():
    n, beta = random_planes(3, 3000, 2)
    got = plic.cut_fraction(n, beta)
    ref = np.array([clip_volume(tuple(v), c) for v, c in zip(n, beta)])
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_plane_constant_inverts_the_fraction(d):
    rng = np.random.default_rng(3 + d)
    n, _ = random_planes(d, 5000, 4 + d)
    f = rng.uniform(1e-9, 1 - 1e-9, n.shape[0])
    f[:50] = 0.5
    beta = plic.plane_constant(n, f)
    assert np.abs(plic.cut_fraction(n, beta) - f).max() < 2e-13


def test_cut_fraction_monotone_and_bounds():
    n, _ = random_planes(3, 200, 9)
    s = np.sum(np.abs(n), axis=1)
    lo = np.sum(np.minimum(n, 0.0), axis=1)
    prev = np.zeros(n.shape[0])
    for t in np.linspace(-0.1, 1.1, 61):
        v = plic.cut_fraction(n, lo + t * s)
        assert np.all(v >= prev - 1e-15) and np.all((v >= 0.0) & (v <= 1.0))
        prev = v
    assert np.all(prev == 1.0)
