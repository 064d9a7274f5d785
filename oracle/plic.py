"""Plane (PLIC) geometry of the geometric interface advection (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper advects the liquid fraction geometrically (Sec. 2.1, Eq. advection, the
isoAdvector scheme): the interface inside a cell is a plane, and the volume of
liquid a face passes in a time step is the volume the plane cuts from the region
the face sweeps.  On a uniform grid both reduce to one function: the fraction of a
box [0, 1]^d on the liquid side {n . xi <= beta} of a plane, and its inverse (the
plane constant that cuts a given fraction).  The fraction is the volume of a
clipped cube, written by inclusion-exclusion over the box corners; the forms below
are arranged so that no term is divided by a vanishing normal component without a
bounded ratio in front of it (grid-aligned interfaces are the common case).

Conventions: normals are in box-scaled coordinates (the component along axis a is
multiplied by the cell size h_a), of any scale; arrays are vectorised over cells.
"""
import numpy as np


def _prep(n, beta):
    """Reflect every axis with a negative normal component (xi_a -> 1 - xi_a), scale
    so that the components sum to one, and return (m sorted ascending [k, d], the
    plane constant a of the reflected, scaled plane [k], zero-normal mask)."""
    n = np.asarray(n, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64) - np.sum(np.minimum(n, 0.0), axis=1)
    m = np.abs(n)
    s = np.sum(m, axis=1)
    zero = s == 0.0
    ss = np.where(zero, 1.0, s)
    return np.sort(m / ss[:, None], axis=1), beta / ss, zero


def _frac2(m1, m2, a):
    """Fraction of the unit square below m1 x + m2 y = a, m1 <= m2, m1 + m2 = 1,
    0 <= a <= 1/2 (a quarter-plane triangle while a <= m1, a trapezoid beyond)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        tri = np.where(m1 > 0.0, (a / m1) * a / (2.0 * m2), 0.0)
    return np.where(a <= m1, tri, (2.0 * a - m1) / (2.0 * m2))


def _frac3(m1, m2, m3, a):
    """Fraction of the unit cube below m . x = a, m1 <= m2 <= m3, sum 1, 0 <= a <= 1/2.
    Inclusion-exclusion: 6 m1 m2 m3 V = a^3 - sum_i (a - m_i)_+^3 (no further terms for
    a <= 1/2 except the slab case m3 >= m1 + m2), rearranged by regions of a."""
    m12 = m1 + m2
    with np.errstate(divide="ignore", invalid="ignore"):
        # a <= m1: tetrahedron a^3 / (6 m1 m2 m3) = (a / m1) a^2 / (6 m2 m3)
        vA = np.where(m1 > 0.0, (a / m1) * a * a / (6.0 * m2 * m3), 0.0)
        # m1 < a <= m2: (a^2 - a m1 + m1^2 / 3) / (2 m2 m3)
        vB = (a * a - a * m1 + m1 * m1 / 3.0) / (2.0 * m2 * m3)
        # m2 < a <= min(m12, m3), and m3 < a <= 1/2 when m3 < m12: the corners beyond
        # m2 and m3 removed, each cube (a - m_i)^3 / m1 written as (t / m1) t^2, t <= m1
        t2 = np.maximum(a - m2, 0.0)
        t3 = np.maximum(a - m3, 0.0)
        r2 = np.where(m1 > 0.0, t2 / m1, 0.0)
        r3 = np.where(m1 > 0.0, t3 / m1, 0.0)
        vC = (3.0 * a * a - 3.0 * a * m1 + m1 * m1 - r2 * t2 * t2 - r3 * t3 * t3) / (6.0 * m2 * m3)
        # m12 <= m3 and a > m12: a slab, linear in a
        vE = (2.0 * a - m12) / (2.0 * m3)
    return np.where(a <= m1, vA, np.where(a <= m2, vB, np.where((m12 <= m3) & (a > m12), vE, vC)))


def cut_fraction(n, beta):
    """Fraction of the box [0, 1]^d (d = n.shape[1]) on the side n . xi <= beta."""
    m, a, zero = _prep(n, beta)
    d = m.shape[1]
    m = np.where(zero[:, None], 1.0 / d, m)
    hi = a > 0.5
    b = np.clip(np.where(hi, 1.0 - a, a), 0.0, 0.5)
    v = _frac2(m[:, 0], m[:, 1], b) if d == 2 else _frac3(m[:, 0], m[:, 1], m[:, 2], b)
    v = np.where(hi, 1.0 - v, v)
    v = np.where(a <= 0.0, 0.0, np.where(a >= 1.0, 1.0, v))
    return np.where(zero, np.where(np.asarray(beta) >= 0.0, 1.0, 0.0), v)


def plane_constant(n, frac, iters=60):
    """beta with cut_fraction(n, beta) = frac (0 < frac < 1): closed forms where the
    fraction is a square-root, linear or cube-root function of a, bisection on the
    monotone cubic pieces.  Returned in the coordinates of n (before reflection);
    0 for a zero normal (no plane)."""
    n = np.asarray(n, dtype=np.float64)
    m, _, zero = _prep(n, np.zeros(n.shape[0]))
    m = np.where(zero[:, None], 1.0 / n.shape[1], m)
    s = np.sum(np.abs(n), axis=1)
    d = m.shape[1]
    f = np.asarray(frac, dtype=np.float64)
    hi = f > 0.5
    g = np.where(hi, 1.0 - f, f)                  # fraction <= 1/2: a <= 1/2
    m1, m2 = m[:, 0], m[:, 1]
    if d == 2:
        g1 = np.where(m1 > 0.0, m1 / (2.0 * m2), 0.0)
        a = np.where(g <= g1, np.sqrt(2.0 * m1 * m2 * g), g * m2 + 0.5 * m1)
    else:
        m3 = m[:, 2]
        m12 = m1 + m2
        gA = _frac3(m1, m2, m3, m1)
        gB = _frac3(m1, m2, m3, m2)
        aA = np.cbrt(6.0 * m1 * m2 * m3 * g)
        aB = 0.5 * (m1 + np.sqrt(np.maximum(8.0 * m2 * m3 * g - m1 * m1 / 3.0, 0.0)))
        slab = m12 <= m3
        gE = np.where(slab, _frac3(m1, m2, m3, m12), 2.0)
        aE = g * m3 + 0.5 * m12
        # bisection on the cubic pieces between a = m2 and a = 1/2 (or m12 for a slab)
        lo = m2.copy()
        up = np.where(slab, m12, 0.5)
        for _ in range(iters):
            mid = 0.5 * (lo + up)
            below = _frac3(m1, m2, m3, mid) < g
            lo = np.where(below, mid, lo)
            up = np.where(below, up, mid)
        aC = 0.5 * (lo + up)
        a = np.where(g <= gA, aA, np.where(g <= gB, aB, np.where(g >= gE, aE, aC)))
    a = np.where(hi, 1.0 - a, a)
    # back to the coordinates of n: scale, then undo the reflections
    return np.where(zero, 0.0, a * s + np.sum(np.minimum(n, 0.0), axis=1))
