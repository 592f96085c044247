"""Pins of the oracle's volume-weighted sum (``oracle.integral``): it equals
the exactly rounded sum of exact products (checked with ``fractions`` on
random inputs spanning many binades), so it is the reference for the GPU
sums; and on the dual volumes it reproduces the sphere's area and the
vanishing integral of an odd field."""
from fractions import Fraction

import numpy as np

from oracle import oracle


def test_exact_against_fractions():
    rng = np.random.default_rng(3)
    n = 400
    V = rng.uniform(0.5, 2.0, n) * 2.0 ** rng.integers(-30, 30, n)
    x = rng.standard_normal((n, 3)) * 2.0 ** rng.integers(-40, 40, (n, 3))
    x[:, 2] = -x[:, 1] * (1 + 2.0 ** -40)  # level 2 mirrors level 1, every value 2^-40 larger in size
    got = oracle.integral(V, x)
    for k in range(3):
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(V, x[:, k]))
        assert got[k] == float(exact)


def test_float32_inputs_are_upcast_exactly():
    rng = np.random.default_rng(4)
    V = rng.uniform(1.0, 3.0, 257)
    x = rng.standard_normal((257, 2)).astype(np.float32)
    exact = [float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(V, x[:, k]))) for k in range(2)]
    assert list(oracle.integral(V, x)) == exact


def test_sphere_area_and_odd_field(omesh):
    m = omesh(32)
    V = m.dual()["V"]
    g = m.grid()
    I = oracle.integral(V, np.stack([np.ones_like(V), np.sin(g["lat_node"])], 1))
    area = 4 * np.pi * oracle.R_EARTH ** 2
    assert abs(I[0] - area) <= 1e-12 * area
    # sin(lat) is odd under the north-south mirror, which maps the grid onto itself
    assert abs(I[1]) <= 1e-13 * area


def test_residual_after_cancelling_the_rounded_sum():
    """Each level holds random products plus one term that cancels their
    correctly rounded sum, so the exact result is the few-ulp residual that
    rounding left: it survives only if every product is exact and the whole
    sum is rounded once.  A naive sum, a product rounded to FP64, or a
    dropped partial product of the splitting each give a different value."""
    rng = np.random.default_rng(7)
    n, nlev = 300, 6
    V = np.concatenate([rng.uniform(0.5, 2.0, n) * 2.0 ** rng.integers(-20, 20, n), [1.0]])
    x = np.empty((n + 1, nlev))
    want = []
    for k in range(nlev):
        x[:n, k] = rng.standard_normal(n) * 2.0 ** rng.integers(-20, 20, n)
        terms = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(V[:n], x[:n, k])]
        s = float(sum(terms))
        x[n, k] = -s
        rest = sum(terms) - Fraction(s)
        assert rest != 0  # the rounded sum is inexact, so a residual is left
        want.append(float(rest))
    assert list(oracle.integral(V, x)) == want
