"""Pins of the oracle's opacity functions (Sec. 2.1, Sec. 2.2) against
quadrature of their definitions, library special functions and limits."""
import numpy as np
import pytest
import scipy.special as ss

from oracle import analytic as A
from oracle import coracle as C

XS = np.array([0.0, 1e-8, 1e-3, 0.05, 0.1999, 0.2, 0.2001, 0.5, 0.9241, 1.0, 1.5, 2.0, 3.255, 5.0,
               7.3, 10.0, 27.0, 60.0, 300.0, 2500.0, 1e5])


def test_damping_parameter_values():
    # a = 4.702e-4 T4^(-1/2) (Sec. 2.1): 4.702e-4 at 1e4 K, x10 at 100 K.
    assert C.damping(1.0e4) == pytest.approx(4.702e-4, rel=1e-15)
    assert C.damping(1.0e2) == pytest.approx(4.702e-3, rel=1e-15)


def test_dawson_matches_scipy_and_is_odd():
    ref = ss.dawsn(XS)
    got = C.dawson(XS)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.all(rel[XS > 0] < 2e-14), rel
    assert np.allclose(C.dawson(-XS), -got, rtol=0, atol=0)


@pytest.mark.parametrize("x", [1e-3, 0.15, 0.7, 1.3, 2.9, 6.0, 15.0])
def test_dawson_matches_quadrature_of_definition(x):
    assert C.dawson(x) == pytest.approx(A.dawson_quad(x), rel=1e-12)


def test_dawson_asymptotic_limit():
    # F(x) -> 1/(2x) + 1/(4x^3) + 3/(8x^5) for large x.
    x = np.array([200.0, 1e3, 1e4])
    asym = 1 / (2 * x) + 1 / (4 * x ** 3) + 3 / (8 * x ** 5)
    assert np.allclose(C.dawson(x), asym, rtol=1e-13, atol=0)


@pytest.mark.parametrize("T", [1.0e4, 10.0, 1.0e2])
def test_voigt_second_order_expansion_error_is_order_a_cubed(T):
    # eq. H_approx is H to second order in a: its error vs the exact Voigt
    # function (Faddeeva, and quadrature of eq. H) is O(a^3) in the core and
    # relatively O(a^2) in the wing.
    a = C.damping(T)
    x = np.array([0.0, 0.3, 1.0, 2.0, 3.0, 4.0, 6.0, 10.0, 30.0])
    exact = A.voigt_faddeeva(a, x)
    got = C.voigt_H(a, x)
    tol = 4.0 * a ** 3 + 4.0 * a ** 2 * np.abs(exact) + 1e-14
    assert np.all(np.abs(got - exact) <= tol), (got - exact, tol)
    for xv in (0.0, 1.0, 3.0):
        assert C.voigt_H(a, xv) == pytest.approx(A.voigt_quad(a, xv), abs=4.0 * a ** 3 + 1e-12)


def test_voigt_limits():
    a = C.damping(1.0e4)
    # core: e^{-x^2}; line centre H(a,0) = 1 - 2a/sqrt(pi) + a^2
    assert C.voigt_H(a, 0.0) == pytest.approx(1 - 2 * a / np.sqrt(np.pi) + a * a, rel=1e-15)
    # wing: a / (sqrt(pi) x^2)
    for x in (50.0, 200.0, 1000.0):
        assert C.voigt_H(a, x) == pytest.approx(a / (np.sqrt(np.pi) * x * x), rel=2.0 / x ** 2)


@pytest.mark.parametrize("T", [1.0e4, 10.0])
def test_integrated_profile_matches_quadrature(T):
    a = C.damping(T)
    for x in (0.1, 0.8, 2.0, 4.0, 12.0):
        q = A.bin_mean_quad(C.voigt_H, a, 0.0, x) * x
        assert C.voigt_Hint(a, x) == pytest.approx(q, rel=1e-11)
    # odd in x, and int_{-inf}^{inf} H = sqrt(pi) (normalisation of the profile)
    assert C.voigt_Hint(a, -2.7) == pytest.approx(-C.voigt_Hint(a, 2.7), rel=1e-15)
    big = C.voigt_Hint(a, 1.0e7)
    assert 2.0 * big == pytest.approx(np.sqrt(np.pi), rel=1e-6)


@pytest.mark.parametrize("T", [1.0e4, 10.0])
@pytest.mark.parametrize("lo,hi", [(-0.117, 0.117), (0.0, 0.234375), (1.2, 1.434375), (-3.1, -2.9),
                                    (5.0, 5.25), (59.765625, 60.0), (-60.0, -59.765625), (2450.5, 2500.0),
                                    (-30.0, -29.53125), (24.0, 74.0)])
def test_bin_mean_matches_quadrature(T, lo, hi):
    # k_j / k0 = (calH(x+) - calH(x-)) / dx_j must equal the bin average of eq. H_approx,
    # including far-wing bins where erf(x) -> 1 would cancel.
    a = C.damping(T)
    ref = A.bin_mean_quad(C.voigt_H, a, lo, hi)
    assert C.bin_mean_H(a, lo, hi) == pytest.approx(ref, rel=5e-10)
