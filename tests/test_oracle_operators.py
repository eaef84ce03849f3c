"""Pins of the reference-element operators (paper Sec. 2.1) against closed forms."""
import numpy as np
import pytest

from oracle.operators import operators


@pytest.mark.parametrize("n", range(1, 10))
def test_extrapolation_exact_for_degree_p(n):
    # Eq. Lmat: u^F = L u^S reproduces every polynomial of degree <= p = n-1.
    o = operators(n)
    for deg in range(n):
        assert np.allclose(o.L @ o.xs ** deg, o.xf ** deg, atol=1e-13)


@pytest.mark.parametrize("n", range(1, 10))
def test_derivative_exact_for_degree_p_plus_1(n):
    # Eq. Mmat: M differentiates every polynomial of degree <= n = p+1 supported on the
    # n+1 flux points exactly.
    o = operators(n)
    for deg in range(n + 1):
        exact = deg * o.xs ** (deg - 1) if deg > 0 else np.zeros(n)
        assert np.allclose(o.M @ o.xf ** deg, exact, atol=1e-11 * max(1, deg) ** 2)


@pytest.mark.parametrize("n", range(1, 10))
def test_row_sums_and_corrections(n):
    o = operators(n)
    assert np.allclose(o.L.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(o.M.sum(axis=1), 0.0, atol=1e-11)
    # Eq. cl:cr: the correction vectors select the interface flux points.
    assert o.xf[0] == -1.0 and o.xf[-1] == 1.0
    assert np.allclose(o.cL @ o.L, o.L[0]) and np.allclose(o.cR @ o.L, o.L[-1])
    # the first and last columns of M are M c_L and M c_R (Sec. 2.2)
    assert np.allclose(o.M @ o.cL, o.M[:, 0]) and np.allclose(o.M @ o.cR, o.M[:, -1])


@pytest.mark.parametrize("n", range(2, 10))
def test_compact_correction_scalars(n):
    # alpha = c_L^T L M c_R is the left-end derivative of the right correction function
    # l_{n+1/2}(x) = (1 + x) P_p(x) / 2, which is P_p(-1)/2 = (-1)^p / 2; beta = -alpha.
    o = operators(n)
    p = n - 1
    assert o.alpha == pytest.approx((-1) ** p / 2.0, abs=1e-12)
    assert o.beta == pytest.approx(-((-1) ** p) / 2.0, abs=1e-12)


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_rule(n):
    # n-point Gauss integrates degree <= 2n-1 exactly; flux points are -1, +1 plus the
    # roots of P_{n-1}.
    o = operators(n)
    for deg in range(2 * n):
        exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
        assert np.sum(o.ws * o.xs ** deg) == pytest.approx(exact, abs=1e-13)
    if n > 1:
        P = np.polynomial.legendre.Legendre.basis(n - 1)
        assert np.allclose(P(o.xf[1:-1]), 0.0, atol=1e-13)
    Pn = np.polynomial.legendre.Legendre.basis(n)
    assert np.allclose(Pn(o.xs), 0.0, atol=1e-13)
