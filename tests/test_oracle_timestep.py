"""Pins of the transcribed Runge-Kutta coefficients: the stability polynomial of each
scheme equals exp(z) through z^4, and the observed order on a nonlinear ODE is 4."""
import math

import numpy as np
import pytest

from oracle.timestep import STEPPERS


@pytest.mark.parametrize("name", ["rk4", "ssprk54", "lsrk54"])
def test_stability_polynomial(name):
    # Apply one step to y' = z y for several z and fit the polynomial R(z) of degree <= 5.
    zs = np.linspace(-0.5, 0.5, 11)
    vals = [STEPPERS[name](lambda y, z=z: z * y, np.array([1.0]), 1.0)[0] for z in zs]
    coef = np.polynomial.polynomial.polyfit(zs, vals, 5)
    for k in range(5):
        assert coef[k] == pytest.approx(1.0 / math.factorial(k), abs=1e-9)


@pytest.mark.parametrize("name", ["rk4", "ssprk54", "lsrk54"])
def test_nonlinear_order_four(name):
    # y' = -y^2 + sin-free autonomous nonlinearity, y(0) = 1: y(t) = 1 / (1 + t).
    def R(y):
        return -y * y
    errs = []
    for nsteps in (10, 20, 40):
        y = np.array([1.0])
        dt = 2.0 / nsteps
        for _ in range(nsteps):
            y = STEPPERS[name](R, y, dt)
        errs.append(abs(y[0] - 1.0 / 3.0))
    rates = [math.log(errs[i] / errs[i + 1], 2) for i in range(2)]
    assert min(rates) > 3.8
