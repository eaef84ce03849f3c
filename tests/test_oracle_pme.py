"""Pins of the porous-medium oracle (Sec. 4.3) against the ZKB/Barenblatt solution
(Eq. zkb): the L2 error on |x|^2 < 0.9 H(t) (the footnote's restriction) is small and
falls with refinement, mass is conserved to round-off, and the t0 formula puts the
support of the initial profile inside one element."""
import numpy as np
import pytest

from oracle.diagnostics import l2_error
from oracle.grid import Grid
from oracle.physics import PorousMedium
from oracle.residual import residual
from oracle.timestep import STEPPERS
from paper_2608_09615_b300 import inputs


def run(E, p, scheme, t0=1.0, T=1.2, m=2.0, C=0.1, dt=None):
    g = Grid(1, (E,), (-10.0,), (10.0,), p)
    U = inputs.barenblatt_1d(E, p, m, C, t0)
    phys = PorousMedium(m)
    nst = int(round((T - t0) / dt))
    m0 = g.integrate(U[0])
    for _ in range(nst):
        U = STEPPERS["ssprk54"](lambda V: residual(V, g, scheme, phys), U, dt)
    (x,) = g.coordinates()
    alpha = 1.0 / ((m - 1.0) + 2.0)
    H = 2.0 * m * C / (alpha * (m - 1.0)) * T ** (2.0 * alpha)
    err = l2_error(U[0], inputs.barenblatt(x, T, m, C), g, mask=(x ** 2 < 0.9 * H))
    return err, g.integrate(U[0]) - m0, m0


def test_barenblatt_convergence_and_mass():
    errs = {}
    for scheme in ("compact", "br1"):
        e1, dm1, m0 = run(32, 4, scheme, dt=4e-4)
        e2, dm2, _ = run(64, 4, scheme, dt=2e-4)
        assert e2 < 0.7 * e1          # the front is a kink: slow but monotone convergence
        assert e2 < 1e-3
        assert abs(dm1) < 1e-12 * m0 and abs(dm2) < 1e-12 * m0
        errs[scheme] = e2
    # Sec. 4.3: the compact scheme's error is below the standard scheme's
    assert errs["compact"] < errs["br1"]


def test_t0_formula_single_element_support():
    # Sec. 4.3: t0 from u = 0 at |x| = dx/2 (m = 5, C = 0.1): the exact profile at t0
    # vanishes exactly at the element's half-width.
    m, C, dx = 5.0, 0.1, 0.1
    a1 = 1.0 / ((m - 1.0) + 2.0)
    t0 = (C * 2.0 * m / (a1 * (m - 1.0)) * (2.0 / dx) ** 2) ** (-1.0 / (2.0 * a1))
    assert inputs.barenblatt(np.array([dx / 2 * (1 - 1e-9)]), t0, m, C)[0] > 0
    assert inputs.barenblatt(np.array([dx / 2 * (1 + 1e-9)]), t0, m, C)[0] == 0
