"""Pins of the oracle's interface viscous flux option (b) of Sec. 2.1 step 4, the average
of the two sides' viscous fluxes (G(u_L, v_L) + G(u_R, v_R)) / 2, against what the
mathematics fixes:
* for the heat equation the flux is linear in v, so (b) equals option (a), G(u_hat, v_hat),
  to round-off, with and without the interior penalty;
* the two options differ by a term quadratic in the interface jumps: about a uniform
  state U0, (b) - (a) scales as eps^2 for U0 + eps dU, while the residual itself scales
  as eps;
* (b) keeps the discrete conservation and the free-stream preservation of the scheme."""
import math

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.physics import Heat, NavierStokes, NSParams, PorousMedium
from oracle.residual import residual
from paper_2608_09615_b300 import inputs

TWO_PI = 2 * math.pi


@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("dim,ne,p", [(1, (7,), 3), (3, (3, 2, 4), 2)])
@pytest.mark.parametrize("eta", [0.0, 0.5])
def test_heat_options_agree(scheme, dim, ne, p, eta):
    g = Grid(dim, ne, (0.0,) * dim, (1.0,) * dim, p)
    U = inputs.random_scalar(dim, ne, p, seed=11)
    Ra = residual(U, g, scheme, Heat(0.7), eta_ip=eta)
    Rb = residual(U, g, scheme, Heat(0.7), eta_ip=eta, viscous="b")
    assert np.abs(Rb - Ra).max() <= 1e-12 * np.abs(Ra).max()


def _ns_state(ne, p, eps, seed):
    prm = NSParams(Re=50.0)
    rng = np.random.default_rng(seed)
    U0 = inputs.tgv_3d(ne, p) * 0.0
    U0[0] = prm.rho0
    U0[4] = prm.p0 / (prm.gamma - 1.0) + 0.5 * prm.rho0 * 0.3 ** 2
    U0[1] = prm.rho0 * 0.3
    dU = rng.uniform(-1.0, 1.0, U0.shape) * np.array([0.1, 0.3, 0.3, 0.3, 1.0]).reshape((5,) + (1,) * (U0.ndim - 1))
    return prm, U0, U0 + eps * dU


@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_options_differ_quadratically_in_the_jumps(scheme):
    ne, p = (3, 2, 2), 2
    g = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p)
    diffs, res = [], []
    for eps in (1e-2, 5e-3, 2.5e-3):
        prm, U0, U = _ns_state(ne, p, eps, seed=3)
        ns = NavierStokes(prm)
        Ra = residual(U, g, scheme, ns)
        Rb = residual(U, g, scheme, ns, viscous="b")
        diffs.append(np.abs(Rb - Ra).max())
        res.append(np.abs(Ra).max())
    # residual ~ eps, (b) - (a) ~ eps^2
    assert 1.8 < res[0] / res[1] < 2.2 and 1.8 < res[1] / res[2] < 2.2
    assert 3.6 < diffs[0] / diffs[1] < 4.4 and 3.6 < diffs[1] / diffs[2] < 4.4
    assert diffs[0] > 1e-9 * res[0]                       # the options do differ


@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_option_b_conserves_and_preserves_free_stream(scheme):
    ne, p = (3, 3, 2), 3
    g = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p)
    prm, U0, U = _ns_state(ne, p, 0.05, seed=5)
    ns = NavierStokes(prm)
    R0 = residual(U0, g, scheme, ns, viscous="b")
    assert np.abs(R0).max() <= 1e-10 * np.abs(U0).max()
    R = residual(U, g, scheme, ns, viscous="b", eta_ip=0.3)
    W = g.quadrature_weights()
    for v in range(5):
        assert abs(np.sum(W * R[v])) <= 1e-12 * np.sum(W * np.abs(R[v]))


def test_pme_option_b_quadratic_in_jumps():
    ne, p = (9,), 3
    g = Grid(1, ne, (0.0,), (1.0,), p)
    dU = np.random.default_rng(2).uniform(-1, 1, (1, 9, 4))
    diffs = []
    for eps in (1e-2, 5e-3):
        U = 1.0 + eps * dU
        Ra = residual(U, g, "compact", PorousMedium(2.0))
        Rb = residual(U, g, "compact", PorousMedium(2.0), viscous="b")
        diffs.append(np.abs(Rb - Ra).max())
    assert 3.6 < diffs[0] / diffs[1] < 4.4


# ------------------------------------------------------------------ PME diffusivity at solution points
@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("viscous", ["a", "b"])
def test_pme_solution_point_coef_exact_cases(scheme, viscous):
    # m = 1: the diffusivity is 1 everywhere, both variants are the heat equation;
    # m = 2 with u > 0: m |u|^(m-1) = 2u is a polynomial of degree p in each element, so
    # extrapolating it from the solution points is exact and the variants agree
    # (the extrapolated traces must stay positive too: small variations about 1.5)
    g = Grid(1, (9,), (0.0,), (1.0,), 3)
    U = 1.5 + 0.2 * inputs.random_scalar(1, (9,), 3, seed=4)
    for m in (1.0, 2.0):
        Rf = residual(U, g, scheme, PorousMedium(m), viscous=viscous)
        Rs = residual(U, g, scheme, PorousMedium(m, coef="solution"), viscous=viscous)
        assert np.abs(Rs - Rf).max() <= 1e-12 * np.abs(Rf).max()
    Rh = residual(U, g, scheme, Heat(1.0), viscous=viscous)
    assert np.abs(residual(U, g, scheme, PorousMedium(1.0, coef="solution"), viscous=viscous) - Rh).max() \
        <= 1e-12 * np.abs(Rh).max()
    # m = 3: 3 u^2 has degree 2p, the variants differ
    Rf = residual(U, g, scheme, PorousMedium(3.0), viscous=viscous)
    Rs = residual(U, g, scheme, PorousMedium(3.0, coef="solution"), viscous=viscous)
    assert np.abs(Rs - Rf).max() > 1e-6 * np.abs(Rf).max()


@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_pme_solution_point_coef_barenblatt(scheme):
    # m = 3 Barenblatt run with the diffusivity at the solution points: mass conserved to
    # round-off, error small and falling with refinement
    from oracle.diagnostics import l2_error
    from oracle.timestep import STEPPERS
    m, C, t0, T = 3.0, 0.1, 1.0, 1.1
    errs = []
    for E, dt in ((32, 2e-4), (64, 1e-4)):
        g = Grid(1, (E,), (-10.0,), (10.0,), 4)
        U = inputs.barenblatt_1d(E, 4, m, C, t0)
        phys = PorousMedium(m, coef="solution")
        m0 = g.integrate(U[0])
        for _ in range(int(round((T - t0) / dt))):
            U = STEPPERS["ssprk54"](lambda V: residual(V, g, scheme, phys), U, dt)
        (x,) = g.coordinates()
        alpha = 1.0 / ((m - 1.0) + 2.0)
        H = 2.0 * m * C / (alpha * (m - 1.0)) * T ** (2.0 * alpha)
        errs.append(l2_error(U[0], inputs.barenblatt(x, T, m, C), g, mask=(x ** 2 < 0.9 * H)))
        assert abs(g.integrate(U[0]) - m0) < 1e-12 * m0
    assert errs[1] < 0.8 * errs[0] and errs[1] < 1e-2
