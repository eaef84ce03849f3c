"""Pin of the 1D oracle residual against the temporal-eigenanalysis operator of the
paper's Sec. 3, which restates the 1D compact scheme as explicit matrices acting on one
element under the Bloch condition u_{e+-1} = u_e exp(+-i theta):

  H(theta)   = L + 1/2 cL cR^T L e^{-i theta} - 1/2 cL cL^T L
                 + 1/2 cR cL^T L e^{+i theta} - 1/2 cR cR^T L
  W^L        = J^-1 M [H - 1/2 cR cL^T L e^{+i theta} + 1/2 cR cR^T L]
  W^R        = J^-1 M [H - 1/2 cL cR^T L e^{-i theta} + 1/2 cL cL^T L]
  Q          = (I - cL cL^T - cR cR^T) L J^-1 M H
               + 1/2 cL cR^T L W^R e^{-i theta} + 1/2 cL cL^T L W^L
               + 1/2 cR cL^T L W^L e^{+i theta} + 1/2 cR cR^T L W^R
  v^{F,C}    = Q u^S

These are written here from the equations of Sec. 3 (not from the oracle): the two
computations share only the operator matrices. For BR1 the same algebra holds with
W^L = W^R = J^-1 M H (both faces extrapolate the one v^S, Sec. 2.1).

Reading of the sign (the paper's B = -M Q is stated for its own sign convention): for
u_t = u_xx the flux is G = -v, so du/dt = -J^-1 M G = J^-1 M Q u; with h = 2 (the
reference element, J = 1) the wavenumber per unit length is theta/2; with h = 1
(J^-1 = 2, the scaling the paper says is folded into the formulation) the physical
eigenvalue must be -theta^2 (decay)."""
import numpy as np
import pytest

from bloch_sec3 import bloch_Q, bloch_Q_ip
from oracle.grid import Grid
from oracle.operators import operators
from oracle.physics import Heat
from oracle.residual import residual


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_residual_matches_bloch_operator(scheme, p):
    n = p + 1
    E = 12
    rng = np.random.default_rng(p)
    for h in (2.0, 1.0, 0.3):
        _check(scheme, p, E, h, rng)


def _check(scheme, p, E, h, rng):
    n = p + 1
    g = Grid(1, (E,), (0.0,), (h * E,), p)
    Jinv = 2.0 / h
    for k in (1, 3, 5):
        theta = 2 * np.pi * k / E
        uhat = rng.normal(size=n) + 1j * rng.normal(size=n)
        U = (np.exp(1j * theta * np.arange(E))[:, None] * uhat[None, :])[None]
        R = residual(U, g, scheme, Heat(1.0))
        B = Jinv * operators(n).M @ bloch_Q(n, theta, scheme, Jinv)
        for e in range(E):
            assert np.allclose(R[0, e], np.exp(1j * theta * e) * (B @ uhat), atol=1e-11)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_bloch_physical_mode_decays_like_theta_squared(scheme, p):
    # Sec. 3: centred schemes have real spectra; the least-damped eigenvalue of B
    # approximates the exact -theta^2 for resolved theta.
    n = p + 1
    for theta in (0.05, 0.1, 0.2):
        B = 2.0 * operators(n).M @ bloch_Q(n, theta, scheme, 2.0)   # h = 1
        ev = np.linalg.eigvals(B)
        assert np.abs(ev.imag).max() < 1e-8
        phys = ev.real[np.argmax(ev.real)]
        assert phys == pytest.approx(-theta ** 2, rel=1e-3)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("eta", [0.01, 1.0])
def test_residual_with_interior_penalty_matches_bloch_operator(scheme, p, eta):
    # Sec. 3: v^{F,C} = (Q + Q_IP) u with tau = eta_IP (p+1)^2 / h
    n = p + 1
    E = 10
    rng = np.random.default_rng(p)
    for h in (2.0, 0.5):
        g = Grid(1, (E,), (0.0,), (h * E,), p)
        Jinv = 2.0 / h
        tau = eta * (p + 1) ** 2 / h
        for k in (1, 4):
            theta = 2 * np.pi * k / E
            uhat = rng.normal(size=n) + 1j * rng.normal(size=n)
            U = (np.exp(1j * theta * np.arange(E))[:, None] * uhat[None, :])[None]
            R = residual(U, g, scheme, Heat(1.0), eta_ip=eta)
            B = Jinv * operators(n).M @ (bloch_Q(n, theta, scheme, Jinv) + bloch_Q_ip(n, theta, tau))
            for e in range(E):
                assert np.allclose(R[0, e], np.exp(1j * theta * e) * (B @ uhat), atol=1e-10)
