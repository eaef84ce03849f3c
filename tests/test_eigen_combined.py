"""The combined-mode Fourier analysis of Appendix A (paper_2608_09615_b300.eigen.combined_mode)
on the Bloch operator built from the paper's Sec. 3 matrices (tests/bloch_sec3.py), CPU only.

Pins: an eigenvector as initial data returns its own eigen-frequency at any t; t -> 0 gives
the Rayleigh quotient of B; the eigen-expansion evolution equals the matrix exponential; the
well-resolved Fourier mode decays as the exact solution (omega = -i theta^2 for u_t = u_xx
with h = 1). And the appendix's observations: the standard (BR1) formulation is less
dissipative than the compact one at medium and high wavenumbers, and the interior penalty
raises the high-wavenumber dissipation as eta_IP grows."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from bloch_sec3 import bloch_B
from oracle.operators import operators
from paper_2608_09615_b300.eigen import combined_mode


def _B(p, scheme, eta=0.0):
    return lambda th: bloch_B(p + 1, th, scheme, h=1.0, eta_ip=eta)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [1, 3])
def test_eigenvector_initial_data_returns_its_eigenvalue(p, scheme):
    xi = operators(p + 1).xs
    th = 1.3
    Bf = _B(p, scheme)
    lam, N = np.linalg.eig(Bf(th))
    for j in range(p + 1):
        for t in (0.01, 0.3):
            G, om = combined_mode(Bf, xi, [th], t, initial=lambda a: N[:, j])
            # (BR1 has nearly parallel eigenvectors at some theta: ill-conditioned N)
            assert abs(om[0] - 1j * lam[j]) <= 1e-6 * max(1.0, abs(lam[j]))


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_expansion_equals_matrix_exponential_and_small_t_limit(scheme):
    p = 3
    xi = operators(p + 1).xs
    th = np.array([0.4, 2.0, 5.5, 9.0])
    Bf = _B(p, scheme)
    for t in (1e-3, 0.05, 0.2):
        G, om = combined_mode(Bf, xi, th, t)
        for k, a in enumerate(th):
            u0 = np.exp(1j * a * (xi + 1) / 2)
            ref = np.vdot(u0, expm(Bf(a) * t) @ u0) / np.vdot(u0, u0)
            assert abs(G[k] - ref) <= 1e-10 * max(1.0, abs(ref))
    # t -> 0: omega -> i (u0* B u0) / (u0* u0)
    G, om = combined_mode(Bf, xi, th, 1e-7)
    for k, a in enumerate(th):
        u0 = np.exp(1j * a * (xi + 1) / 2)
        rq = np.vdot(u0, Bf(a) @ u0) / np.vdot(u0, u0)
        assert abs(om[k] - 1j * rq) <= 1e-5 * abs(rq)
    G0, _ = combined_mode(Bf, xi, [0.3], 0.0 + 1e-12)
    assert abs(G0[0] - 1) < 1e-10


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_resolved_modes_decay_as_the_exact_solution(p, scheme):
    xi = operators(p + 1).xs
    th = np.array([0.25, 0.5, 1.0])
    G, om = combined_mode(_B(p, scheme), xi, th, 0.1)
    # omega = -i theta^2 for the exact solution of u_t = u_xx (h = nu = 1)
    assert np.all(np.abs(om.imag + th ** 2) <= 2e-2 * th ** 2), om
    assert np.all(np.abs(G) <= 1.0 + 1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_standard_formulation_less_dissipative_at_high_wavenumbers(p):
    xi = operators(p + 1).xs
    th = np.linspace(0.5 * (p + 1) * math.pi, (p + 1) * math.pi, 25)
    _, om_c = combined_mode(_B(p, "compact"), xi, th, 0.1)
    _, om_b = combined_mode(_B(p, "br1"), xi, th, 0.1)
    # dissipation = -Im(omega)
    assert np.mean(-om_c.imag) > np.mean(-om_b.imag)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [3, 4])
def test_interior_penalty_raises_high_wavenumber_dissipation(p, scheme):
    xi = operators(p + 1).xs
    th = np.linspace(0.75 * (p + 1) * math.pi, (p + 1) * math.pi, 9)
    d = []
    for eta in (0.0, 0.01, 0.02, 0.05):
        _, om = combined_mode(_B(p, scheme, eta), xi, th, 0.1)
        d.append(np.mean(-om.imag))
    assert all(b > a for a, b in zip(d, d[1:])), d
