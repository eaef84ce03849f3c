"""Pins of the NS oracle and its diagnostics against the Taylor-Green closed forms
(Sec. 4.4): E_k/|Omega| = u0^2/8 and int omega.omega/|Omega| = 3/4 (u0/L)^2 at t = 0,
and the initial kinetic-energy decay -dE_k/dt = nu int omega.omega of the
incompressible limit (the flow is at Ma = 0.1 and smooth at t = 0, so the numerical and
compressible contributions are O(1e-3))."""
import numpy as np
import pytest

from oracle.diagnostics import ns_diagnostics
from oracle.grid import Grid
from oracle.physics import NavierStokes, NSParams
from oracle.residual import residual
from paper_2608_09615_b300 import inputs


@pytest.mark.parametrize("p", [3, 4])
def test_tgv_initial_energy_enstrophy(p):
    ne = (6, 6, 6)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, p)
    U = inputs.tgv_3d(ne, p)
    d = ns_diagnostics(U, g)
    vol = (2 * np.pi) ** 3
    assert d["volume"] == pytest.approx(vol, rel=1e-14)
    assert d["ke"] / vol == pytest.approx(1.0 / 8.0, abs=1e-12)
    assert d["ke_rho"] / vol == pytest.approx(1.0 / 8.0, abs=1e-12)
    assert d["enstrophy"] / vol == pytest.approx(0.75, abs=1e-4)
    assert d["mass"] / vol == pytest.approx(1.0, abs=1e-12)
    assert max(abs(m) for m in d["mom"]) < 1e-12
    prm = NSParams()
    # mean of p over the cube is p0; E = p/(gamma-1) + rho |u|^2 / 2
    assert d["energy"] / vol == pytest.approx(prm.p0 / (prm.gamma - 1) + 1.0 / 8.0, rel=1e-12)
    assert d["nonfinite"] == 0


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_tgv_initial_dissipation_rate(scheme):
    ne = (6, 6, 6)
    p = 4
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, p)
    U = inputs.tgv_3d(ne, p)
    prm = NSParams(Re=1600.0)
    R = residual(U, g, scheme, NavierStokes(prm))
    W = g.quadrature_weights()
    rho = U[0]
    vel = [U[1 + i] / rho for i in range(3)]
    dudt = [(R[1 + i] - vel[i] * R[0]) / rho for i in range(3)]
    dEk = np.sum(W * sum(vel[i] * dudt[i] for i in range(3)))
    eps = prm.mu0 / prm.rho0 * ns_diagnostics(U, g)["enstrophy"]
    assert -dEk == pytest.approx(eps, rel=5e-3)


def test_nonfinite_flag():
    ne = (2, 2, 2)
    g = Grid(3, ne, (0.0,) * 3, (1.0,) * 3, 2)
    U = inputs.tgv_3d(ne, 2)
    U[4, 1, 0, 1, 2, 0, 1] = np.nan
    assert ns_diagnostics(U, g)["nonfinite"] == 1
