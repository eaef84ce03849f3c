"""Pins of the three Navier-Stokes ingredients of Sec. 4.4 that the residual pins elsewhere
never reach on their own: Sutherland's viscosity law away from the reference temperature,
the viscous stress tensor (its transpose and its zero bulk viscosity, lambda = 0) and the
Harten entropy fix of the Roe flux.

Each pin compares the oracle with a closed form derived by hand from the mathematics, and
each has a companion test that plants the plausible one-line mistake in a subclass of the
oracle (on the CPU) and checks that the pin then fails."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle.physics import NavierStokes, NSParams
from oracle.residual import residual
from paper_2608_09615_b300 import inputs

SCHEMES = ("br1", "compact")


# ------------------------------------------------------------------------ Sutherland
def test_sutherland_textbook_ratio():
    # Sutherland's law for air (S = 110.4 K, T0 = 300 K): mu(600 K)/mu(300 K)
    # = 2^(3/2) * 410.4 / 710.4 = 1.633990, mu(150 K)/mu(300 K) = 2^(-3/2) 410.4/260.4
    # = 0.557213.
    # e/e0 = T/T0 for a calorically perfect gas.
    ns = NavierStokes(NSParams(sutherland=True))
    e0, mu0 = ns.prm.e0, ns.prm.mu0
    r = ns.viscosity(np.array([2.0 * e0, 0.5 * e0, e0])) / mu0
    assert abs(r[0] - 1.6339900) < 1e-6
    assert abs(r[1] - 0.5572132) < 1e-6
    assert abs(r[2] - 1.0) < 1e-15
    # high-temperature limit: mu ~ T^(1/2) (the law's defining asymptote)
    big = ns.viscosity(np.array([1e6 * e0, 4e6 * e0]))
    assert abs(big[1] / big[0] - 2.0) < 1e-5


def _sutherland_heat_case(phys, scheme):
    """Fluid at rest with uniform pressure and rho = rho0 (1 + eps sin x), eps = 0.3: the
    internal energy e = e0 / (1 + eps sin x) spans T/T0 in [0.77, 1.43]. Only the energy
    equation moves: d(rho E)/dt = d/dx (kappa dT/dx) = (gamma/Pr) d/dx (mu(e) e'), written
    out as (gamma/Pr) (mu'(e) e'^2 + mu(e) e'') with Sutherland's mu(e) and its derivative
    done by hand. Returns (R, expected energy residual)."""
    prm = phys.prm
    ne = (12, 1, 1)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi, 1.0, 1.0), 5)
    X = g.coordinates()
    eps = 0.3
    s, c = np.sin(X[0]), np.cos(X[0])
    rho = prm.rho0 * (1 + eps * s)
    zero = np.zeros_like(rho)
    U = inputs.primitive_to_conservative(rho, (zero, zero, zero), prm.p0 + zero, prm.gamma)
    R = residual(U, g, scheme, phys)
    e0, S, mu0 = prm.e0, prm.suth_s, prm.mu0
    e = e0 / (1 + eps * s)
    ep = -e0 * eps * c / (1 + eps * s) ** 2
    epp = e0 * (eps * s * (1 + eps * s) + 2 * eps ** 2 * c ** 2) / (1 + eps * s) ** 3
    th = e / e0
    mu = mu0 * (1 + S) * th ** 1.5 / (th + S)
    # d mu / d theta = mu0 (1+S) theta^(1/2) (theta/2 + 3S/2) / (theta + S)^2
    dmu = mu0 * (1 + S) * np.sqrt(th) * (0.5 * th + 1.5 * S) / (th + S) ** 2 / e0
    expect = prm.gamma / prm.Pr * (dmu * ep ** 2 + mu * epp)
    return R, expect


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sutherland_heat_conduction_closed_form(scheme):
    phys = NavierStokes(NSParams(Re=10.0, sutherland=True))
    R, expect = _sutherland_heat_case(phys, scheme)
    assert np.abs(R[:4]).max() < 1e-9 * np.abs(expect).max()
    assert np.abs(R[4] - expect).max() < 2e-3 * np.abs(expect).max()


class _SutherlandWrongExponent(NavierStokes):
    """Planted mistake: theta^(1/2) in place of theta^(3/2)."""

    def viscosity(self, e):
        prm = self.prm
        th = e / prm.e0
        return prm.mu0 * th ** 0.5 * (1.0 + prm.suth_s) / (th + prm.suth_s)


class _SutherlandNoConstant(NavierStokes):
    """Planted mistake: the factor (1 + S/T0) dropped."""

    def viscosity(self, e):
        prm = self.prm
        th = e / prm.e0
        return prm.mu0 * th ** 1.5 / (th + prm.suth_s)


@pytest.mark.parametrize("mutant", [_SutherlandWrongExponent, _SutherlandNoConstant])
def test_sutherland_pin_catches_planted_mistakes(mutant):
    R, expect = _sutherland_heat_case(mutant(NSParams(Re=10.0, sutherland=True)), "compact")
    assert np.abs(R[4] - expect).max() > 2e-2 * np.abs(expect).max()


# ------------------------------------------------------------------ viscous stress
def _viscous_part(phys_cls, U, g, scheme, **kw):
    """The viscous part of the residual: with constant mu the residual is R_c + mu0 V, so
    V = (R(mu_a) - R(mu_b)) / (mu_a - mu_b) removes the convective part exactly."""
    pa = NSParams(Re=10.0, sutherland=False, **kw)
    pb = NSParams(Re=20.0, sutherland=False, **kw)
    Ra = residual(U, g, scheme, phys_cls(pa))
    Rb = residual(U, g, scheme, phys_cls(pb))
    return (Ra - Rb) / (pa.mu0 - pb.mu0)


def _stress_case(phys_cls, scheme, field):
    """rho = rho0, p = p0 uniform; velocity eps*(sin x, sin y, sin z) ("compressive": div u
    != 0) or eps*(sin y, sin z, sin x) ("shear": div u = 0). With tau = mu (grad u +
    grad u^T) and lambda = 0 the momentum residual's viscous part is
    mu (lap u + grad div u):
      compressive: -2 mu eps sin x_i  (lap u_i = grad_i div u = -eps sin x_i)
      shear:       -mu eps sin x_{i+1} (grad div u = 0)
    and the energy row's viscous part div(u . tau) (the temperature is not uniform, since e
    = E - |u|^2/2 with p and rho uniform is constant: no heat flux):
      compressive: tau_ij = 2 mu eps cos x_i delta_ij, so div(u.tau) = 2 mu eps^2 sum cos 2x_j
      shear:       eps^2 sum cos 2x_j (worked out below).
    Returns (V / mu0 for momentum and energy, expected)."""
    prm = NSParams()
    ne = (6, 6, 6)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, 5)
    X = g.coordinates()
    eps = 0.05
    if field == "compressive":
        vel = [eps * np.sin(X[i]) for i in range(3)]
    else:
        vel = [eps * np.sin(X[(i + 1) % 3]) for i in range(3)]
    rho = prm.rho0 + 0 * X[0]
    U = inputs.primitive_to_conservative(rho, vel, prm.p0 + 0 * X[0], prm.gamma)
    V = _viscous_part(phys_cls, U, g, scheme)
    if field == "compressive":
        mom = [-2 * eps * np.sin(X[i]) for i in range(3)]
        en = 2 * eps ** 2 * sum(np.cos(2 * X[j]) for j in range(3))
    else:
        # u_i = eps sin x_{i+1}: the only nonzero velocity derivatives are
        # d u_i / d x_{i+1} = eps cos x_{i+1}, so tau_{i,i+1} = tau_{i+1,i} = mu eps cos x_{i+1}
        mom = [-eps * np.sin(X[(i + 1) % 3]) for i in range(3)]
        # (u . tau)_j = u_{j+1} tau_{j+1,j} + u_{j+2} tau_{j+2,j} (indices mod 3)
        #            = eps sin x_{j+2} * eps cos x_{j+1} + eps sin x_j * eps cos x_j;
        # only the second term depends on x_j: div(u . tau) = eps^2 sum_j cos 2 x_j
        en = eps ** 2 * sum(np.cos(2 * X[j]) for j in range(3))
    return V, mom, en


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("field", ["compressive", "shear"])
def test_viscous_stress_closed_form(scheme, field):
    V, mom, en = _stress_case(NavierStokes, scheme, field)
    sc = max(np.abs(m).max() for m in mom)
    assert np.abs(V[0]).max() < 1e-9 * sc
    for i in range(3):
        assert np.abs(V[1 + i] - mom[i]).max() < 5e-3 * sc
    # (the energy row is O(eps^2); BR1 at odd p carries a larger discretisation error)
    assert np.abs(V[4] - en).max() < 2e-2 * np.abs(en).max()


class _StressNoTranspose(NavierStokes):
    """Planted mistake: tau = mu grad u (the transpose dropped)."""

    def viscous_flux(self, U, grad, m):
        Fv = super().viscous_flux(U, grad, m)
        rho, vel, E, e, p = self.primitives(U)
        mu = self.viscosity(e)
        du = [[(grad[k][1 + i] - vel[i] * grad[k][0]) / rho for i in range(3)] for k in range(3)]
        for i in range(3):
            wrong = mu * du[m][i]
            Fv[4] += vel[i] * (wrong - Fv[1 + i])
            Fv[1 + i] = wrong
        return Fv


class _StressStokesLambda(NavierStokes):
    """Planted mistake: Stokes' bulk viscosity lambda = -2/3 mu instead of the paper's 0."""

    def viscous_flux(self, U, grad, m):
        Fv = super().viscous_flux(U, grad, m)
        rho, vel, E, e, p = self.primitives(U)
        mu = self.viscosity(e)
        div = sum((grad[k][1 + k] - vel[k] * grad[k][0]) / rho for k in range(3))
        extra = -2.0 / 3.0 * mu * div
        Fv[1 + m] = Fv[1 + m] + extra
        Fv[4] = Fv[4] + vel[m] * extra
        return Fv


class _StressTransposeOnly(NavierStokes):
    """Planted mistake: tau = mu grad u^T only (the indices of du swapped)."""

    def viscous_flux(self, U, grad, m):
        Fv = super().viscous_flux(U, grad, m)
        rho, vel, E, e, p = self.primitives(U)
        mu = self.viscosity(e)
        du = [[(grad[k][1 + i] - vel[i] * grad[k][0]) / rho for i in range(3)] for k in range(3)]
        for i in range(3):
            wrong = mu * du[i][m]
            Fv[4] += vel[i] * (wrong - Fv[1 + i])
            Fv[1 + i] = wrong
        return Fv


@pytest.mark.parametrize("mutant,field", [(_StressNoTranspose, "compressive"),
                                          (_StressStokesLambda, "compressive"),
                                          (_StressTransposeOnly, "shear")])
def test_viscous_stress_pin_catches_planted_mistakes(mutant, field):
    V, mom, en = _stress_case(mutant, "compact", field)
    sc = max(np.abs(m).max() for m in mom)
    err = max(np.abs(V[1 + i] - mom[i]).max() for i in range(3))
    assert err > 0.2 * sc


# ---------------------------------------------------------------------- Harten fix
def _roe_average(UL, UR, gamma):
    """Roe's averaged velocity, enthalpy and sound speed (the sqrt(rho)-weighted means)."""
    def prim(U):
        rho = U[0]
        vel = [U[1 + i] / rho for i in range(3)]
        p = (gamma - 1) * (U[4] - 0.5 * rho * sum(v * v for v in vel))
        return rho, vel, (U[4] + p) / rho
    rl, vl, Hl = prim(UL)
    rr, vr, Hr = prim(UR)
    a, b = np.sqrt(rl), np.sqrt(rr)
    ut = [(a * vl[i] + b * vr[i]) / (a + b) for i in range(3)]
    Ht = (a * Hl + b * Hr) / (a + b)
    c = np.sqrt((gamma - 1) * (Ht - 0.5 * sum(w * w for w in ut)))
    return ut, Ht, c


def _slow_acoustic_pair(gamma, qn_target_minus_c, strength):
    """A pair of states joined by a pure slow acoustic wave of the Roe matrix along x:
    U_R - U_L = s r_1(U~) with r_1 = (1, u~ - c~, v~, w~, H~ - u~ c~) evaluated at the Roe
    average of the pair itself (found by fixed-point iteration), and the Roe-averaged
    eigenvalue lambda_1 = u~ - c~ near the given value."""
    rho, v, w, p = 1.0, 0.1, -0.05, 1.0
    c_guess = np.sqrt(gamma * p / rho)
    u = c_guess + qn_target_minus_c
    UL = inputs.primitive_to_conservative(np.array([rho]), (np.array([u]), np.array([v]), np.array([w])),
                                          np.array([p]), gamma)
    UR = UL.copy()
    for _ in range(200):
        ut, Ht, c = _roe_average(UL, UR, gamma)
        r1 = np.stack([np.ones_like(c), ut[0] - c, ut[1], ut[2], Ht - ut[0] * c])
        UR_new = UL + strength * r1
        if np.abs(UR_new - UR).max() < 1e-16:
            UR = UR_new
            break
        UR = UR_new
    ut, Ht, c = _roe_average(UL, UR, gamma)
    return UL, UR, ut[0] - c, c


@pytest.mark.parametrize("offset", [0.0, 0.02, -0.03])
def test_harten_fix_on_a_sonic_acoustic_wave(offset):
    # For a jump that is a pure 1-wave (alpha_2 = alpha_5 = 0, no shear), Roe's flux is
    # (F_L + F_R)/2 - |lambda_1|* (U_R - U_L)/2, and with Harten's fix |lambda_1|* =
    # (lambda_1^2 + delta^2)/(2 delta) when |lambda_1| < delta = harten * c~. At the sonic
    # point (lambda_1 = 0) the unfixed flux has no dissipation at all on this wave.
    gamma = 1.4
    UL, UR, lam1, c = _slow_acoustic_pair(gamma, offset, 0.01)
    assert abs(lam1) < 0.05 * c
    dU = UR - UL
    for harten in (0.1, 0.3):
        ns = NavierStokes(NSParams(harten=harten))
        delta = harten * c
        fixed = (lam1 ** 2 + delta ** 2) / (2 * delta)
        assert fixed > abs(lam1)
        expect = 0.5 * (ns.convective_flux(UL, 0) + ns.convective_flux(UR, 0)) - 0.5 * fixed * dU
        assert np.allclose(ns.roe(UL, UR, 0), expect, rtol=0, atol=1e-12)
        # the same wave along a general normal (curved faces) with n = x
        assert np.allclose(ns.roe_normal(UL, UR, [1.0, 0.0, 0.0]), expect, rtol=0, atol=1e-12)
    ns0 = NavierStokes(NSParams(harten=0.0))
    expect0 = 0.5 * (ns0.convective_flux(UL, 0) + ns0.convective_flux(UR, 0)) - 0.5 * abs(lam1) * dU
    assert np.allclose(ns0.roe(UL, UR, 0), expect0, rtol=0, atol=1e-12)


def test_harten_fix_inactive_outside_its_band():
    # |lambda_1| > delta: the fixed and unfixed fluxes are the same Roe flux.
    gamma = 1.4
    UL, UR, lam1, c = _slow_acoustic_pair(gamma, 0.3, 0.01)
    assert abs(lam1) > 0.2 * c
    a = NavierStokes(NSParams(harten=0.1)).roe(UL, UR, 0)
    b = NavierStokes(NSParams(harten=0.0)).roe(UL, UR, 0)
    assert np.array_equal(a, b)


class _HartenDoubled(NavierStokes):
    """Planted mistake: |lambda| -> (lambda^2 + delta^2) / delta, twice the published value."""

    def entropy_fix(self, lam, c):
        delta = self.prm.harten * c
        return np.where(lam < delta, (lam ** 2 + delta ** 2) / delta, lam)


class _HartenOnSquare(NavierStokes):
    """Planted mistake: (lambda^2 - delta^2) / (2 delta), a sign slip in the fixed value."""

    def entropy_fix(self, lam, c):
        delta = self.prm.harten * c
        return np.where(lam < delta, (lam ** 2 - delta ** 2) / (2.0 * delta), lam)


@pytest.mark.parametrize("mutant", [_HartenDoubled, _HartenOnSquare])
def test_harten_pin_catches_planted_mistakes(mutant):
    gamma = 1.4
    UL, UR, lam1, c = _slow_acoustic_pair(gamma, 0.0, 0.01)
    ns = mutant(NSParams(harten=0.1))
    delta = 0.1 * c
    fixed = (lam1 ** 2 + delta ** 2) / (2 * delta)
    expect = 0.5 * (ns.convective_flux(UL, 0) + ns.convective_flux(UR, 0)) - 0.5 * fixed * (UR - UL)
    assert not np.allclose(ns.roe(UL, UR, 0), expect, rtol=0, atol=1e-6)
