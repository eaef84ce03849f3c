"""Pins of the oracle residual against what the paper and the mathematics fix:
exactness on polynomials, conservation, the 3-versus-5 element stencil (Secs. 2.1, 2.2:
the compact stencil spans e-1..e+1, BR1 spans e-2..e+2), separability of the Cartesian
operator, free-stream preservation, symmetries, and closed-form NS responses."""
import itertools

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.physics import Heat, NavierStokes, NSParams, PorousMedium
from oracle.residual import residual
from paper_2608_09615_b300 import inputs

SCHEMES = ("br1", "compact")


# ---------------------------------------------------------------- polynomial exactness
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_heat_exact_on_polynomials_1d(scheme, p):
    # Continuous data => every interface correction vanishes (Sec. 2.1) and the residual
    # of u_t = nu u_xx is exact for degree <= p away from the periodic seam.
    rng = np.random.default_rng(p)
    g = Grid(1, (8,), (-4.0,), (4.0,), p)
    (x,) = g.coordinates()
    c = rng.uniform(-1, 1, p + 1)
    u = sum(c[k] * x ** k for k in range(p + 1))
    d2 = sum(c[k] * k * (k - 1) * x ** (k - 2) for k in range(2, p + 1)) if p >= 2 else 0 * x
    nu = 0.7
    R = residual(u[None], g, scheme, Heat(nu))[0]
    # elements 2..5 do not see the seam between elements 7 and 0
    assert np.allclose(R[2:6], nu * d2[2:6], atol=1e-10 * 4 ** p)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("p", [2, 3])
def test_heat_exact_on_polynomials_3d(scheme, p):
    rng = np.random.default_rng(10 + p)
    g = Grid(3, (6, 6, 6), (-3.0,) * 3, (3.0,) * 3, p)
    X = g.coordinates()
    u = np.zeros_like(X[0])
    lap = np.zeros_like(X[0])
    for a, b, cc in itertools.product(range(p + 1), repeat=3):
        if a + b + cc > p + 1:
            continue
        k = rng.uniform(-1, 1)
        u += k * X[0] ** a * X[1] ** b * X[2] ** cc
        if a >= 2:
            lap += k * a * (a - 1) * X[0] ** (a - 2) * X[1] ** b * X[2] ** cc
        if b >= 2:
            lap += k * b * (b - 1) * X[0] ** a * X[1] ** (b - 2) * X[2] ** cc
        if cc >= 2:
            lap += k * cc * (cc - 1) * X[0] ** a * X[1] ** b * X[2] ** (cc - 2)
    R = residual(u[None], g, scheme, Heat(1.0))[0]
    sl = (slice(2, 4),) * 3
    assert np.allclose(R[sl], lap[sl], atol=1e-10 * 3 ** (p + 1))


# ------------------------------------------------------------------------ conservation
def _total(R, g):
    W = g.quadrature_weights()
    return np.array([np.sum(W * R[v]) for v in range(R.shape[0])]), \
        np.array([np.sum(W * np.abs(R[v])) for v in range(R.shape[0])])


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dim", [1, 3])
def test_conservation_heat_pme(scheme, dim):
    # Periodic grid: the Gauss-weighted sum of the residual is zero to round-off
    # (M G has degree n-1, integrated exactly, and interface fluxes telescope).
    ne = (16,) if dim == 1 else (3, 4, 5)
    g = Grid(dim, ne, (0.0,) * dim, (1.0,) * dim, 3)
    U = inputs.random_scalar(dim, ne, 3, seed=3, lo=0.1, hi=1.0)
    for phys in (Heat(0.3), PorousMedium(2.0), PorousMedium(5.0)):
        tot, scale = _total(residual(U, g, scheme, phys), g)
        assert np.all(np.abs(tot) <= 1e-13 * scale)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
def test_conservation_ns(scheme, riemann):
    ne = (3, 4, 3)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, 2)
    U = inputs.random_state(ne, 2, seed=5)
    phys = NavierStokes(NSParams(riemann=riemann, Re=100.0))
    tot, scale = _total(residual(U, g, scheme, phys), g)
    assert np.all(np.abs(tot) <= 1e-13 * scale)


# ---------------------------------------------------------------------------- stencil
def _changed_elements(g, phys, scheme, U, centre, dim):
    R0 = residual(U, g, scheme, phys)
    V = U.copy()
    rng = np.random.default_rng(1)
    idx = (slice(None),) + tuple(reversed(centre))
    V[idx] += 1e-3 * rng.uniform(-1, 1, V[idx].shape)
    R1 = residual(V, g, scheme, phys)
    diff = np.abs(R1 - R0)
    axes = tuple([0] + list(range(1 + dim, 1 + 2 * dim)))
    changed = np.argwhere(diff.max(axis=axes) > 0)
    return {tuple(int(v) - c for v, c in zip(reversed(row), centre)) for row in changed}


@pytest.mark.parametrize("scheme,expected", [("compact", {-1, 0, 1}), ("br1", {-2, -1, 0, 1, 2})])
def test_stencil_1d(scheme, expected):
    # Sec. 2.1: BR1 couples e-2..e+2; Sec. 2.2: the compact scheme couples e-1..e+1.
    g = Grid(1, (9,), (0.0,), (1.0,), 3)
    U = inputs.random_scalar(1, (9,), 3, seed=2)
    got = _changed_elements(g, Heat(1.0), scheme, U, (4,), 1)
    assert {d[0] for d in got} == expected
    got = _changed_elements(g, PorousMedium(2.0), scheme, np.abs(U) + 0.1, (4,), 1)
    assert {d[0] for d in got} == expected


def _ball(dim, linf, l1):
    return {d for d in itertools.product(range(-2, 3), repeat=dim)
            if max(abs(v) for v in d) <= linf and sum(abs(v) for v in d) <= l1}


@pytest.mark.parametrize("scheme", SCHEMES)
def test_stencil_3d_heat(scheme):
    # Linear diffusion on a Cartesian grid is a sum of 1D operators: the element
    # stencil is the centre plus the 1D stencil along each axis (7 compact, 13 BR1).
    g = Grid(3, (5, 5, 5), (0.0,) * 3, (1.0,) * 3, 2)
    U = inputs.random_scalar(3, (5, 5, 5), 2, seed=4)
    got = _changed_elements(g, Heat(1.0), scheme, U, (2, 2, 2), 3)
    expect = {d for d in _ball(3, 2, 2) if sum(1 for v in d if v != 0) <= 1}
    if scheme == "compact":
        expect = {d for d in expect if max(abs(v) for v in d) <= 1}
    assert got == expect
    assert len(got) == (7 if scheme == "compact" else 13)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_stencil_3d_ns(scheme):
    # NS couples the gradient components across directions: the compact scheme reaches
    # the elements with max|d| <= 1 and |d|_1 <= 2 (19), BR1 those with |d|_1 <= 2 (25).
    ne = (5, 5, 5)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, 1)
    U = inputs.random_state(ne, 1, seed=6)
    got = _changed_elements(g, NavierStokes(NSParams(Re=50.0)), scheme, U, (2, 2, 2), 3)
    expect = _ball(3, 1 if scheme == "compact" else 2, 2)
    assert got == expect
    assert len(got) == (19 if scheme == "compact" else 25)


# ------------------------------------------------------------------------ separability
@pytest.mark.parametrize("scheme", SCHEMES)
def test_heat_3d_is_kronecker_sum_of_1d(scheme):
    rng = np.random.default_rng(7)
    p = 3
    ne = (4, 3, 5)
    g3 = Grid(3, ne, (0.0,) * 3, (1.0, 2.0, 1.5), p)
    g1 = [Grid(1, (ne[d],), (0.0,), ((1.0, 2.0, 1.5)[d],), p) for d in range(3)]
    f = [rng.uniform(-1, 1, (ne[d], p + 1)) for d in range(3)]
    # u(x, y, z) = f0(x) f1(y) f2(z) in the layout U[ez][ey][ex][k][j][i]
    u = np.einsum("ck,bj,ai->cbakji", f[2], f[1], f[0])
    R = residual(u[None], g3, scheme, Heat(1.0))[0]
    r = [residual(f[d][None], g1[d], scheme, Heat(1.0))[0] for d in range(3)]
    expect = (np.einsum("ck,bj,ai->cbakji", f[2], f[1], r[0])
              + np.einsum("ck,bj,ai->cbakji", f[2], r[1], f[0])
              + np.einsum("ck,bj,ai->cbakji", r[2], f[1], f[0]))
    assert np.allclose(R, expect, atol=1e-11 * np.abs(expect).max())


# ------------------------------------------------------------------ Navier-Stokes pins
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
def test_ns_free_stream(scheme, riemann):
    ne = (3, 3, 2)
    g = Grid(3, ne, (0.0,) * 3, (1.0, 1.3, 0.7), 3)
    shp = g.shape(1)[1:]
    rho = 1.2 * np.ones(shp)
    vel = [0.3 * np.ones(shp), -0.2 * np.ones(shp), 0.1 * np.ones(shp)]
    U = inputs.primitive_to_conservative(rho, vel, 50.0 * np.ones(shp), 1.4)
    R = residual(U, g, scheme, NavierStokes(NSParams(riemann=riemann)))
    assert np.abs(R).max() < 1e-11


def _swap_xy(A):
    # U[v][ez][ey][ex][k][j][i] -> exchange the x and y roles
    B = np.swapaxes(np.swapaxes(A, 2, 3), 5, 6)
    B = B.copy()
    if B.shape[0] == 5:
        B[[1, 2]] = B[[2, 1]]
    return B


def _reflect_x(A):
    B = A[:, :, :, ::-1, :, :, ::-1].copy()
    if B.shape[0] == 5:
        B[1] = -B[1]
    return B


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ns_axis_exchange_symmetry(scheme):
    # Exchanging x and y (and the u, v momenta) commutes with the residual: catches
    # transposed operands and misplaced direction indices.
    ne = (3, 3, 2)
    g = Grid(3, ne, (0.0,) * 3, (1.0, 1.0, 0.8), 2)
    U = inputs.random_state(ne, 2, seed=8)
    phys = NavierStokes(NSParams(Re=200.0))
    R = residual(U, g, scheme, phys)
    Rs = residual(_swap_xy(U), g, scheme, phys)
    assert np.allclose(Rs, _swap_xy(R), atol=1e-11 * np.abs(R).max())


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ns_reflection_symmetry(scheme):
    ne = (3, 2, 2)
    g = Grid(3, ne, (0.0,) * 3, (1.0, 1.0, 0.8), 2)
    U = inputs.random_state(ne, 2, seed=9)
    phys = NavierStokes(NSParams(Re=200.0))
    R = residual(U, g, scheme, phys)
    Rr = residual(_reflect_x(U), g, scheme, phys)
    assert np.allclose(Rr, _reflect_x(R), atol=1e-11 * np.abs(R).max())


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ns_heat_conduction_closed_form(scheme):
    # Fluid at rest, uniform pressure, density varying along x: the only nonzero
    # residual is the energy equation, d(rho E)/dt = div(kappa grad T) =
    # (mu gamma / Pr) e'' with e = p / ((gamma-1) rho) (constant mu). Fixes the sign and
    # size of the heat-conduction term (Sec. 4.4).
    prm = NSParams(Re=10.0, sutherland=False)
    ne = (12, 1, 1)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi, 1.0, 1.0), 5)
    X = g.coordinates()
    eps = 0.1
    rho = prm.rho0 * (1 + eps * np.sin(X[0]))
    zero = np.zeros_like(rho)
    U = inputs.primitive_to_conservative(rho, (zero, zero, zero), prm.p0 + zero, prm.gamma)
    R = residual(U, g, scheme, NavierStokes(prm))
    e0 = prm.e0
    s, c = np.sin(X[0]), np.cos(X[0])
    # e = e0 / (1 + eps s): e'' = e0 (eps s (1+eps s) + 2 eps^2 c^2) / (1+eps s)^3
    epp = e0 * (eps * s * (1 + eps * s) + 2 * eps ** 2 * c ** 2) / (1 + eps * s) ** 3
    expect = prm.mu0 * prm.gamma / prm.Pr * epp
    assert np.abs(R[:4]).max() < 1e-9 * np.abs(expect).max()
    assert np.abs(R[4] - expect).max() < 2e-3 * np.abs(expect).max()


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
def test_ns_entropy_wave_closed_form(scheme, riemann):
    # Uniform velocity and pressure, density wave: an inviscid entropy wave travels
    # with the flow, rho_t = -U0 rho_x, (rho u)_t = -U0^2 rho_x, (rho E)_t = -U0^3 rho_x / 2.
    prm = NSParams(Re=1e14, riemann=riemann)
    ne = (12, 1, 1)
    g = Grid(3, ne, (0.0,) * 3, (2 * np.pi, 1.0, 1.0), 5)
    X = g.coordinates()
    U0 = 0.4
    eps = 0.05
    rho = prm.rho0 * (1 + eps * np.sin(X[0]))
    rhox = prm.rho0 * eps * np.cos(X[0])
    zero = np.zeros_like(rho)
    U = inputs.primitive_to_conservative(rho, (U0 + zero, zero, zero), prm.p0 + zero, prm.gamma)
    R = residual(U, g, scheme, NavierStokes(prm))
    scale = np.abs(rhox).max() * U0
    assert np.abs(R[0] + U0 * rhox).max() < 1e-5 * scale
    assert np.abs(R[1] + U0 ** 2 * rhox).max() < 1e-5 * scale
    assert np.abs(R[2]).max() < 1e-9 * scale and np.abs(R[3]).max() < 1e-9 * scale
    assert np.abs(R[4] + 0.5 * U0 ** 3 * rhox).max() < 1e-4 * scale


def test_roe_flux_textbook_properties():
    # Consistency F(U, U) = F(U); the Roe property F(U_R) - F(U_L) = A~ (U_R - U_L)
    # gives pure upwinding for a supersonic pair (Harten fix inactive there).
    phys = NavierStokes(NSParams(harten=0.0))
    rng = np.random.default_rng(3)
    shp = (7,)
    rho = rng.uniform(0.5, 2, shp)
    vel = [rng.uniform(-1, 1, shp) for _ in range(3)]
    pr = rng.uniform(0.5, 2, shp)
    UL = inputs.primitive_to_conservative(rho, vel, pr, 1.4)
    for m in range(3):
        assert np.allclose(phys.roe(UL, UL, m), phys.convective_flux(UL, m), atol=1e-13)
    rho2 = rng.uniform(0.5, 2, shp)
    vel_sup = [5.0 + rng.uniform(0, 1, shp), rng.uniform(-1, 1, shp), rng.uniform(-1, 1, shp)]
    vel_sup2 = [5.0 + rng.uniform(0, 1, shp), rng.uniform(-1, 1, shp), rng.uniform(-1, 1, shp)]
    A = inputs.primitive_to_conservative(rho, vel_sup, pr, 1.4)
    B = inputs.primitive_to_conservative(rho2, vel_sup2, rng.uniform(0.5, 2, shp), 1.4)
    assert np.allclose(phys.roe(A, B, 0), phys.convective_flux(A, 0), rtol=1e-12, atol=1e-12)
    assert np.allclose(phys.roe(A * np.array([1, -1, -1, -1, 1])[:, None],
                                B * np.array([1, -1, -1, -1, 1])[:, None], 0),
                       phys.convective_flux(B * np.array([1, -1, -1, -1, 1])[:, None], 0),
                       rtol=1e-12, atol=1e-12)


def test_roe_resolves_stationary_contact_exactly():
    # A density jump at rest with equal pressures: the Roe solver puts no dissipation on the
    # contact wave (its speed is zero) and none on the acoustic waves (their strengths
    # vanish), so the flux is the exact (0, p n, 0); with or without the entropy fix, along an
    # axis and along a general normal.
    rng = np.random.default_rng(5)
    shp = (6,)
    pr = rng.uniform(0.5, 2, shp)
    zero = [np.zeros(shp)] * 3
    UL = inputs.primitive_to_conservative(rng.uniform(0.5, 2, shp), zero, pr, 1.4)
    UR = inputs.primitive_to_conservative(rng.uniform(0.5, 2, shp), zero, pr, 1.4)
    nv = np.array([0.3, -0.5, 0.8])
    nv = nv / np.linalg.norm(nv)
    for harten in (0.0, 0.1):
        phys = NavierStokes(NSParams(harten=harten))
        for m in range(3):
            F = phys.roe(UL, UR, m)
            expect = np.zeros_like(F)
            expect[1 + m] = pr
            assert np.allclose(F, expect, rtol=1e-13, atol=1e-13)
        F = phys.roe_normal(UL, UR, list(nv))
        expect = np.zeros_like(F)
        for i in range(3):
            expect[1 + i] = pr * nv[i]
        assert np.allclose(F, expect, rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------- extended precision
@pytest.mark.parametrize("scheme", SCHEMES)
def test_extended_precision_evaluation_agrees(scheme):
    # The same definition evaluated in np.longdouble (x86 80-bit) agrees with the float64
    # evaluation to the float64 round-off, and its operators are exact to ~1e-18.
    from oracle.operators import operators
    o = operators(5, np.longdouble)
    assert np.abs(o.M.sum(axis=1)).max() < 1e-17
    assert np.abs(o.L.sum(axis=1) - 1).max() < 1e-18
    ne, p = (3, 2, 3), 4
    U = inputs.tgv_3d(ne, p, perturb_seed=5)
    phys = NavierStokes(NSParams())
    R64 = residual(U, Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, p), scheme, phys)
    R80 = residual(U, Grid(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, p, dtype=np.longdouble), scheme, phys)
    assert R80.dtype == np.longdouble
    for v in range(5):
        assert np.abs(R64[v] - R80[v]).max() < 1e-10 * np.abs(R80[v]).max()
    g = Grid(1, (8,), (-4.0,), (4.0,), 3, dtype=np.longdouble)
    (x,) = g.coordinates()
    u = x ** 3 - 0.5 * x
    R = residual(u[None], g, scheme, Heat(1.0))[0]
    assert np.abs(R[2:6] - 6 * x[2:6]).max() < 1e-15
