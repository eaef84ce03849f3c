"""Pins of the curvilinear-grid oracle (Sec. 2 mapping with K = 8 corner nodes, Eqs.
ns:mapped and adj:f, the steps of Sec. 2.3 with per-point metric terms) against what the
paper and the mathematics fix:
  * an undeformed lattice gives the Cartesian oracle's residual (itself pinned);
  * a rigid rotation of grid and field rotates the residual (the equations are
    rotation invariant), which exercises every off-diagonal metric term, the Riemann
    solver along a general normal and the full viscous tensor;
  * the discrete metric identities (the footnote to Eq. ns:mapped) and free-stream
    preservation hold on jittered grids;
  * for u_t = nu lap u and quadratic u, the residual is exactly nu lap u (a constant) on
    jittered trilinear grids when p >= 3 (the fluxes H = u S are then polynomials the
    flux points resolve), and 0 for linear u when p >= 2;
  * conservation, the element stencil of the two schemes (Secs. 2.1-2.3: the compact
    scheme stays within one element per axis), the domain volume, and the scaling of
    the residual (with interior penalty) under a uniform dilation of the grid;
  * the volume diagnostics of the Taylor-Green field on a curved grid against their
    closed forms (Sec. 4.4);
  * the truncation error of the discrete Laplacian on a smooth periodic field converges on
    a curved grid at the rate it has on the Cartesian grid.
"""
import itertools
import math

import numpy as np
import pytest

from oracle.curvilinear import CurvGrid, ns_diagnostics as curv_ns_diagnostics
from oracle.curvilinear import residual as curv_residual
from oracle.grid import Grid
from oracle.physics import Heat, NavierStokes, NSParams, PorousMedium
from oracle.residual import along, residual
from paper_2608_09615_b300 import inputs

SCHEMES = ("br1", "compact")
BOX = ((0.0,) * 3, (2 * math.pi,) * 3)


def _rel(a, b):
    return max(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max() for v in range(a.shape[0]))


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("eta_ip,viscous", [(0.0, "a"), (0.5, "a"), (0.0, "b"), (0.5, "b")])
def test_undeformed_lattice_equals_cartesian_ns(scheme, eta_ip, viscous):
    ne, p = (3, 2, 2), 3
    lo, hi = (0.0, -1.0, 0.5), (2 * math.pi, 3.0, 4.0)
    U = inputs.random_state(ne, p, seed=1)
    phys = NavierStokes(NSParams())
    a = residual(U, Grid(3, ne, lo, hi, p), scheme, phys, eta_ip=eta_ip, viscous=viscous)
    b = curv_residual(U, CurvGrid(inputs.periodic_lattice(ne, lo, hi), p), scheme, phys,
                      eta_ip=eta_ip, viscous=viscous)
    assert _rel(b, a) <= 1e-13


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("phys", [Heat(0.7), PorousMedium(2.0)], ids=["heat", "pme"])
def test_undeformed_lattice_equals_cartesian_scalar(scheme, phys):
    ne, p = (3, 4, 2), 2
    lo, hi = (0.0, 0.0, 0.0), (1.0, 2.0, 1.5)
    U = np.abs(inputs.random_scalar(3, ne, p, seed=3)) + 0.1
    for eta in (0.0, 1.0):
        a = residual(U, Grid(3, ne, lo, hi, p), scheme, phys, eta_ip=eta)
        b = curv_residual(U, CurvGrid(inputs.periodic_lattice(ne, lo, hi), p), scheme, phys, eta_ip=eta)
        assert _rel(b, a) <= 1e-13


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
def test_rotation_equivariance_ns(scheme, riemann):
    ne, p = (3, 3, 2), 2
    N0 = inputs.jittered_lattice(ne, *BOX, seed=3, amp=0.12)
    Rm = inputs.rotation_matrix((1.0, 2.0, 3.0), 0.7)
    N1 = np.einsum("ij,jzyx->izyx", Rm, N0)
    U = inputs.random_state(ne, p, seed=2)
    U1 = U.copy()
    U1[1:4] = np.einsum("ij,j...->i...", Rm, U[1:4])
    phys = NavierStokes(NSParams(riemann=riemann, Re=200.0))
    for eta, vis in ((0.0, "a"), (0.3, "a"), (0.3, "b")):
        a = curv_residual(U, CurvGrid(N0, p), scheme, phys, eta_ip=eta, viscous=vis)
        b = curv_residual(U1, CurvGrid(N1, p), scheme, phys, eta_ip=eta, viscous=vis)
        a[1:4] = np.einsum("ij,j...->i...", Rm, a[1:4])
        assert _rel(b, a) <= 1e-12


@pytest.mark.parametrize("scheme", SCHEMES)
def test_rotation_invariance_heat(scheme):
    ne, p = (3, 2, 3), 3
    N0 = inputs.wavy_lattice(ne, *BOX, amp=0.15)
    N1 = np.einsum("ij,jzyx->izyx", inputs.rotation_matrix((0.0, 1.0, 1.0), -1.1), N0)
    U = inputs.random_scalar(3, ne, p, seed=8)
    a = curv_residual(U, CurvGrid(N0, p), scheme, Heat(1.0), eta_ip=0.7)
    b = curv_residual(U, CurvGrid(N1, p), scheme, Heat(1.0), eta_ip=0.7)
    assert _rel(b, a) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 4])
def test_metric_identities_and_volume(p):
    ne = (3, 4, 2)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 2.0, 0.5)
    g = CurvGrid(inputs.jittered_lattice(ne, lo, hi, seed=p, amp=0.15), p)
    # sum_d d/dxi_d S_dm = 0 at the solution points, with the discrete derivative M
    for m in range(3):
        acc = sum(along(g.ops.M, g.Sf[d][m], 3 + (2 - d)) for d in range(3))
        assert np.abs(acc).max() <= 1e-13
    # the trilinear elements tile the periodic box exactly
    assert abs(g.volume.sum() - 1.0) <= 1e-13
    assert abs(np.sum(g.quadrature_weights()) - 1.0) <= 1e-13


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
def test_free_stream_preserved_on_jittered_grid(scheme, riemann):
    g = CurvGrid(inputs.jittered_lattice((3, 3, 3), *BOX, seed=5, amp=0.12), 3)
    rho, vel, pr = 1.2, (0.3, -0.2, 0.5), 71.4
    U = np.zeros(g.shape(5))
    U[0] = rho
    for i in range(3):
        U[1 + i] = rho * vel[i]
    U[4] = pr / 0.4 + 0.5 * rho * sum(v * v for v in vel)
    R = curv_residual(U, g, scheme, NavierStokes(NSParams(riemann=riemann)), eta_ip=0.5)
    # each flux is O(p) ~ 70; the residual vanishes to round-off
    assert np.abs(R).max() <= 1e-11


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("lattice", ["jitter", "wavy"])
def test_heat_exact_on_quadratics_jittered(scheme, lattice):
    ne, p = (6, 6, 6), 3
    lo, hi = (-3.0,) * 3, (3.0,) * 3
    nodes = (inputs.jittered_lattice(ne, lo, hi, seed=7, amp=0.12) if lattice == "jitter"
             else inputs.wavy_lattice(ne, lo, hi, amp=0.15))
    g = CurvGrid(nodes, p)
    X = g.coordinates()
    rng = np.random.default_rng(1)
    A = rng.uniform(-1, 1, (3, 3))
    A = A + A.T
    b = rng.uniform(-1, 1, 3)
    u = sum(A[i, j] * X[i] * X[j] for i in range(3) for j in range(3)) + sum(b[i] * X[i] for i in range(3))
    nu = 0.7
    R = curv_residual(u[None], g, scheme, Heat(nu), eta_ip=0.5)[0]
    sl = (slice(2, 4),) * 3                      # elements the periodic seam cannot reach
    assert np.abs(R[sl] - nu * 2.0 * np.trace(A)).max() <= 1e-11


@pytest.mark.parametrize("scheme", SCHEMES)
def test_heat_zero_on_linear_fields_p2(scheme):
    ne, p = (6, 6, 6), 2
    g = CurvGrid(inputs.jittered_lattice(ne, (-3.0,) * 3, (3.0,) * 3, seed=2, amp=0.12), p)
    X = g.coordinates()
    u = 0.3 * X[0] - 1.1 * X[1] + 0.7 * X[2] + 2.0
    R = curv_residual(u[None], g, scheme, Heat(1.3))[0]
    assert np.abs(R[(slice(2, 4),) * 3]).max() <= 1e-12


def _total(R, g):
    W = g.quadrature_weights()
    return np.array([np.sum(W * R[v]) for v in range(R.shape[0])]), \
        np.array([np.sum(W * np.abs(R[v])) for v in range(R.shape[0])])


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("viscous", ["a", "b"])
def test_conservation_jittered(scheme, viscous):
    ne, p = (3, 3, 3), 2
    g = CurvGrid(inputs.jittered_lattice(ne, *BOX, seed=9, amp=0.12), p)
    U = inputs.random_state(ne, p, seed=4)
    tot, scale = _total(curv_residual(U, g, scheme, NavierStokes(NSParams(Re=100.0)), eta_ip=0.4,
                                      viscous=viscous), g)
    assert np.all(np.abs(tot) <= 1e-13 * scale)
    U = inputs.random_scalar(3, ne, p, seed=5)
    tot, scale = _total(curv_residual(U, g, scheme, Heat(1.0), eta_ip=0.4), g)
    assert abs(tot[0]) <= 1e-13 * scale[0]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_stencil_jittered(scheme):
    # with a non-diagonal metric even linear diffusion couples the directions: the
    # compact scheme reaches max|d| <= 1, |d|_1 <= 2 (19 elements), BR1 |d|_1 <= 2 (25)
    ne = (5, 5, 5)
    g = CurvGrid(inputs.jittered_lattice(ne, (0.0,) * 3, (1.0,) * 3, seed=11, amp=0.12), 2)
    U = inputs.random_scalar(3, ne, 2, seed=4)
    R0 = curv_residual(U, g, scheme, Heat(1.0))
    V = U.copy()
    V[:, 2, 2, 2] += 1e-3 * np.random.default_rng(1).uniform(-1, 1, V[:, 2, 2, 2].shape)
    diff = np.abs(curv_residual(V, g, scheme, Heat(1.0)) - R0)
    got = {tuple(int(v) - 2 for v in reversed(r)) for r in np.argwhere(diff.max(axis=(0, 4, 5, 6)) > 0)}
    expect = {d for d in itertools.product(range(-2, 3), repeat=3)
              if sum(abs(v) for v in d) <= 2 and max(abs(v) for v in d) <= (1 if scheme == "compact" else 2)}
    assert got == expect
    assert len(got) == (19 if scheme == "compact" else 25)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_dilation_scaling_with_penalty(scheme):
    # u_t = lap u: dilating the grid by s (same nodal values) divides the residual by s^2;
    # the penalty scale 1/h = |A_f| / V must scale as 1/s for this to hold
    ne, p, s = (3, 3, 3), 2, 2.5
    N = inputs.jittered_lattice(ne, *BOX, seed=13, amp=0.12)
    U = inputs.random_scalar(3, ne, p, seed=6)
    a = curv_residual(U, CurvGrid(N, p), scheme, Heat(1.0), eta_ip=1.0)
    b = curv_residual(U, CurvGrid(s * N, p), scheme, Heat(1.0), eta_ip=1.0)
    assert _rel(b * s * s, a) <= 1e-12


def test_penalty_changes_jittered_residual():
    # the penalty is not silently dropped on curved faces
    ne, p = (3, 3, 3), 2
    g = CurvGrid(inputs.jittered_lattice(ne, *BOX, seed=13, amp=0.12), p)
    U = inputs.random_scalar(3, ne, p, seed=6)
    a = curv_residual(U, g, "compact", Heat(1.0), eta_ip=0.0)
    b = curv_residual(U, g, "compact", Heat(1.0), eta_ip=1.0)
    assert _rel(b, a) > 1e-3


def test_roe_normal_reduces_to_axis_solver_and_rotates():
    rng = np.random.default_rng(3)
    phys = NavierStokes(NSParams())
    shp = (7,)
    UL = inputs.primitive_to_conservative(1 + 0.1 * rng.uniform(-1, 1, shp),
                                          [rng.uniform(-1, 1, shp) for _ in range(3)],
                                          71.4 * (1 + 0.1 * rng.uniform(-1, 1, shp)), 1.4)
    UR = inputs.primitive_to_conservative(1 + 0.1 * rng.uniform(-1, 1, shp),
                                          [rng.uniform(-1, 1, shp) for _ in range(3)],
                                          71.4 * (1 + 0.1 * rng.uniform(-1, 1, shp)), 1.4)
    for m in range(3):
        e = [1.0 if i == m else 0.0 for i in range(3)]
        assert np.allclose(phys.roe_normal(UL, UR, e), phys.roe(UL, UR, m), rtol=1e-14, atol=1e-13)
    # rotation: F(R UL, R UR; R n) = R F(UL, UR; n) on the momentum rows
    Rm = inputs.rotation_matrix((0.3, -0.5, 1.0), 0.9)
    nv = np.array([0.2, -0.6, 0.3])
    nv = nv / np.linalg.norm(nv)
    F = phys.roe_normal(UL, UR, list(nv))
    rot = lambda U: np.concatenate([U[:1], Rm @ U[1:4], U[4:]])
    G = phys.roe_normal(rot(UL), rot(UR), list(Rm @ nv))
    assert np.allclose(G, rot(F), rtol=1e-13, atol=1e-12)
    # consistency: equal states give the physical normal flux
    assert np.allclose(phys.roe_normal(UL, UL, list(nv)), phys.normal_flux(UL, list(nv)), rtol=1e-14, atol=1e-12)


def test_diagnostics_taylor_green_closed_forms_on_wavy_grid():
    # The Taylor-Green field of Sec. 4.4 sampled on a curved grid: E_k / |Omega| = u0^2 / 8
    # and enstrophy / |Omega| = 3/4 (u0 / L)^2 up to the discretisation error, the domain
    # volume exactly, and zero net momentum.
    ne, p = (8, 8, 8), 4
    N = inputs.wavy_lattice(ne, *BOX, amp=0.15)
    U = inputs.tgv_3d(ne, p, X=inputs.curvilinear_coordinates(N, p))
    d = curv_ns_diagnostics(U, CurvGrid(N, p))
    vol = (2 * math.pi) ** 3
    assert abs(d["volume"] - vol) <= 1e-12 * vol
    assert abs(d["ke"] / vol - 0.125) <= 2e-4
    assert abs(d["enstrophy"] / vol - 0.75) <= 2e-2
    for i in range(3):
        assert abs(d["mom"][i]) <= 1e-10 * vol


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("p", [2, 3])
def test_truncation_error_converges_like_the_cartesian_grid(scheme, p):
    # R(u) - nu lap u for a smooth periodic u: the discrete Laplacian's truncation error.
    # On the wavy grid it converges at the Cartesian grid's rate (p - 1 for this pointwise
    # second-derivative error) and stays within 1.5 times the Cartesian error.
    def err(nodes=None, ne=None):
        if nodes is not None:
            g = CurvGrid(nodes, p)
            X = g.coordinates()
        else:
            g = Grid(3, (ne,) * 3, *BOX, p)
            X = g.coordinates()
        u = np.sin(X[0] + 0.3) * np.sin(2 * X[1] + 0.1) * np.cos(X[2])
        R = (curv_residual if nodes is not None else residual)(u[None], g, scheme, Heat(1.0))[0]
        W = g.quadrature_weights()
        return math.sqrt(np.sum(W * (R + 6.0 * u) ** 2) / np.sum(W))

    curved = [err(nodes=inputs.wavy_lattice((ne,) * 3, *BOX, amp=0.15)) for ne in (6, 12)]
    cart = [err(ne=ne) for ne in (6, 12)]
    rate_curved = math.log(curved[0] / curved[1]) / math.log(2.0)
    rate_cart = math.log(cart[0] / cart[1]) / math.log(2.0)
    assert rate_curved >= p - 1 - 0.15, (curved, rate_curved)
    assert abs(rate_curved - rate_cart) <= 0.25, (rate_curved, rate_cart)
    assert curved[1] <= 1.5 * cart[1], (curved, cart)
