"""Pins of the closure data definitions (oracle/closure.py): projection exactness and
conservation, vanishing sub-grid flux where the filter loses nothing, conservative
injection, and closed-form features."""
import numpy as np
import pytest

from oracle.closure import features, project, projection_matrix, sgs_target
from oracle.grid import Grid
from oracle.physics import NavierStokes, NSParams
from oracle.residual import residual
from paper_2608_09615_b300 import inputs

TWO_PI = 2 * np.pi


def _grids(nf=8, nc=2, pf=4, pc=3):
    return (Grid(3, (nf,) * 3, (0.0,) * 3, (TWO_PI,) * 3, pf),
            Grid(3, (nc,) * 3, (0.0,) * 3, (TWO_PI,) * 3, pc))


def test_projection_exact_and_conservative():
    gf, gc = _grids()
    X = gf.coordinates()
    f = lambda x, y, z: 1 + x - 0.3 * y ** 2 + x * z ** 3 / 40 + (x * y * z) / 7  # noqa: E731
    uc = project(f(*X)[None], gf, gc)[0]
    Xc = gc.coordinates()
    assert np.abs(uc - f(*Xc)).max() < 1e-12 * np.abs(f(*Xc)).max()
    U = inputs.tgv_3d((8, 8, 8), 4, perturb_seed=3)
    Uc = project(U, gf, gc)
    for v in range(5):
        assert gc.integrate(Uc[v]) == pytest.approx(gf.integrate(U[v]), rel=1e-13)
    # the rows of the 1D projection sum to one (constants are reproduced)
    P = projection_matrix(4, 3, 4)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)


def test_sgs_target_vanishes_without_subfilter_content():
    gf, gc = _grids()
    phys = NavierStokes(NSParams())
    shp = gf.shape(1)[1:]
    one = np.ones(shp)
    U = inputs.primitive_to_conservative(1.1 * one, (0.3 * one, -0.2 * one, 0.1 * one), 70.0 * one, 1.4)
    tau, _ = sgs_target(U, gf, gc, phys)
    assert np.abs(tau).max() < 1e-11
    # the mass flux is linear in U: its sub-grid part vanishes for any field
    U = inputs.tgv_3d((8, 8, 8), 4, perturb_seed=1)
    tau, _ = sgs_target(U, gf, gc, phys)
    assert np.abs(tau[0]).max() < 1e-13
    assert np.abs(tau[1:]).max() > 1e-6


def test_injection_is_conservative_and_acts_through_jumps():
    ne, p = (3, 2, 3), 3
    g = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p)
    phys = NavierStokes(NSParams())
    U = inputs.tgv_3d(ne, p, perturb_seed=2)
    R0 = residual(U, g, "compact", phys)
    rng = np.random.default_rng(0)
    tau = rng.normal(size=(5,) + tuple(reversed(ne)) + (3,))
    R1 = residual(U, g, "compact", phys, tau=tau)
    W = g.quadrature_weights()
    for v in range(5):
        assert abs(np.sum(W * (R1[v] - R0[v]))) < 1e-12 * np.sum(W * np.abs(R1[v] - R0[v]))
    # a tau that is the same in every element has zero divergence
    uni = np.broadcast_to(rng.normal(size=(5, 1, 1, 1, 3)), tau.shape).copy()
    R2 = residual(U, g, "compact", phys, tau=uni)
    assert np.abs(R2 - R0).max() < 1e-9 * np.abs(R0).max()


def test_features_closed_forms():
    gc = Grid(3, (2, 2, 2), (0.0,) * 3, (TWO_PI,) * 3, 3)
    prm = NSParams(Re=1600.0)
    phys = NavierStokes(prm)
    X = gc.coordinates()
    shp = X[0].shape
    one = np.ones(shp)
    # uniform state: means only, everything else zero
    U = inputs.primitive_to_conservative(1.05 * one, (0.2 * one, 0.0 * one, -0.1 * one), prm.p0 * one, prm.gamma)
    F = features(U, gc, phys)
    assert np.allclose(F[:, 0], 0.05, atol=1e-12)
    assert np.allclose(F[:, 1], 1.05 * 0.2, atol=1e-12)
    assert np.allclose(F[:, 5:47], 0.0, atol=1e-9)
    assert np.allclose(F[:, 47:63], 0.0, atol=1e-12)
    assert np.allclose(F[:, 63], 1000.0 / 1600.0)
    # density linear in x inside each element: rho = 1 + b xi_x, velocity zero
    h = TWO_PI / 2
    xi = ((X[0] % h) / (h / 2)) - 1.0
    b = 0.01
    U = inputs.primitive_to_conservative(1.0 + b * xi, (0 * one, 0 * one, 0 * one), prm.p0 * one, prm.gamma)
    F = features(U, gc, phys)
    assert np.allclose(F[:, 5 + 0], b, atol=1e-12)            # linear moment of rho along x
    assert np.allclose(F[:, 52], b * b / 3.0, atol=1e-14)      # variance of rho
    assert np.allclose(F[:, 47], 0.0, atol=1e-12)              # no energy in degree-3 modes
