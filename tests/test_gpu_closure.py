"""GPU closure data kernels against the oracle's closure definitions (FP64 contexts):
box filter, per-element flux means, sub-grid flux targets, the 64 features, and the
per-element flux injection in the residual."""
import math

import numpy as np
import pytest

from oracle.closure import features as o_features
from oracle.closure import point_fluxes, project, sgs_target
from oracle.grid import Grid
from oracle.physics import NavierStokes, NSParams
from oracle.residual import residual as oracle_residual
from paper_2608_09615_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402

TWO_PI = 2 * math.pi


def test_filter_matches_oracle():
    gf = Grid(3, (8, 8, 8), (0.0,) * 3, (TWO_PI,) * 3, 4)
    gc = Grid(3, (2, 2, 2), (0.0,) * 3, (TWO_PI,) * 3, 3)
    U = inputs.tgv_3d((8, 8, 8), 4, perturb_seed=1)
    Uc = sd.filter_project(torch.from_numpy(U).cuda(), (2, 2, 2), 4, 4, 3).cpu().numpy()
    Uo = project(U, gf, gc)
    assert np.abs(Uc - Uo).max() <= 1e-12 * np.abs(Uo).max()


@pytest.mark.parametrize("p", [3, 4])
def test_flux_means_and_features_match_oracle(p):
    ne = (4, 3, 5)
    g = Grid(3, ne, (0.0,) * 3, (TWO_PI, 0.75 * TWO_PI, 1.25 * TWO_PI), p)
    hi = (TWO_PI, 0.75 * TWO_PI, 1.25 * TWO_PI)
    prm = NSParams(Re=3000.0)
    U = inputs.tgv_3d(ne, p, perturb_seed=2)
    ctx = sd.SD(3, ne, (0.0,) * 3, hi, p, "compact",
                sd.Physics(kind="ns", Re=3000.0), "f64")
    X, Mn = ctx.closure_data(torch.from_numpy(U).cuda())
    ctx.close()
    X, Mn = X.cpu().numpy(), Mn.cpu().numpy()
    F = point_fluxes(U, g, NavierStokes(prm))
    w = g.ops.ws
    W = np.einsum("k,j,i->kji", w, w, w) / 8.0
    for d in range(3):
        mo = np.einsum("v...kji,kji->v...", F[d], W).reshape(5, -1)
        for v in range(5):
            assert np.abs(Mn[:, 3 * v + d] - mo[v]).max() <= 1e-10 * (1 + np.abs(mo[v]).max())
    Xo = o_features(U, g, NavierStokes(prm))
    # features are stored in FP32: relative 1e-6 of each column's scale (the modal fractions
    # are ratios of small energies and get an absolute 1e-6)
    scale = np.maximum(np.abs(Xo).max(axis=0), 1e-3)
    assert np.all(np.abs(X - Xo) <= 2e-6 * scale + 1e-7), np.argmax(np.abs(X - Xo).max(axis=0) / scale)


def test_targets_match_oracle():
    gf = Grid(3, (8, 8, 8), (0.0,) * 3, (TWO_PI,) * 3, 4)
    gc = Grid(3, (2, 2, 2), (0.0,) * 3, (TWO_PI,) * 3, 3)
    U = inputs.tgv_3d((8, 8, 8), 4, perturb_seed=4)
    prm = NSParams()
    tau_o, Uc_o = sgs_target(U, gf, gc, NavierStokes(prm))
    Uf = torch.from_numpy(U).cuda()
    cf = sd.SD(3, (8, 8, 8), (0.0,) * 3, (TWO_PI,) * 3, 4, "compact", sd.Physics(kind="ns"), "f64")
    cc = sd.SD(3, (2, 2, 2), (0.0,) * 3, (TWO_PI,) * 3, 3, "compact", sd.Physics(kind="ns"), "f64")
    _, mf = cf.closure_data(Uf, features=False)
    Uc = sd.filter_project(Uf, (2, 2, 2), 4, 4, 3)
    _, mc = cc.closure_data(Uc, features=False)
    tau = sd.closure_targets(mf, mc, (2, 2, 2), 4).cpu().numpy()
    cf.close()
    cc.close()
    to = np.moveaxis(tau_o.reshape(5, 8, 3), 1, 0).reshape(8, 15)    # [e][3 v + d]
    assert np.abs(tau - to).max() <= 1e-6 * np.abs(to).max() + 1e-12


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_flux_injection_matches_oracle(scheme):
    ne, p = (3, 4, 2), 3
    U = inputs.tgv_3d(ne, p, perturb_seed=5)
    rng = np.random.default_rng(0)
    tau = rng.normal(size=(int(np.prod(ne)), 15)).astype(np.float32)
    g = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, dtype=np.longdouble)
    to = np.moveaxis(tau.astype(np.float64).reshape(ne[2], ne[1], ne[0], 5, 3), 3, 0)
    Ro = oracle_residual(U, g, scheme, NavierStokes(NSParams()), tau=to).astype(np.float64)
    ctx = sd.SD(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, scheme, sd.Physics(kind="ns"), "f64")
    tg = torch.from_numpy(tau).cuda()
    ctx.set_flux_tau(tg)
    Rg = ctx.residual(torch.from_numpy(U).cuda()).cpu().numpy()
    ctx.close()
    for v in range(5):
        assert np.abs(Rg[v] - Ro[v]).max() <= 1e-12 * np.abs(Ro[v]).max()
