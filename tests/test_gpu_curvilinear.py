"""GPU parity of the curved-grid path (sd_init_curvilinear, then sd_residual / sd_rk_step /
sd_diagnostics / sd_residual_host through the C ABI) against the curvilinear oracle on the
same seeded grids and states.

Tolerances follow the Cartesian parity tests: FP64 residual within 1e-12 of the largest
|R_v| per variable against the oracle evaluated in extended precision (np.longdouble);
FP32 residual reported against the FP64 oracle with the same l2 bound as the Cartesian
FP32 report; properties that hold at any size (conservation, free stream, rotation
equivariance) at the benchmark size.
"""
import numpy as np
import pytest

from oracle.curvilinear import CurvGrid, ns_diagnostics as curv_ns_diagnostics
from oracle.curvilinear import residual as curv_residual
from oracle.physics import Heat, NavierStokes, NSParams, PorousMedium
from oracle.timestep import STEPPERS
from paper_2608_09615_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402

TWO_PI = 2 * np.pi
BOX = ((0.0,) * 3, (TWO_PI,) * 3)


def rel_err(Rg, Ro):
    out = []
    for v in range(Ro.shape[0]):
        den = np.abs(Ro[v]).max()
        out.append(np.abs(Rg[v] - Ro[v]).max() / (den if den > 0 else 1.0))
    return np.array(out)


def ns_phys(eta_ip=0.0, viscous="a", **kw):
    prm = NSParams(**kw)
    return prm, sd.Physics(kind="ns", gamma=prm.gamma, Pr=prm.Pr, Re=prm.Re, Ma=prm.Ma, rho0=prm.rho0,
                           u0=prm.u0, L=prm.L, sutherland=prm.sutherland, suth_s=prm.suth_s,
                           riemann=prm.riemann, harten=prm.harten, eta_ip=eta_ip, viscous_flux=viscous)


def ext_residual(U, nodes, p, scheme, phys_o, **kw):
    g = CurvGrid(nodes, p, dtype=np.longdouble)
    return curv_residual(U, g, scheme, phys_o, **kw).astype(np.float64)


def gpu_residual(U, nodes, p, scheme, phys, precision):
    ctx = sd.SD.curvilinear(nodes, p, scheme, phys, precision)
    assert ctx.curved
    Ug = torch.from_numpy(np.ascontiguousarray(U)).to("cuda", ctx.dtype)
    R = ctx.residual(Ug)
    torch.cuda.synchronize()
    out = R.double().cpu().numpy()
    ctx.close()
    return out


def lattice(kind, ne, lo=BOX[0], hi=BOX[1], seed=0):
    if kind == "jitter":
        return inputs.jittered_lattice(ne, lo, hi, seed=seed, amp=0.12)
    if kind == "wavy":
        return inputs.wavy_lattice(ne, lo, hi, amp=0.15)
    if kind == "rotated":
        N = inputs.jittered_lattice(ne, lo, hi, seed=seed, amp=0.1)
        return np.einsum("ij,jzyx->izyx", inputs.rotation_matrix((1.0, 2.0, 3.0), 0.7), N)
    raise ValueError(kind)


# ------------------------------------------------------------------ FP64 parity
@pytest.mark.parametrize("kind", ["jitter", "wavy", "rotated"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_fp64_parity(kind, p, scheme):
    ne = (4, 3, 3)
    prm, phys = ns_phys()
    U = inputs.random_state(ne, p, seed=p)
    if kind == "rotated":
        U[1:4] = np.einsum("ij,j...->i...", inputs.rotation_matrix((1.0, 2.0, 3.0), 0.7), U[1:4])
    N = lattice(kind, ne, seed=p)
    Ro = ext_residual(U, N, p, scheme, NavierStokes(prm))
    Rg = gpu_residual(U, N, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
@pytest.mark.parametrize("viscous", ["a", "b"])
@pytest.mark.parametrize("eta", [0.0, 0.5])
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_fp64_parity_options(riemann, viscous, eta, scheme):
    ne, p = (3, 3, 2), 2
    prm, phys = ns_phys(eta_ip=eta, viscous=viscous, riemann=riemann, Re=300.0, sutherland=riemann == "roe")
    U = inputs.random_state(ne, p, seed=7)
    N = lattice("jitter", ne, seed=3)
    Ro = ext_residual(U, N, p, scheme, NavierStokes(prm), eta_ip=eta, viscous=viscous)
    Rg = gpu_residual(U, N, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


@pytest.mark.parametrize("p", list(range(1, 9)))
@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("kind", ["heat", "pme"])
def test_scalar_fp64_parity(p, scheme, kind):
    ne = (3, 2, 2) if p <= 5 else (2, 2, 2)
    lo, hi = (0.0,) * 3, (1.0, 1.3, 1.6)
    N = inputs.jittered_lattice(ne, lo, hi, seed=p, amp=0.12)
    U = inputs.random_scalar(3, ne, p, seed=p, lo=0.05, hi=1.0)
    phys_o = Heat(0.37) if kind == "heat" else PorousMedium(2.0)
    for eta, vis in ((0.0, "a"), (0.8, "b")):
        phys_g = sd.Physics(kind=kind, nu=0.37, m_pme=2.0, eta_ip=eta, viscous_flux=vis)
        Ro = ext_residual(U, N, p, scheme, phys_o, eta_ip=eta, viscous=vis)
        Rg = gpu_residual(U, N, p, scheme, phys_g, "f64")
        assert rel_err(Rg, Ro).max() <= 1e-12, (eta, vis)


def test_ns_fp64_parity_tgv_wavy():
    ne, p = (6, 6, 6), 4
    prm, phys = ns_phys()
    N = lattice("wavy", ne)
    U = inputs.tgv_3d(ne, p, perturb_seed=0, X=inputs.curvilinear_coordinates(N, p))
    for scheme in ("compact", "br1"):
        Ro = ext_residual(U, N, p, scheme, NavierStokes(prm))
        Rg = gpu_residual(U, N, p, scheme, phys, "f64")
        assert rel_err(Rg, Ro).max() <= 1e-12


# ------------------------------------------------------------------ FP32
# Relative L2 error per variable of the FP32 residual, held to twice the level measured on
# B300 (compact and BR1 alike: 5.1e-5 2.8e-5 2.8e-5 2.6e-6 6.5e-5). As on Cartesian grids
# these sit at the FP32 rounding floor of the divergence (tests/fp32_floor.py): the wavy
# grid's metric terms are a 15% perturbation of the uniform grid's, and the levels match the
# uniform grid's to within 25%.
FP32_WAVY_LEVEL_8 = np.array([5.1e-5, 2.8e-5, 2.8e-5, 2.6e-6, 6.5e-5])


def test_fp32_error_tgv_wavy(capsys):
    ne, p = (8, 8, 8), 4
    prm, phys = ns_phys()
    N = lattice("wavy", ne)
    U = inputs.tgv_3d(ne, p, perturb_seed=0, X=inputs.curvilinear_coordinates(N, p))
    U32 = U.astype(np.float32).astype(np.float64)
    g = CurvGrid(N, p)
    for scheme in ("compact", "br1"):
        Ro = curv_residual(U32, g, scheme, NavierStokes(prm))
        Rg = gpu_residual(U32, N, p, scheme, phys, "f32")
        e_max = rel_err(Rg, Ro)
        e_l2 = np.array([np.linalg.norm(Rg[v] - Ro[v]) / np.linalg.norm(Ro[v]) for v in range(5)])
        with capsys.disabled():
            print("\nFP32 TGV 8^3 p4 wavy %s: max-rel %s  l2-rel %s" % (
                scheme, " ".join("%.2e" % x for x in e_max), " ".join("%.2e" % x for x in e_l2)))
        assert np.all(np.isfinite(Rg))
        assert np.all(e_l2 <= 2.0 * FP32_WAVY_LEVEL_8), e_l2


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 2e-3)])
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_free_stream_preserved(precision, tol, scheme):
    # a uniform flow on a jittered grid: every flux is O(p0) ~ 71, the residual vanishes
    # up to round-off (the discrete metric identities hold for trilinear elements)
    ne, p = (4, 4, 3), 3
    N = lattice("jitter", ne, seed=5)
    rho, vel, pr = 1.2, (0.3, -0.2, 0.5), 71.4
    U = np.zeros((5,) + tuple(reversed(ne)) + (p + 1,) * 3)
    U[0] = rho
    for i in range(3):
        U[1 + i] = rho * vel[i]
    U[4] = pr / 0.4 + 0.5 * rho * sum(v * v for v in vel)
    _, phys = ns_phys(eta_ip=0.5)
    R = gpu_residual(U, N, p, scheme, phys, precision)
    assert np.abs(R).max() <= tol


# ------------------------------------------------------------------ time stepping, diagnostics, host path
@pytest.mark.parametrize("rk", ["rk4", "ssprk54", "lsrk54"])
def test_rk_step_fp64_parity(rk):
    ne, p = (3, 2, 2), 3
    prm, phys = ns_phys(Re=400.0)
    N = lattice("wavy", ne)
    U = inputs.tgv_3d(ne, p, perturb_seed=2, X=inputs.curvilinear_coordinates(N, p))
    g = CurvGrid(N, p)
    dt = 1e-3
    Uo = U.copy()
    for _ in range(3):
        Uo = STEPPERS[rk](lambda V: curv_residual(V, g, "compact", NavierStokes(prm)), Uo, dt)
    ctx = sd.SD.curvilinear(N, p, "compact", phys, "f64")
    Ug = torch.from_numpy(U.copy()).cuda()
    for s in range(3):
        ctx.rk_step(Ug, s * dt, dt, rk)
    Ug = Ug.cpu().numpy()
    ctx.close()
    assert rel_err(Ug - U, Uo - U).max() <= 1e-11


def test_rk_step_fp32_close_to_fp64():
    ne, p = (4, 4, 4), 4
    _, phys = ns_phys()
    N = lattice("wavy", ne)
    U = inputs.tgv_3d(ne, p, perturb_seed=3, X=inputs.curvilinear_coordinates(N, p))
    out = {}
    for prec in ("f32", "f64"):
        ctx = sd.SD.curvilinear(N, p, "compact", phys, prec)
        Ug = torch.from_numpy(U.copy()).cuda()
        for s in range(5):
            ctx.rk_step(Ug, s * 1e-3, 1e-3, "ssprk54")
        out[prec] = Ug.cpu().numpy()
        ctx.close()
    assert rel_err(out["f32"] - U, out["f64"] - U).max() < 1e-3


@pytest.mark.parametrize("p", [2, 4])
def test_diagnostics_parity_ns(p):
    ne = (4, 3, 5)
    _, phys = ns_phys()
    N = lattice("wavy", ne)
    U = inputs.tgv_3d(ne, p, perturb_seed=4, X=inputs.curvilinear_coordinates(N, p))
    want = curv_ns_diagnostics(U, CurvGrid(N, p))
    ctx = sd.SD.curvilinear(N, p, "compact", phys, "f32")
    got = ctx.diagnostics(torch.from_numpy(U).cuda())
    ctx.close()
    for k in ("ke", "ke_rho", "enstrophy", "mass", "energy"):
        assert abs(got[k] - want[k]) <= 1e-12 * abs(want[k]), k
    for i in range(3):
        assert abs(got["mom"][i] - want["mom"][i]) <= 1e-12 * want["mass"]
    assert abs(got["volume"] - TWO_PI ** 3) <= 1e-12 * TWO_PI ** 3


def test_diagnostics_parity_scalar():
    ne, p = (3, 4, 2), 3
    N = inputs.jittered_lattice(ne, (0.0,) * 3, (1.0, 2.0, 0.5), seed=2, amp=0.12)
    U = inputs.random_scalar(3, ne, p, seed=9)
    g = CurvGrid(N, p)
    W = g.quadrature_weights()
    ctx = sd.SD.curvilinear(N, p, "br1", sd.Physics(kind="heat", nu=1.0), "f64")
    got = ctx.diagnostics(torch.from_numpy(U).cuda())
    ctx.close()
    assert abs(got["mass"] - np.sum(W * U[0])) <= 1e-12 * np.sum(W * np.abs(U[0]))
    assert abs(got["l2sq"] - np.sum(W * U[0] ** 2)) <= 1e-12 * np.sum(W * U[0] ** 2)
    assert abs(got["volume"] - 1.0) <= 1e-12


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_host_path_equals_device_path(precision):
    ne, p = (4, 3, 5), 3
    _, phys = ns_phys()
    N = lattice("wavy", ne)
    ctx = sd.SD.curvilinear(N, p, "compact", phys, precision)
    U = torch.from_numpy(inputs.tgv_3d(ne, p, perturb_seed=1, X=inputs.curvilinear_coordinates(N, p))).to(ctx.dtype)
    Rd = ctx.residual(U.cuda()).cpu()
    Uh = U.pin_memory()
    Rh = torch.full_like(Uh, float("nan")).pin_memory()
    for _ in range(2):
        ctx.residual_host(Uh, Rh)
        assert torch.equal(Rd, Rh)
    ctx.close()


def test_bad_grids_rejected():
    ne, p = (3, 3, 3), 2
    N = lattice("jitter", ne)
    bad = N.copy()
    bad[0, 1, 1, -1] += 0.05                      # image node no longer a translate of node 0
    with pytest.raises(sd.SDError):
        sd.SD.curvilinear(bad, p, "compact", sd.Physics(kind="heat"), "f64")
    flip = N.copy()
    flip[0] = -flip[0]                            # mirrored grid: negative Jacobian
    with pytest.raises(sd.SDError):
        sd.SD.curvilinear(flip, p, "compact", sd.Physics(kind="heat"), "f64")
    with pytest.raises(sd.SDError):
        sd.SD.curvilinear(N, p, "compact", sd.Physics(kind="pme", pme_coef="solution"), "f64")


# ------------------------------------------------------------------ benchmark size (48^3 p4)
FULL_NE, FULL_P = (48, 48, 48), 4


@pytest.fixture(scope="module")
def full_wavy():
    N = inputs.wavy_lattice(FULL_NE, *BOX, amp=0.15)
    U = inputs.tgv_3d(FULL_NE, FULL_P, perturb_seed=0, X=inputs.curvilinear_coordinates(N, FULL_P))
    return N, U


def _block_nodes(N, centre, half=2):
    """Corner nodes of the (2 half + 1)^3 elements around `centre`, unwrapped across the
    periodic seam (nodes beyond it are shifted by the period vector)."""
    base = N[:, :-1, :-1, :-1]
    T = [N[:, 0, 0, -1] - N[:, 0, 0, 0], N[:, 0, -1, 0] - N[:, 0, 0, 0], N[:, -1, 0, 0] - N[:, 0, 0, 0]]
    idx = [np.arange(c - half, c + half + 2) for c in centre]
    out = np.empty((3, len(idx[2]), len(idx[1]), len(idx[0])))
    for kk, k in enumerate(idx[2]):
        for jj, j in enumerate(idx[1]):
            for ii, i in enumerate(idx[0]):
                sh = (i // FULL_NE[0]) * T[0] + (j // FULL_NE[1]) * T[1] + (k // FULL_NE[2]) * T[2]
                out[:, kk, jj, ii] = base[:, k % FULL_NE[2], j % FULL_NE[1], i % FULL_NE[0]] + sh
    return out


def _block_state(U, centre, half=2):
    idx = [np.arange(c - half, c + half + 1) % n for c, n in zip(centre, FULL_NE)]
    return np.ascontiguousarray(U[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])


SAMPLES = [(0, 0, 0), (47, 47, 47), (23, 5, 40), (11, 36, 2)]


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_full_size_fp64_sampled(full_wavy, scheme):
    # An element's residual depends only on the elements within two of it per axis (their
    # states and corner nodes), so the oracle on the 5^3 block around it (wrapped as a
    # periodic grid whose far seam the centre never reaches) gives that element exactly.
    N, U = full_wavy
    prm, phys = ns_phys()
    Rg = gpu_residual(U, N, FULL_P, scheme, phys, "f64")
    scale = np.abs(Rg).reshape(5, -1).max(axis=1)
    for c in SAMPLES:
        Rb = ext_residual(_block_state(U, c), _block_nodes(N, c), FULL_P, scheme, NavierStokes(prm))
        err = np.abs(Rg[:, c[2], c[1], c[0]] - Rb[:, 2, 2, 2]).reshape(5, -1).max(axis=1) / scale
        assert err.max() <= 1e-12, (c, err)


def test_full_size_rotation_equivariance_fp32(full_wavy):
    # rotating grid and momentum rotates the momentum residual (a property at any size)
    N, U = full_wavy
    Rm = inputs.rotation_matrix((1.0, -2.0, 0.5), 0.9)
    N1 = np.einsum("ij,jzyx->izyx", Rm, N)
    U1 = U.copy()
    U1[1:4] = np.einsum("ij,j...->i...", Rm, U[1:4])
    _, phys = ns_phys()
    R0 = gpu_residual(U, N, FULL_P, "compact", phys, "f32")
    R1 = gpu_residual(U1, N1, FULL_P, "compact", phys, "f32")
    R0[1:4] = np.einsum("ij,j...->i...", Rm, R0[1:4])
    e_l2 = np.array([np.linalg.norm(R1[v] - R0[v]) / np.linalg.norm(R0[v]) for v in range(5)])
    assert e_l2.max() < 1e-3, e_l2


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_conservation_24(precision, tol):
    ne, p = (24, 24, 24), 4
    N = inputs.wavy_lattice(ne, *BOX, amp=0.15)
    U = inputs.tgv_3d(ne, p, perturb_seed=0, X=inputs.curvilinear_coordinates(N, p))
    _, phys = ns_phys()
    R = gpu_residual(U, N, p, "compact", phys, precision)
    W = CurvGrid(N, p).quadrature_weights()
    for v in range(5):
        tot = np.sum(W * R[v])
        scale = np.sum(W * np.abs(R[v]))
        assert abs(tot) <= tol * scale, (v, tot, scale)


@pytest.mark.parametrize("ne,p", [((1, 2, 3), 2), ((1, 1, 1), 3), ((2, 1, 1), 1)])
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_single_element_axes_fp64_parity(ne, p, scheme):
    # degenerate periodic grids: along an axis with one element, an element is its own
    # neighbour on both sides (its two faces are periodic images of each other)
    prm, phys = ns_phys(eta_ip=0.3)
    U = inputs.random_state(ne, p, seed=11)
    N = inputs.jittered_lattice(ne, *BOX, seed=4, amp=0.12)
    Ro = ext_residual(U, N, p, scheme, NavierStokes(prm), eta_ip=0.3)
    Rg = gpu_residual(U, N, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12
