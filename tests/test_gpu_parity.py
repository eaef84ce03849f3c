"""GPU parity of the CUDA path (called through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances:
  * FP64 residual: max |R_gpu - R_ref| <= 1e-12 * max |R_ref|, per variable (the FP64
    target). R_ref is the oracle evaluated in x86 80-bit extended precision: at Ma = 0.1
    the momentum flux carries p0 ~ 71 while the residual is O(1), so the FP64 oracle's own
    round-off reaches ~8e-12 on smooth Taylor-Green fields (measured against the extended
    evaluation); the extended evaluation is the same definition with ~2000x less round-off.
  * FP32 residual: see test_fp32_* below; the bound is stated and derived in each test.
"""
import numpy as np
import pytest

from oracle.diagnostics import ns_diagnostics, scalar_diagnostics
from oracle.grid import Grid
from oracle.physics import Heat, NavierStokes, NSParams, PorousMedium
from oracle.residual import residual as oracle_residual
from oracle.timestep import STEPPERS
from paper_2608_09615_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402

TWO_PI = 2 * np.pi


def rel_err(Rg, Ro):
    out = []
    for v in range(Ro.shape[0]):
        den = np.abs(Ro[v]).max()
        out.append(np.abs(Rg[v] - Ro[v]).max() / (den if den > 0 else 1.0))
    return np.array(out)


def ns_phys(**kw):
    prm = NSParams(**{k: v for k, v in kw.items() if k in NSParams.__dataclass_fields__})
    return prm, sd.Physics(kind="ns", gamma=prm.gamma, Pr=prm.Pr, Re=prm.Re, Ma=prm.Ma,
                           rho0=prm.rho0, u0=prm.u0, L=prm.L, sutherland=prm.sutherland,
                           suth_s=prm.suth_s, riemann=prm.riemann, harten=prm.harten)


def ext_residual(U, dim, ne, lo, hi, p, scheme, phys_o):
    """The oracle residual evaluated in extended precision (np.longdouble)."""
    g = Grid(dim, ne, lo, hi, p, dtype=np.longdouble)
    return oracle_residual(U, g, scheme, phys_o).astype(np.float64)


def gpu_residual(U, dim, ne, lo, hi, p, scheme, phys, precision):
    ctx = sd.SD(dim, ne, lo, hi, p, scheme, phys, precision)
    dt = ctx.dtype
    Ug = torch.from_numpy(np.ascontiguousarray(U)).to("cuda", dt)
    R = ctx.residual(Ug)
    torch.cuda.synchronize()
    out = R.double().cpu().numpy()
    ctx.close()
    return out


# ------------------------------------------------------------------ scalar, FP64
SCALAR_CASES = [(1, (7,), p) for p in range(1, 9)] + [(3, (3, 4, 2), p) for p in range(1, 7)] + \
    [(3, (2, 1, 2), 7), (3, (1, 2, 1), 8), (3, (1, 1, 1), 3)]


@pytest.mark.parametrize("dim,ne,p", SCALAR_CASES)
@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("kind", ["heat", "pme"])
def test_scalar_fp64_parity(dim, ne, p, scheme, kind):
    lo, hi = (0.0,) * dim, tuple(1.0 + 0.3 * d for d in range(dim))
    g = Grid(dim, ne, lo, hi, p)
    U = inputs.random_scalar(dim, ne, p, seed=p + 10 * dim, lo=0.05, hi=1.0)
    phys_o = Heat(0.37) if kind == "heat" else PorousMedium(2.0)
    phys_g = sd.Physics(kind=kind, nu=0.37, m_pme=2.0)
    Ro = ext_residual(U, dim, ne, lo, hi, p, scheme, phys_o)
    Rg = gpu_residual(U, dim, ne, lo, hi, p, scheme, phys_g, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


def test_pme_exponent_five_fp64():
    g = Grid(1, (9,), (-1.0,), (1.0,), 4)
    U = inputs.random_scalar(1, (9,), 4, seed=3, lo=0.0, hi=1.0)
    Ro = ext_residual(U, 1, (9,), (-1.0,), (1.0,), 4, "compact", PorousMedium(5.0))
    Rg = gpu_residual(U, 1, (9,), (-1.0,), (1.0,), 4, "compact", sd.Physics(kind="pme", m_pme=5.0), "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


# ------------------------------------------------------------------ Navier-Stokes, FP64
NS_CASES = [((3, 2, 4), 1), ((2, 3, 2), 2), ((3, 2, 2), 3), ((2, 2, 3), 4), ((2, 2, 2), 5),
            ((2, 1, 2), 6), ((1, 2, 1), 7), ((1, 1, 2), 8), ((1, 1, 1), 2)]


@pytest.mark.parametrize("ne,p", NS_CASES)
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_fp64_parity_random_state(ne, p, scheme):
    prm, phys = ns_phys(Re=300.0)
    lo, hi = (0.0,) * 3, (TWO_PI, 0.8 * TWO_PI, 1.1 * TWO_PI)
    g = Grid(3, ne, lo, hi, p)
    U = inputs.random_state(ne, p, seed=p)
    Ro = ext_residual(U, 3, ne, lo, hi, p, scheme, NavierStokes(prm))
    Rg = gpu_residual(U, 3, ne, lo, hi, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


@pytest.mark.parametrize("riemann", ["roe", "rusanov"])
@pytest.mark.parametrize("sutherland", [True, False])
@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_fp64_parity_options(riemann, sutherland, scheme):
    prm, phys = ns_phys(Re=500.0, riemann=riemann, sutherland=sutherland, harten=0.3)
    ne, p = (3, 3, 2), 3
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    g = Grid(3, ne, lo, hi, p)
    U = inputs.random_state(ne, p, seed=11, rel=0.3)
    Ro = ext_residual(U, 3, ne, lo, hi, p, scheme, NavierStokes(prm))
    Rg = gpu_residual(U, 3, ne, lo, hi, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


@pytest.mark.parametrize("scheme", ["br1", "compact"])
def test_ns_fp64_parity_tgv(scheme):
    prm, phys = ns_phys()
    ne, p = (6, 6, 6), 4
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    g = Grid(3, ne, lo, hi, p)
    U = inputs.tgv_3d(ne, p, perturb_seed=0)
    Ro = ext_residual(U, 3, ne, lo, hi, p, scheme, NavierStokes(prm))
    Rg = gpu_residual(U, 3, ne, lo, hi, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


# ------------------------------------------------------------------ FP32 error
# The FP32 residual against the oracle on the same FP32-rounded input, relative L2 error per
# variable (||R32_v - R_v||_2 / ||R_v||_2). Its floor is u kappa_v (tests/fp32_floor.py): the
# sum of the magnitudes of the divergence terms over the residual, times FP32's unit
# roundoff. On these Taylor-Green fields u kappa is already 8e-5 for rho and rho E at 8^3 and
# grows like 1/h, so the benchmark's 1e-5 per residual is out of reach for any evaluation
# that rounds the flux-point values to FP32; the tests hold the kernels to a small multiple
# of that floor and to the measured levels (recorded on B300 at 8^3, compact and BR1: l2
# 4.1e-5 2.8e-5 2.8e-5 2.0e-6 5.8e-5; ratio to u kappa 0.53 3.9 4.0 0.91 0.72).
FP32_LEVEL_8 = np.array([4.1e-5, 2.8e-5, 2.8e-5, 2.0e-6, 5.8e-5])
FLOOR_FACTOR = 8.0


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_fp32_error_tgv_within_rounding_floor(scheme, capsys):
    from fp32_floor import U32 as UNIT_ROUNDOFF, conditioning, kappa
    prm, phys = ns_phys()
    ne, p = (8, 8, 8), 4
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    g = Grid(3, ne, lo, hi, p)
    U = inputs.tgv_3d(ne, p, perturb_seed=0)
    U32 = U.astype(np.float32).astype(np.float64)       # both sides see the FP32 input
    Ro, C = conditioning(U32, g, scheme, prm)
    Rg = gpu_residual(U32, 3, ne, lo, hi, p, scheme, phys, "f32")
    e_max = rel_err(Rg, Ro)
    e_l2 = np.array([np.linalg.norm(Rg[v] - Ro[v]) / np.linalg.norm(Ro[v]) for v in range(5)])
    floor = UNIT_ROUNDOFF * kappa(Ro, C)
    with capsys.disabled():
        print("\nFP32 TGV 8^3 p4 %s: max-rel %s  l2-rel %s  u*kappa %s" % (
            scheme, " ".join("%.2e" % x for x in e_max), " ".join("%.2e" % x for x in e_l2),
            " ".join("%.2e" % x for x in floor)))
    assert np.all(np.isfinite(Rg))
    assert np.all(e_l2 <= FLOOR_FACTOR * floor), (e_l2, floor)
    assert np.all(e_l2 <= 2.0 * FP32_LEVEL_8), e_l2


# ------------------------------------------------------------------ host path, RK, diagnostics
@pytest.mark.parametrize("ne,precision,scheme", [((4, 3, 2), "f32", "compact"),     # one pass
                                                   ((4, 3, 7), "f32", "compact"),     # 7 z-slabs
                                                   ((3, 5, 20), "f32", "br1"),        # 16 uneven slabs
                                                   ((2, 3, 40), "f32", "compact"),    # thin wrap slabs
                                                   ((2, 2, 33), "f64", "br1"),        # thin wrap slabs
                                                   ((3, 2, 9), "f64", "compact")])
def test_host_path_equals_device_path(ne, precision, scheme):
    # sd_residual_host: whole-grid copies for thin grids, the slab pipeline (copies on
    # their own streams, phases per z-slab) otherwise; bitwise the device residual
    prm, phys = ns_phys()
    p = 3
    ctx = sd.SD(3, ne, (0,) * 3, (TWO_PI,) * 3, p, scheme, phys, precision)
    U = torch.from_numpy(inputs.tgv_3d(ne, p, perturb_seed=1)).to(ctx.dtype)
    Rd = ctx.residual(U.cuda()).cpu()
    Uh = U.pin_memory()
    Rh = torch.full_like(Uh, float("nan")).pin_memory()
    for _ in range(2):
        ctx.residual_host(Uh, Rh)
        assert torch.equal(Rd, Rh)
    ctx.close()


@pytest.mark.parametrize("rk", ["rk4", "ssprk54", "lsrk54"])
def test_rk_step_fp64_parity(rk):
    prm, phys = ns_phys(Re=400.0)
    ne, p = (3, 2, 2), 3
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    g = Grid(3, ne, lo, hi, p)
    U = inputs.tgv_3d(ne, p, perturb_seed=2)
    dt = 1e-3
    Uo = U.copy()
    for _ in range(3):
        Uo = STEPPERS[rk](lambda V: oracle_residual(V, g, "compact", NavierStokes(prm)), Uo, dt)
    ctx = sd.SD(3, ne, lo, hi, p, "compact", phys, "f64")
    Ug = torch.from_numpy(U.copy()).cuda()
    for s in range(3):
        ctx.rk_step(Ug, s * dt, dt, rk)
    Ug = Ug.cpu().numpy()
    ctx.close()
    assert rel_err(Ug - U, Uo - U).max() <= 1e-11


def test_rk_step_fp32_residual_close_to_fp64():
    prm, phys = ns_phys()
    ne, p = (4, 4, 4), 4
    U = inputs.tgv_3d(ne, p, perturb_seed=3)
    out = {}
    for prec in ("f32", "f64"):
        ctx = sd.SD(3, ne, (0,) * 3, (TWO_PI,) * 3, p, "compact", phys, prec)
        Ug = torch.from_numpy(U.copy()).cuda()
        for s in range(5):
            ctx.rk_step(Ug, s * 1e-3, 1e-3, "ssprk54")
        out[prec] = Ug.cpu().numpy()
        ctx.close()
    dU = out["f64"] - U
    assert rel_err(out["f32"] - U, dU).max() < 1e-3


@pytest.mark.parametrize("case", ["ns_compact", "ns_br1", "heat3d", "ns_closure_tau"])
def test_rk_step_equals_stage_by_stage(case):
    # sd_rk_step and sd_rk_prepare followed by sd_rk_stage for every stage (the form a
    # decomposed grid uses, exchanging halos between stages) give the same state to the bit,
    # over several steps, on odd and even grids.
    import ctypes
    if case == "heat3d":
        ne, p, scheme = (5, 3, 4), 3, "compact"
        phys = sd.Physics(kind="heat", nu=0.05)
        U = inputs.heat_modes_3d(ne, p, seed=2)[0]
    else:
        ne, p = (5, 4, 3), 4
        scheme = "br1" if case == "ns_br1" else "compact"
        phys = sd.Physics(kind="ns", Re=500.0)
        U = inputs.tgv_3d(ne, p, perturb_seed=6)
    dt = 2e-3
    out = []
    for whole_step in (True, False):
        ctx = sd.SD(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, scheme, phys, "f32")
        if case == "ns_closure_tau":
            tau = torch.linspace(-1e-3, 1e-3, int(np.prod(ne)) * 15, device="cuda").view(-1, 15).contiguous()
            ctx.set_flux_tau(tau)
        Ug = torch.from_numpy(U.copy()).cuda()
        for k in range(3):
            if whole_step:
                ctx.rk_step(Ug, k * dt, dt, "ssprk54")
            else:
                x = sd.rk_prepare(ctx, Ug)
                for j in range(5):
                    x = sd.rk_stage(ctx, Ug, j, dt, "ssprk54")
        torch.cuda.synchronize()
        out.append(Ug.cpu().numpy())
        ctx.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])
    del ctypes


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("p,ne", [(2, (4, 3, 5)), (4, (4, 3, 5)), (2, (24, 20, 18))])
def test_diagnostics_parity_ns(p, ne, precision):
    # FP64 contexts: every integrand in FP64 (1e-12). FP32 contexts form the kinetic-energy
    # and enstrophy integrands in FP32 from the offset state and sum them in FP64 (FP32
    # rounding of each point's value: 1e-6 relative on the sums); the conserved totals come
    # from the FP64 state in both (1e-12). The 24 x 20 x 18 grid has more element groups
    # than the persistent diagnostics kernel has blocks, so each block sums several.
    prm, phys = ns_phys()
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    g = Grid(3, ne, lo, hi, p)
    U = inputs.tgv_3d(ne, p, perturb_seed=4)
    do = ns_diagnostics(U, g)
    ctx = sd.SD(3, ne, lo, hi, p, "compact", phys, precision)
    dg = ctx.diagnostics(torch.from_numpy(U).cuda(), 0.5)
    ctx.close()
    tol = 1e-12 if precision == "f64" else 1e-6
    for k in ("ke", "ke_rho", "enstrophy"):
        assert dg[k] == pytest.approx(do[k], rel=tol), k
    for k in ("mass", "energy", "volume"):
        assert dg[k] == pytest.approx(do[k], rel=1e-12), k
    for i in range(3):
        assert dg["mom"][i] == pytest.approx(do["mom"][i], abs=1e-12 * do["mass"])
    assert dg["nonfinite"] == 0 and dg["t"] == 0.5


@pytest.mark.parametrize("dim,ne", [(1, (9,)), (3, (3, 2, 4))])
def test_diagnostics_parity_scalar(dim, ne):
    p = 3
    lo, hi = (0.0,) * dim, (1.0,) * dim
    g = Grid(dim, ne, lo, hi, p)
    U = inputs.random_scalar(dim, ne, p, seed=5)
    do = scalar_diagnostics(U, g)
    ctx = sd.SD(dim, ne, lo, hi, p, "compact", sd.Physics(kind="heat"), "f64")
    dg = ctx.diagnostics(torch.from_numpy(U).cuda())
    ctx.close()
    assert dg["mass"] == pytest.approx(do["mass"], rel=1e-12, abs=1e-14)
    assert dg["l2sq"] == pytest.approx(do["l2sq"], rel=1e-12)


def test_diagnostics_flags_nonfinite():
    ne, p = (2, 2, 2), 2
    U = inputs.tgv_3d(ne, p)
    U[4, 1, 0, 1, 2, 0, 1] = np.inf
    ctx = sd.SD(3, ne, (0,) * 3, (TWO_PI,) * 3, p, "compact", sd.Physics(), "f32")
    Ug = torch.from_numpy(U).cuda()
    with pytest.raises(sd.SDError) as ei:
        ctx.diagnostics(Ug)
    assert ei.value.status == sd.SD_ENONFINITE
    d = ctx.diagnostics(Ug, raise_nonfinite=False)
    assert d["nonfinite"] == 1
    ctx.close()


# ------------------------------------------------------------------ 1D sin(x) diffusion run
def test_sin_diffusion_rk4_run():
    # 1D u_t = u_xx on [0, 2 pi], 16 elements, p = 3, u0 = sin x, RK4 dt = 1e-4 to t = 1.
    p, E = 3, 16
    U = inputs.sin_1d(E, p)
    (x,) = inputs.coordinates(1, (E,), (0.0,), (TWO_PI,), p)
    errs = {}
    for scheme in ("compact", "br1"):
        ctx = sd.SD(1, (E,), (0.0,), (TWO_PI,), p, scheme, sd.Physics(kind="heat", nu=1.0), "f64")
        Ug = torch.from_numpy(U.copy()).cuda()
        for s in range(10000):
            ctx.rk_step(Ug, s * 1e-4, 1e-4, "rk4")
        uT = Ug.cpu().numpy()[0]
        ctx.close()
        errs[scheme] = np.abs(uT - np.exp(-1.0) * np.sin(x)).max()
        # the first 100 steps against the oracle's RK4
        g = Grid(1, (E,), (0.0,), (TWO_PI,), p)
        Uo = U.copy()
        for _ in range(100):
            Uo = STEPPERS["rk4"](lambda V: oracle_residual(V, g, scheme, Heat(1.0)), Uo, 1e-4)
        ctx = sd.SD(1, (E,), (0.0,), (TWO_PI,), p, scheme, sd.Physics(kind="heat", nu=1.0), "f64")
        Ug = torch.from_numpy(U.copy()).cuda()
        for s in range(100):
            ctx.rk_step(Ug, s * 1e-4, 1e-4, "rk4")
        assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-13
        ctx.close()
    assert errs["compact"] < 1e-4
    assert errs["compact"] < errs["br1"]   # p = 3 is an even order: BR1 loses one order


# ------------------------------------------------------------------ full size (48^3 p4)
FULL_NE, FULL_P = (48, 48, 48), 4


@pytest.fixture(scope="module")
def full_tgv():
    return inputs.tgv_3d(FULL_NE, FULL_P, perturb_seed=0)


def _block_around(U, centre, half=2):
    """The (2 half + 1)^3 elements around `centre` (periodic wrap) of the full field."""
    idx = [np.arange(c - half, c + half + 1) % n for c, n in zip(centre, FULL_NE)]
    B = U[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    return np.ascontiguousarray(B)


SAMPLES = [(0, 0, 0), (47, 47, 47), (23, 5, 40), (11, 36, 2)]


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_full_size_fp64_sampled(full_tgv, scheme):
    # At the benchmark size the oracle cannot run on the whole grid; an element's
    # residual depends only on elements within distance 2 (BR1) / 1 (compact), so the
    # oracle evaluated on a periodic 5^3 block around it gives that element exactly.
    # The relative error uses the same scale as the other parity tests: the largest
    # |R_v| over the whole field (here the GPU field, whose maximum agrees with the oracle's
    # to ~1e-12 wherever both exist).
    prm, phys = ns_phys()
    h = 2 * np.pi / 48
    Rg = gpu_residual(full_tgv, 3, FULL_NE, (0.0,) * 3, (2 * np.pi,) * 3, FULL_P, scheme, phys, "f64")
    scale = np.abs(Rg).reshape(5, -1).max(axis=1)
    for c in SAMPLES:
        B = _block_around(full_tgv, c)
        Rb = ext_residual(B, 3, (5, 5, 5), (0.0,) * 3, (5 * h,) * 3, FULL_P, scheme, NavierStokes(prm))
        ro = Rb[:, 2, 2, 2]
        rg = Rg[:, c[2], c[1], c[0]]
        err = np.abs(rg - ro).reshape(5, -1).max(axis=1) / scale
        assert err.max() <= 1e-12, (c, err)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_fp64_p8_many_groups_per_block_sampled(scheme):
    # FP64 Navier-Stokes at p = 8 has the largest shared-memory staging of the line kernels
    # (one or two resident blocks per SM). 336 elements are more than the resident blocks,
    # so each block runs its staging pipeline over several groups. Sampled elements against
    # the oracle on their periodic 5^3 blocks (an element's residual depends only on
    # elements within distance 2).
    ne, p, h = (8, 7, 6), 8, 0.35
    prm, phys = ns_phys(Re=300.0)
    U = inputs.random_state(ne, p, seed=8)
    Rg = gpu_residual(U, 3, ne, (0.0,) * 3, tuple(h * n for n in ne), p, scheme, phys, "f64")
    scale = np.abs(Rg).reshape(5, -1).max(axis=1)
    for c in [(0, 0, 0), (7, 6, 5), (3, 2, 4)]:
        idx = [np.arange(ci - 2, ci + 3) % n for ci, n in zip(c, ne)]
        B = np.ascontiguousarray(U[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])
        Rb = ext_residual(B, 3, (5, 5, 5), (0.0,) * 3, (5 * h,) * 3, p, scheme, NavierStokes(prm))
        err = np.abs(Rg[:, c[2], c[1], c[0]] - Rb[:, 2, 2, 2]).reshape(5, -1).max(axis=1) / scale
        assert err.max() <= 1e-12, (c, err)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_full_size_fp32_sampled_within_rounding_floor(full_tgv, scheme, capsys):
    # The FP32 residual of the benchmark grid (48^3 p4, the launch configuration the bench
    # times) at the sampled elements, against the oracle on their 5^3 blocks (FP32-rounded
    # input on both sides), relative L2 over the sampled elements' points: within a small
    # multiple of the rounding floor u kappa of those points (fp32_floor.py). At this
    # resolution the floor is 6x the 8^3 one.
    from fp32_floor import U32 as UNIT_ROUNDOFF, conditioning, kappa
    prm, phys = ns_phys()
    h = 2 * np.pi / 48
    U = full_tgv.astype(np.float32).astype(np.float64)
    Rg = gpu_residual(U, 3, FULL_NE, (0.0,) * 3, (2 * np.pi,) * 3, FULL_P, scheme, phys, "f32")
    ro, rg, cc = [], [], []
    for c in SAMPLES:
        B = _block_around(U, c)
        Rb, Cb = conditioning(B, Grid(3, (5, 5, 5), (0.0,) * 3, (5 * h,) * 3, FULL_P), scheme, prm)
        ro.append(Rb[:, 2, 2, 2])
        cc.append(Cb[:, 2, 2, 2])
        rg.append(Rg[:, c[2], c[1], c[0]])
    ro, rg, cc = (np.stack(x, axis=1) for x in (ro, rg, cc))
    e_l2 = np.array([np.linalg.norm(rg[v] - ro[v]) / np.linalg.norm(ro[v]) for v in range(5)])
    floor = UNIT_ROUNDOFF * kappa(ro, cc)
    with capsys.disabled():
        print("\nFP32 TGV 48^3 p4 %s, sampled elements: l2-rel %s  u*kappa %s" % (
            scheme, " ".join("%.2e" % x for x in e_l2), " ".join("%.2e" % x for x in floor)))
    assert np.all(e_l2 <= FLOOR_FACTOR * floor), (e_l2, floor)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_full_size_conservation(full_tgv, precision, tol):
    # Periodic grid: the Gauss-weighted total of every residual component vanishes.
    prm, phys = ns_phys()
    R = gpu_residual(full_tgv, 3, FULL_NE, (0.0,) * 3, (2 * np.pi,) * 3, FULL_P, "compact", phys, precision)
    _, w = inputs.gl_points(FULL_P + 1)
    W = np.einsum("k,j,i->kji", w, w, w)[None, None, None]
    for v in range(5):
        tot = np.sum(W * R[v])
        scale = np.sum(W * np.abs(R[v]))
        assert abs(tot) <= tol * scale, (v, tot, scale)


# ------------------------------------------------------------------ interior penalty
@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("eta", [0.02, 1.0])
def test_interior_penalty_fp64_parity(scheme, eta):
    # scalar 1D/3D and Navier-Stokes with the Sec. 3 interior-penalty term
    g1 = (1, (9,), (0.0,), (1.0,), 3)
    U1 = inputs.random_scalar(1, (9,), 3, seed=21)
    gg = Grid(1, (9,), (0.0,), (1.0,), 3, dtype=np.longdouble)
    Ro = oracle_residual(U1, gg, scheme, Heat(0.5), eta_ip=eta).astype(np.float64)
    Rg = gpu_residual(U1, *g1, scheme, sd.Physics(kind="heat", nu=0.5, eta_ip=eta), "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12
    prm, phys = ns_phys(Re=300.0)
    phys.eta_ip = eta
    ne, p = (3, 2, 3), 3
    U = inputs.random_state(ne, p, seed=22)
    gg = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, dtype=np.longdouble)
    Ro = oracle_residual(U, gg, scheme, NavierStokes(prm), eta_ip=eta).astype(np.float64)
    Rg = gpu_residual(U, 3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


# ------------------------------------------------------------------ interface viscous flux option (b)
@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("eta", [0.0, 0.3])
def test_viscous_flux_option_b_fp64_parity(scheme, eta):
    # Sec. 2.1 step 4 option (b): the average of the two sides' viscous fluxes
    prm, phys = ns_phys(Re=200.0)
    phys.eta_ip = eta
    phys.viscous_flux = "b"
    ne, p = (3, 3, 2), 3
    U = inputs.random_state(ne, p, seed=31)
    gg = Grid(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, dtype=np.longdouble)
    Ro = oracle_residual(U, gg, scheme, NavierStokes(prm), eta_ip=eta, viscous="b").astype(np.float64)
    Rg = gpu_residual(U, 3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, scheme, phys, "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12
    # porous medium, 1D
    U1 = 1.0 + 0.3 * inputs.random_scalar(1, (11,), 4, seed=32)
    gg = Grid(1, (11,), (0.0,), (1.0,), 4, dtype=np.longdouble)
    Ro = oracle_residual(U1, gg, scheme, PorousMedium(2.0), eta_ip=eta, viscous="b").astype(np.float64)
    Rg = gpu_residual(U1, 1, (11,), (0.0,), (1.0,), 4, scheme,
                      sd.Physics(kind="pme", m_pme=2.0, eta_ip=eta, viscous_flux="b"), "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12


@pytest.mark.parametrize("scheme", ["br1", "compact"])
@pytest.mark.parametrize("viscous", ["a", "b"])
@pytest.mark.parametrize("eta", [0.0, 0.3])
def test_pme_solution_point_diffusivity_fp64_parity(scheme, viscous, eta):
    # Sec. 4.3 variant: m |u|^(m-1) at the solution points, extrapolated
    for m, ne, p in ((3.0, (13,), 4), (2.0, (8,), 2)):
        U = 1.0 + 0.4 * inputs.random_scalar(1, ne, p, seed=41)
        gg = Grid(1, ne, (0.0,), (1.0,), p, dtype=np.longdouble)
        Ro = oracle_residual(U, gg, scheme, PorousMedium(m, coef="solution"), eta_ip=eta,
                             viscous=viscous).astype(np.float64)
        Rg = gpu_residual(U, 1, ne, (0.0,), (1.0,), p, scheme,
                          sd.Physics(kind="pme", m_pme=m, eta_ip=eta, viscous_flux=viscous,
                                     pme_coef="solution"), "f64")
        assert rel_err(Rg, Ro).max() <= 1e-12
    # 3D scalar grid (the layout path of 3D scalar blocks)
    ne, p = (3, 4, 2), 3
    U = 1.0 + 0.4 * inputs.random_scalar(3, ne, p, seed=42)
    gg = Grid(3, ne, (0.0,) * 3, (1.0,) * 3, p, dtype=np.longdouble)
    Ro = oracle_residual(U, gg, scheme, PorousMedium(3.0, coef="solution"), eta_ip=eta,
                         viscous=viscous).astype(np.float64)
    Rg = gpu_residual(U, 3, ne, (0.0,) * 3, (1.0,) * 3, p, scheme,
                      sd.Physics(kind="pme", m_pme=3.0, eta_ip=eta, viscous_flux=viscous, pme_coef="solution"),
                      "f64")
    assert rel_err(Rg, Ro).max() <= 1e-12
