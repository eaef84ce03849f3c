"""Block decomposition on one GPU: 2 x 2 x 2 sub-domains (and uneven splits), each an
ordinary context over its owned block plus ghost layers, their halos exchanged by the
library's pack / unpack kernels. The sub-domains' residuals equal the single-domain residual
bitwise on every owned element, for the compact scheme (one state exchange, one ghost
layer) and for BR1 (one ghost layer with the second, face-gradient exchange; or two ghost
layers and one exchange), in FP64 and FP32; decomposed Runge-Kutta steps (one exchange per
stage) equal the single-domain steps bitwise; the owned-box diagnostics summed over the
sub-domains equal the single-domain diagnostics to FP64 round-off."""
import math

import numpy as np
import pytest

from paper_2608_09615_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402
from paper_2608_09615_b300.decomp import LocalDecomposition  # noqa: E402

LO, HI = (0.0,) * 3, (2 * math.pi,) * 3


def _nan_ghosts(dec, boxes):
    """Ghost elements start as NaN: only the exchanges may fill them."""
    out = []
    for r, B in enumerate(boxes):
        (lo, hi) = dec.part.owned_local(r)
        C = torch.full_like(B, float("nan"))
        sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        C[sl] = B[sl]
        out.append(C)
    return out


CASES = [("compact", False, (2, 2, 2), (6, 5, 4)), ("br1", True, (2, 2, 2), (6, 5, 4)),
         ("br1", False, (2, 2, 2), (6, 5, 4)), ("compact", False, (3, 1, 2), (7, 3, 5)),
         ("br1", True, (1, 3, 2), (3, 6, 4))]


@pytest.mark.parametrize("scheme,gx,parts,ne", CASES)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_subdomain_residuals_equal_single_domain_bitwise(scheme, gx, parts, ne, precision):
    p = 3
    phys = sd.Physics(kind="ns", Re=400.0)
    U = inputs.tgv_3d(ne, p, perturb_seed=4)
    one = sd.SD(3, ne, LO, HI, p, scheme, phys, precision)
    Ug = torch.from_numpy(U).to("cuda", one.dtype)
    R1 = one.residual(Ug).double().cpu().numpy()
    one.close()
    dec = LocalDecomposition(ne, parts, LO, HI, p, scheme, phys, precision, grad_exchange=gx)
    Us = _nan_ghosts(dec, dec.scatter(U))
    Rs = [torch.full_like(x, float("nan")) for x in Us]
    dec.residual(Us, Rs)
    torch.cuda.synchronize()
    R = dec.gather(Rs, U)
    dec.close()
    assert np.all(np.isfinite(R))
    assert np.array_equal(R, R1)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_decomposed_rk_steps_equal_single_domain(scheme):
    ne, p, parts = (6, 4, 4), 3, (2, 2, 1)
    phys = sd.Physics(kind="ns", Re=800.0)
    U = inputs.tgv_3d(ne, p, perturb_seed=1)
    one = sd.SD(3, ne, LO, HI, p, scheme, phys, "f32")
    U1 = torch.from_numpy(U).cuda()
    dt = 2e-3
    for k in range(3):
        one.rk_step(U1, k * dt, dt, "ssprk54")
    d1 = one.diagnostics(U1, 3 * dt)
    one.close()
    dec = LocalDecomposition(ne, parts, LO, HI, p, scheme, phys, "f32")
    Us = _nan_ghosts(dec, dec.scatter(U, dtype=torch.float64))
    for k in range(3):
        dec.rk_step(Us, k * dt, dt, "ssprk54")
    torch.cuda.synchronize()
    got = dec.gather(Us, U)
    d = dec.diagnostics(Us, 3 * dt)
    dec.close()
    assert np.array_equal(got, U1.cpu().numpy())
    for k in ("ke", "enstrophy", "mass", "energy", "volume"):
        assert d[k] == pytest.approx(d1[k], rel=1e-12, abs=1e-14), k
    for i in range(3):
        assert d["mom"][i] == pytest.approx(d1["mom"][i], abs=1e-12 * d1["mass"])


def test_split_residual_equals_residual_and_guards():
    ne, p = (3, 4, 2), 2
    phys = sd.Physics(kind="ns")
    ctx = sd.SD(3, ne, LO, HI, p, "br1", phys, "f64")
    U = torch.from_numpy(inputs.tgv_3d(ne, p, perturb_seed=2)).cuda()
    R0 = ctx.residual(U)
    R = torch.empty_like(U)
    sd.residual_begin(ctx, U)
    sd.residual_end(ctx, U, R)
    torch.cuda.synchronize()
    assert torch.equal(R, R0)
    # index lists with out-of-range entries are skipped, never dereferenced
    bad = torch.tensor([0, 10 ** 6, -3, 1], dtype=torch.int32, device="cuda")
    buf = sd.pack_elements(ctx, U, bad)
    n1 = ctx.nvar * ctx.n ** 3
    torch.cuda.synchronize()
    assert torch.equal(buf.view(ctx.nvar, 4, -1)[:, 0], U.view(ctx.nvar, -1, ctx.n ** 3)[:, 0])
    assert buf.numel() == 4 * n1
    ctx.close()
