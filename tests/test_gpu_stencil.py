"""The element stencil of the CUDA residual (Secs. 2.1, 2.2): perturbing one element
changes the residual of exactly the elements the scheme couples. The compact scheme couples
3 elements per direction, BR1 5. For Navier-Stokes the gradient components couple
directions, so the compact scheme reaches the elements with max|d| <= 1 and |d|_1 <= 2
(19) and BR1 those with |d|_1 <= 2 (25). For the scalar equations the stencil is the centre
plus the 1D stencil along each axis (7 and 13). Elements outside the stencil see bitwise
identical inputs, so their residuals do not change at all; this checks the kernels'
neighbour indexing at every face, including the periodic wrap (the perturbed element sits
at a corner of the grid)."""
import itertools

import numpy as np
import pytest

from paper_2608_09615_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402


def _changed(ctx, U, centre, ne):
    Ug = torch.from_numpy(U).to("cuda", ctx.dtype)
    R0 = ctx.residual(Ug).cpu().numpy()
    V = U.copy()
    idx = (slice(None),) + tuple(reversed(centre))
    V[idx] += 1e-3 * np.random.default_rng(1).uniform(-1, 1, V[idx].shape)
    R1 = ctx.residual(torch.from_numpy(V).to("cuda", ctx.dtype)).cpu().numpy()
    d = np.abs(R1 - R0).max(axis=tuple([0] + list(range(4, 7))))
    out = set()
    for ez, ey, ex in np.argwhere(d > 0):
        rel = []
        for v, c, n in zip((ex, ey, ez), centre, ne):
            r = (int(v) - c) % n
            rel.append(r - n if r > n // 2 else r)
        out.add(tuple(rel))
    return out


def _ball(linf, l1):
    return {d for d in itertools.product(range(-2, 3), repeat=3)
            if max(abs(v) for v in d) <= linf and sum(abs(v) for v in d) <= l1}


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_ns_stencil(scheme, precision):
    ne, p = (6, 7, 6), 2
    ctx = sd.SD(3, ne, (0.0,) * 3, (2 * np.pi,) * 3, p, scheme, sd.Physics(kind="ns", Re=50.0), precision)
    got = _changed(ctx, inputs.random_state(ne, p, seed=6), (0, 6, 5), ne)
    ctx.close()
    assert got == _ball(1 if scheme == "compact" else 2, 2)
    assert len(got) == (19 if scheme == "compact" else 25)


@pytest.mark.parametrize("scheme", ["compact", "br1"])
def test_scalar_stencil(scheme):
    ne, p = (6, 5, 7), 3
    ctx = sd.SD(3, ne, (0.0,) * 3, (1.0,) * 3, p, scheme, sd.Physics(kind="heat", nu=1.0), "f64")
    got = _changed(ctx, inputs.random_scalar(3, ne, p, seed=4), (5, 0, 3), ne)
    ctx.close()
    expect = {d for d in _ball(2, 2) if sum(1 for v in d if v != 0) <= 1}
    if scheme == "compact":
        expect = {d for d in expect if max(abs(v) for v in d) <= 1}
    assert got == expect
