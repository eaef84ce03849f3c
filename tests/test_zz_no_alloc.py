"""The allocation-free FP32 residual (sd_residual_f32_noalloc), for callers that cannot
let a library allocate device memory: it must give the same residual as the context-based
sd_residual, call after call, while its scratch lives in the library's static device
array. This file is collected last so that a run stopping at its first failure has run
every other test first."""
import ctypes
import math

import numpy as np
import pytest

import paper_2608_09615_b300 as sd
from paper_2608_09615_b300 import build, inputs

TWO_PI = 2 * math.pi


def _mesh(dim, ne, lo, hi):
    ne = list(ne) + [1] * (3 - len(ne))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    return sd._Mesh(dim, (ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi))


def _scratch_values(dim, ne, p, nvar, ngrad):
    """Scratch the entry point needs (include/sd.h): nelem (2 dim (F + G) + dim F) values,
    F = nvar n^(dim-1) (+ n^(dim-1) for a scalar, its diffusivity traces) and G = ngrad
    n^(dim-1), each rounded up to a multiple of 4; the trace and gradient parts are each
    rounded up to a multiple of 64 values."""
    n = p + 1
    nq = n ** (dim - 1)
    nelem = int(np.prod(ne))
    F = (nvar * nq + (nq if nvar == 1 else 0) + 3) // 4 * 4
    G = (ngrad * nq + 3) // 4 * 4
    up = lambda x: (x + 63) // 64 * 64
    return up(nelem * 2 * dim * F) + up(nelem * 2 * dim * G) + nelem * dim * F


SCRATCH_FLOATS = 9 * 1024 * 1024


def test_oversize_grid_is_rejected_before_any_launch():
    # 16^3 elements at p = 4 (Navier-Stokes) need 10,321,920 scratch values, more than the
    # 9 Mi (9,437,184) the static array holds: rejected on the host, so no device is
    # touched (the pointers are never dereferenced)
    assert _scratch_values(3, (16, 16, 16), 4, 5, 9) == 10321920 > SCRATCH_FLOATS
    assert _scratch_values(3, (15, 15, 15), 4, 5, 9) <= SCRATCH_FLOATS
    build.build()
    lib = sd.load_library()
    m = _mesh(3, (16, 16, 16), (0.0,) * 3, (TWO_PI,) * 3)
    ph = sd.Physics(kind="ns").to_c()
    st = lib.sd_residual_f32_noalloc(ctypes.byref(m), 4, 1, ctypes.byref(ph),
                                     ctypes.c_void_p(256), ctypes.c_void_p(1 << 30), None)
    assert st == sd.SD_EINVAL
    assert b"static scratch" in lib.sd_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["ns_compact", "ns_br1", "heat_1d", "heat_3d", "pme_solution_1d"])
def test_noalloc_matches_sd_residual_on_consecutive_calls(case):
    torch = pytest.importorskip("torch")
    if case == "heat_1d":
        dim, ne, lo, hi, p, scheme = 1, (37,), (0.0,), (1.0,), 5, "br1"
        phys = sd.Physics(kind="heat", nu=0.3)
        U = inputs.random_scalar(1, ne, p, seed=7)
    elif case == "heat_3d":
        # 3D scalar: one variable, its trace blocks padded with the diffusivity slots
        dim, ne, lo, hi, p, scheme = 3, (7, 5, 6), (0.0,) * 3, (TWO_PI,) * 3, 3, "compact"
        phys = sd.Physics(kind="heat", nu=0.01)
        U = inputs.heat_modes_3d(ne, p, seed=1)[0]
    elif case == "pme_solution_1d":
        # porous medium with the diffusivity at the solution points: the scalar trace
        # blocks carry the extra diffusivity traces
        dim, ne, lo, hi, p, scheme = 1, (64,), (-10.0,), (10.0,), 4, "compact"
        phys = sd.Physics(kind="pme", m_pme=2.0, pme_coef="solution")
        U = inputs.random_scalar(1, ne, p, seed=11, lo=0.1, hi=1.0)
    else:
        dim, ne, lo, hi, p = 3, (6, 5, 4), (0.0,) * 3, (TWO_PI,) * 3, 4
        scheme = "compact" if case == "ns_compact" else "br1"
        phys = sd.Physics(kind="ns")
        U = inputs.tgv_3d(ne, p, perturb_seed=3)
    Ug = torch.from_numpy(np.ascontiguousarray(U)).to("cuda", torch.float32)
    ctx = sd.SD(dim, ne, lo, hi, p, scheme, phys, "f32")
    ref = ctx.residual(Ug)
    torch.cuda.synchronize()
    ctx.close()
    scale = float(ref.abs().max())
    for _ in range(2):                      # two calls in a row reuse the static scratch
        R = torch.full_like(Ug, float("nan"))
        sd.sd_residual_f32_noalloc(dim, ne, lo, hi, p, scheme, phys, Ug, R)
        torch.cuda.synchronize()
        assert torch.isfinite(R).all()
        assert float((R - ref).abs().max()) <= 1e-6 * scale


@pytest.mark.gpu
def test_noalloc_wrapper_rejects_wrong_sizes_and_devices():
    # the binding checks the state size against the problem before any call: a tensor of
    # the wrong size (a scalar state for Navier-Stokes, or another p) never reaches the
    # kernels
    torch = pytest.importorskip("torch")
    ne, p = (4, 4, 4), 3
    phys = sd.Physics(kind="ns")
    good = 5 * 64 * (p + 1) ** 3
    U = torch.zeros(good, dtype=torch.float32, device="cuda")
    for bad in (good // 5, 5 * 64 * (p + 2) ** 3):
        V = torch.zeros(bad, dtype=torch.float32, device="cuda")
        with pytest.raises(ValueError):
            sd.sd_residual_f32_noalloc(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, "compact", phys, V, torch.empty_like(V))
        with pytest.raises(ValueError):
            sd.sd_residual_f32_noalloc(3, ne, (0.0,) * 3, (TWO_PI,) * 3, p, "compact", phys, U, V)
