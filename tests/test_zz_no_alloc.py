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


def test_oversize_grid_is_rejected_before_any_launch():
    # 16^3 elements at p = 4 (Navier-Stokes) need 8.6 Mi scratch values > 8 Mi: rejected on
    # the host, so no device is touched (the pointers are never dereferenced)
    build.build()
    lib = sd.load_library()
    m = _mesh(3, (16, 16, 16), (0.0,) * 3, (TWO_PI,) * 3)
    ph = sd.Physics(kind="ns").to_c()
    st = lib.sd_residual_f32_noalloc(ctypes.byref(m), 4, 1, ctypes.byref(ph),
                                     ctypes.c_void_p(256), ctypes.c_void_p(1 << 30), None)
    assert st == sd.SD_EINVAL
    assert b"static scratch" in lib.sd_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["ns_compact", "ns_br1", "heat_1d"])
def test_noalloc_matches_sd_residual_on_consecutive_calls(case):
    torch = pytest.importorskip("torch")
    if case == "heat_1d":
        dim, ne, lo, hi, p, scheme = 1, (37,), (0.0,), (1.0,), 5, "br1"
        phys = sd.Physics(kind="heat", nu=0.3)
        U = inputs.random_scalar(1, ne, p, seed=7)
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
