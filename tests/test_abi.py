"""CPU checks of the C ABI: libsd.so builds, loads, exports every function include/sd.h
declares, and rejects bad arguments on the host before any device work."""
import ctypes
import os
import re

import pytest

import paper_2608_09615_b300 as sd
from paper_2608_09615_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sd.load_library()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(\w+)\s*\(", text):
            name = m.group(1)
            if name.startswith("sd_") and not name.endswith("_t"):
                names.add(name)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"sd_init", "sd_residual", "sd_rk_step", "sd_diagnostics"} <= names
    for name in names:
        assert hasattr(lib, name), name
    assert set(sd.EXPORTS) <= names


def test_status_strings(lib):
    assert lib.sd_status_str(0) == b"ok"
    assert lib.sd_status_str(4) == b"unsupported configuration"


def _init(lib, dim=3, ne=(2, 2, 2), p=3, kind="heat", scheme=1, prec=1, **kw):
    m = sd._Mesh(dim, (ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(0, 0, 0),
                 (ctypes.c_double * 3)(1, 1, 1))
    ph = sd.Physics(kind=kind, **kw).to_c()
    out = ctypes.c_void_p()
    st = lib.sd_init(ctypes.byref(m), p, scheme, ctypes.byref(ph), prec, None, ctypes.byref(out))
    return st, out


def test_host_validation(lib):
    assert _init(lib, p=0)[0] == sd.SD_EUNSUPPORTED
    assert _init(lib, p=9)[0] == sd.SD_EUNSUPPORTED
    assert _init(lib, dim=2)[0] == sd.SD_EUNSUPPORTED
    assert _init(lib, dim=1, kind="ns")[0] == sd.SD_EUNSUPPORTED
    assert _init(lib, ne=(0, 2, 2))[0] == sd.SD_EINVAL
    assert _init(lib, scheme=7)[0] == sd.SD_EINVAL
    assert _init(lib, prec=5)[0] == sd.SD_EINVAL
    assert _init(lib, kind="ns", Ma=0.0)[0] == sd.SD_EINVAL
    assert _init(lib, kind="pme", m_pme=0.5)[0] == sd.SD_EINVAL
    assert lib.sd_residual(None, None, None) == sd.SD_EINVAL
    assert lib.sd_rk_step(None, None, 0.0, 1.0, 0) == sd.SD_EINVAL
    assert lib.sd_diagnostics(None, None, 0.0, None) == sd.SD_EINVAL
    assert b"null" in lib.sd_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.reload(sd)
    try:
        mod._lib_handle = None
        with pytest.raises(RuntimeError, match="missing"):
            mod.load_library(str(tmp_path / "absent.so"))
    finally:
        mod._lib_handle = None
