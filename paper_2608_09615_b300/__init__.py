"""Python binding of the B300 Spectral Difference residual library (include/sd.h).

Argument marshalling only: every step of the residual, the Runge-Kutta stages and the
diagnostics run in the CUDA library libsd.so that sits next to this file (built by
paper_2608_09615_b300.build). The library is loaded on first use; if it is missing the
call raises -- there is no CPU fallback.

Low-level functions carry the C names (sd_init, sd_residual, sd_residual_host,
sd_rk_step, sd_diagnostics, sd_destroy); the SD class wraps one context.
Tensors are torch tensors: device buffers for sd_residual / sd_rk_step / sd_diagnostics,
host (ideally pinned) buffers for sd_residual_host, all contiguous and laid out as
U[var][E_{dim-1}]...[E_0][n]...[n].
"""
import ctypes
import os
from dataclasses import dataclass, field

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsd.so")

SD_OK, SD_EINVAL, SD_ENOMEM, SD_ECUDA, SD_EUNSUPPORTED, SD_ENONFINITE, SD_ETIMEOUT = range(7)
SCHEMES = {"br1": 0, "compact": 1}
KINDS = {"heat": 0, "pme": 1, "ns": 2}
RIEMANN = {"roe": 0, "rusanov": 1}
VISCOUS_FLUX = {"a": 0, "b": 1}
PME_COEF = {"flux": 0, "solution": 1}
PRECISIONS = {"f64": 0, "f32": 1}
RK = {"rk4": 0, "ssprk54": 1, "lsrk54": 2}
RK_STAGES = {"f32": 0, "f64": 1}


class SDError(RuntimeError):
    def __init__(self, status, where, text):
        super().__init__("%s: status %d (%s)%s" % (where, status, text[0], (": " + text[1]) if text[1] else ""))
        self.status = status


class _Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ne", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class _Physics(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nu", ctypes.c_double), ("m_pme", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("Ma", ctypes.c_double), ("rho0", ctypes.c_double), ("u0", ctypes.c_double),
                ("L", ctypes.c_double), ("sutherland", ctypes.c_int), ("suth_s", ctypes.c_double),
                ("riemann", ctypes.c_int), ("harten", ctypes.c_double), ("eta_ip", ctypes.c_double),
                ("viscous_flux", ctypes.c_int), ("pme_coef", ctypes.c_int)]


class _Diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("ke", ctypes.c_double), ("ke_rho", ctypes.c_double),
                ("enstrophy", ctypes.c_double), ("mass", ctypes.c_double),
                ("mom", ctypes.c_double * 3), ("energy", ctypes.c_double),
                ("l2sq", ctypes.c_double), ("volume", ctypes.c_double), ("nonfinite", ctypes.c_int)]


EXPORTS = ("sd_init", "sd_destroy", "sd_set_stream", "sd_state_size", "sd_nvar", "sd_points",
           "sd_residual", "sd_residual_host", "sd_rk_step", "sd_diagnostics", "sd_status_str",
           "sd_last_error", "sd_profile_enable", "sd_profile_read", "sd_launch_count",
           "sd_mlp_param_count", "sd_mlp_cast", "sd_mlp_forward", "sd_mlp_loss", "sd_mlp_backward",
           "sd_mlp_adam", "sd_residual_f32_noalloc", "sd_set_flux_tau", "sd_closure_data",
           "sd_filter_matrix", "sd_filter_project", "sd_closure_targets", "sd_colstats",
           "sd_standardise", "sd_unstandardise", "sd_closure_enable", "sd_init_curvilinear",
           "sd_is_curvilinear", "sd_set_rk_stages", "sd_measure_fp32_peak", "sd_rk_prepare",
           "sd_rk_stage", "sd_pack_elements", "sd_unpack_elements", "sd_face_gradient_size",
           "sd_pack_face_gradients", "sd_unpack_face_gradients", "sd_residual_begin",
           "sd_residual_end", "sd_set_owned_box")
KERNEL_CLASSES = ("trace", "grad", "flux_div", "other", "face")

_lib_handle = None


def load_library(path=LIB_PATH):
    """Load libsd.so (raises if it is missing: build it with paper_2608_09615_b300.build)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing; run `python -m paper_2608_09615_b300.build`"
                           % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.sd_init.argtypes = [ctypes.POINTER(_Mesh), I, I, ctypes.POINTER(_Physics), I, P,
                            ctypes.POINTER(P)]
    lib.sd_init.restype = I
    lib.sd_init_curvilinear.argtypes = [ctypes.POINTER(_Mesh), P, I, I, ctypes.POINTER(_Physics), I, P,
                                        ctypes.POINTER(P)]
    lib.sd_init_curvilinear.restype = I
    lib.sd_is_curvilinear.argtypes = [P]
    lib.sd_is_curvilinear.restype = I
    lib.sd_destroy.argtypes = [P]
    lib.sd_destroy.restype = None
    lib.sd_set_stream.argtypes = [P, P]
    lib.sd_set_stream.restype = I
    lib.sd_state_size.argtypes = [P]
    lib.sd_state_size.restype = S
    lib.sd_nvar.argtypes = [P]
    lib.sd_nvar.restype = I
    lib.sd_points.argtypes = [P, P, P]
    lib.sd_points.restype = I
    lib.sd_residual.argtypes = [P, P, P]
    lib.sd_residual.restype = I
    lib.sd_residual_host.argtypes = [P, P, P]
    lib.sd_residual_host.restype = I
    lib.sd_rk_step.argtypes = [P, P, D, D, I]
    lib.sd_rk_step.restype = I
    lib.sd_rk_prepare.argtypes = [P, P, ctypes.POINTER(P)]
    lib.sd_rk_prepare.restype = I
    lib.sd_rk_stage.argtypes = [P, P, I, D, I, ctypes.POINTER(P)]
    lib.sd_rk_stage.restype = I
    lib.sd_pack_elements.argtypes = [P, P, I, P, I, P]
    lib.sd_pack_elements.restype = I
    lib.sd_unpack_elements.argtypes = [P, P, I, P, I, P]
    lib.sd_unpack_elements.restype = I
    lib.sd_face_gradient_size.argtypes = [P]
    lib.sd_face_gradient_size.restype = S
    lib.sd_pack_face_gradients.argtypes = [P, P, P, I, P]
    lib.sd_pack_face_gradients.restype = I
    lib.sd_unpack_face_gradients.argtypes = [P, P, P, P, I]
    lib.sd_unpack_face_gradients.restype = I
    lib.sd_residual_begin.argtypes = [P, P]
    lib.sd_residual_begin.restype = I
    lib.sd_residual_end.argtypes = [P, P, P]
    lib.sd_residual_end.restype = I
    lib.sd_set_owned_box.argtypes = [P, P, P]
    lib.sd_set_owned_box.restype = I
    lib.sd_measure_fp32_peak.argtypes = [I, P]
    lib.sd_measure_fp32_peak.restype = I
    lib.sd_set_rk_stages.argtypes = [P, I]
    lib.sd_set_rk_stages.restype = I
    lib.sd_diagnostics.argtypes = [P, P, D, ctypes.POINTER(_Diag)]
    lib.sd_diagnostics.restype = I
    lib.sd_status_str.argtypes = [I]
    lib.sd_status_str.restype = ctypes.c_char_p
    lib.sd_last_error.argtypes = []
    lib.sd_last_error.restype = ctypes.c_char_p
    lib.sd_profile_enable.argtypes = [P, I]
    lib.sd_profile_enable.restype = I
    lib.sd_profile_read.argtypes = [P, P, P]
    lib.sd_profile_read.restype = I
    lib.sd_launch_count.argtypes = [P]
    lib.sd_launch_count.restype = ctypes.c_longlong
    lib.sd_mlp_param_count.argtypes = []
    lib.sd_mlp_param_count.restype = I
    lib.sd_mlp_cast.argtypes = [P, P, P]
    lib.sd_mlp_cast.restype = I
    lib.sd_mlp_forward.argtypes = [P, I, P, P, P, P, P]
    lib.sd_mlp_forward.restype = I
    lib.sd_mlp_loss.argtypes = [P, P, I, P, P, P, P]
    lib.sd_mlp_loss.restype = I
    lib.sd_mlp_backward.argtypes = [P, P, P, I, P, P, P, P]
    lib.sd_mlp_backward.restype = I
    lib.sd_mlp_adam.argtypes = [P, P, P, P, P, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, P]
    lib.sd_mlp_adam.restype = I
    lib.sd_residual_f32_noalloc.argtypes = [ctypes.POINTER(_Mesh), I, I, ctypes.POINTER(_Physics),
                                            P, P, P]
    lib.sd_residual_f32_noalloc.restype = I
    lib.sd_set_flux_tau.argtypes = [P, P]
    lib.sd_set_flux_tau.restype = I
    lib.sd_closure_data.argtypes = [P, P, P, P]
    lib.sd_closure_data.restype = I
    lib.sd_filter_matrix.argtypes = [I, I, I, P]
    lib.sd_filter_matrix.restype = I
    lib.sd_filter_project.argtypes = [P, P, P, I, P, I, I, I, P]
    lib.sd_filter_project.restype = I
    lib.sd_closure_targets.argtypes = [P, P, P, P, I, P]
    lib.sd_closure_targets.restype = I
    lib.sd_colstats.argtypes = [P, I, I, P, P, P]
    lib.sd_colstats.restype = I
    lib.sd_standardise.argtypes = [P, I, I, P, P, P, P, P]
    lib.sd_standardise.restype = I
    lib.sd_unstandardise.argtypes = [P, I, I, P, P, P, P]
    lib.sd_unstandardise.restype = I
    lib.sd_closure_enable.argtypes = [P, P, P, P, P, P, P]
    lib.sd_closure_enable.restype = I
    _lib_handle = lib
    return lib


def measure_fp32_peak(packed=False):
    """Measured FP32 FMA throughput of the current device, TFLOP/s (sd_measure_fp32_peak)."""
    out = ctypes.c_double()
    _check(load_library().sd_measure_fp32_peak(int(bool(packed)), ctypes.byref(out)), "sd_measure_fp32_peak")
    return out.value


def _check(status, where):
    if status != SD_OK:
        lib = load_library()
        raise SDError(status, where, (lib.sd_status_str(status).decode(), lib.sd_last_error().decode()))


@dataclass
class Physics:
    """sd_physics. kind: "heat", "pme" or "ns"; NS defaults are the Taylor-Green setup."""
    kind: str = "ns"
    nu: float = 1.0
    m_pme: float = 2.0
    gamma: float = 1.4
    Pr: float = 0.71
    Re: float = 1600.0
    Ma: float = 0.1
    rho0: float = 1.0
    u0: float = 1.0
    L: float = 1.0
    sutherland: bool = True
    suth_s: float = 110.4 / 300.0
    riemann: str = "roe"
    harten: float = 0.1
    eta_ip: float = 0.0
    viscous_flux: str = "a"         # interface viscous flux, Sec. 2.1 step 4: option "a" or "b"
    pme_coef: str = "flux"          # porous-medium diffusivity at the "flux" or "solution" points

    def to_c(self):
        return _Physics(KINDS[self.kind], self.nu, self.m_pme, self.gamma, self.Pr, self.Re,
                        self.Ma, self.rho0, self.u0, self.L, int(bool(self.sutherland)),
                        self.suth_s, RIEMANN[self.riemann], self.harten, self.eta_ip,
                        VISCOUS_FLUX[self.viscous_flux], PME_COEF[self.pme_coef])


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def sd_init(dim, ne, lo, hi, p, scheme, physics, precision, stream=None):
    """Create a context (sd_init). Returns an opaque handle (c_void_p)."""
    lib = load_library()
    ne = list(ne) + [1] * (3 - len(ne))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    m = _Mesh(dim, (ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi))
    ph = physics.to_c()
    out = ctypes.c_void_p()
    st = lib.sd_init(ctypes.byref(m), int(p), SCHEMES[scheme], ctypes.byref(ph),
                     PRECISIONS[precision], _stream_handle(stream), ctypes.byref(out))
    _check(st, "sd_init")
    return out


def sd_init_curvilinear(nodes, p, scheme, physics, precision, stream=None):
    """Create a context on a periodic grid of trilinear hexahedra (sd_init_curvilinear).
    nodes: array (3, nz+1, ny+1, nx+1) of corner-node coordinates, the last node along each
    axis being the periodic image of the first. Returns an opaque handle (c_void_p)."""
    import numpy as np
    lib = load_library()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    if nodes.ndim != 4 or nodes.shape[0] != 3 or min(nodes.shape[1:]) < 2:
        raise ValueError("nodes must have shape (3, nz+1, ny+1, nx+1)")
    ne = [nodes.shape[3] - 1, nodes.shape[2] - 1, nodes.shape[1] - 1]
    m = _Mesh(3, (ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(0.0, 0.0, 0.0),
              (ctypes.c_double * 3)(1.0, 1.0, 1.0))
    ph = physics.to_c()
    out = ctypes.c_void_p()
    st = lib.sd_init_curvilinear(ctypes.byref(m), ctypes.c_void_p(nodes.ctypes.data), int(p), SCHEMES[scheme],
                                 ctypes.byref(ph), PRECISIONS[precision], _stream_handle(stream),
                                 ctypes.byref(out))
    _check(st, "sd_init_curvilinear")
    return out


def sd_residual_f32_noalloc(dim, ne, lo, hi, p, scheme, physics, U, R, stream=None):
    """FP32 residual through the allocation-free entry point (no context, no device
    allocation; the library's static scratch is shared by all calls). U, R: contiguous
    CUDA float32 tensors on one device, each holding the nvar * prod(ne) * (p+1)^dim values
    of the state layout. The call runs on U's device."""
    import torch
    for t, nm in ((U, "U"), (R, "R")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or \
                not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA float32 tensor" % nm)
    if U.device != R.device:
        raise ValueError("U and R must be on the same device")
    ne = list(ne) + [1] * (3 - len(ne))
    nelem = 1
    for d in range(dim):
        nelem *= int(ne[d])
    nvar = 5 if physics.kind == "ns" else 1
    expect = nvar * nelem * (int(p) + 1) ** int(dim)
    for t, nm in ((U, "U"), (R, "R")):
        if t.numel() != expect:
            raise ValueError("%s must hold %d values (nvar %d, %d elements, p = %d), not %d"
                             % (nm, expect, nvar, nelem, p, t.numel()))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    m = _Mesh(dim, (ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi))
    ph = physics.to_c()
    with torch.cuda.device(U.device):
        st = load_library().sd_residual_f32_noalloc(ctypes.byref(m), int(p), SCHEMES[scheme],
                                                    ctypes.byref(ph), ctypes.c_void_p(U.data_ptr()),
                                                    ctypes.c_void_p(R.data_ptr()), _stream_handle(stream))
    _check(st, "sd_residual_f32_noalloc")
    return R


def sd_destroy(ctx):
    load_library().sd_destroy(ctx)


def _dev_ptr(t, dtype, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s must be a contiguous %s tensor of %d values" % (name, dtype, numel))
    return ctypes.c_void_p(t.data_ptr())


def sd_residual(ctx, U, R, dtype, numel):
    _check(load_library().sd_residual(ctx, _dev_ptr(U, dtype, numel, "U"),
                                      _dev_ptr(R, dtype, numel, "R")), "sd_residual")


def sd_residual_host(ctx, U, R, dtype, numel):
    import torch
    for t, nm in ((U, "U"), (R, "R")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype or \
                not t.is_contiguous() or t.numel() != numel:
            raise ValueError("%s must be a contiguous host %s tensor of %d values" % (nm, dtype, numel))
    _check(load_library().sd_residual_host(ctx, ctypes.c_void_p(U.data_ptr()),
                                           ctypes.c_void_p(R.data_ptr())), "sd_residual_host")


def sd_rk_step(ctx, U64, t, dt, rk, numel):
    import torch
    _check(load_library().sd_rk_step(ctx, _dev_ptr(U64, torch.float64, numel, "U64"),
                                     float(t), float(dt), RK[rk]), "sd_rk_step")


def sd_diagnostics(ctx, U64, t, numel, raise_nonfinite=True):
    import torch
    d = _Diag()
    st = load_library().sd_diagnostics(ctx, _dev_ptr(U64, torch.float64, numel, "U64"), float(t),
                                       ctypes.byref(d))
    if st != SD_ENONFINITE or raise_nonfinite:
        _check(st, "sd_diagnostics")
    return dict(t=d.t, ke=d.ke, ke_rho=d.ke_rho, enstrophy=d.enstrophy, mass=d.mass,
                mom=[d.mom[0], d.mom[1], d.mom[2]], energy=d.energy, l2sq=d.l2sq,
                volume=d.volume, nonfinite=d.nonfinite)


class SD:
    """One SD residual context (grid, p, scheme, physics, residual precision)."""

    def __init__(self, dim, ne, lo, hi, p, scheme="compact", physics=None, precision="f32",
                 stream=None, nodes=None):
        """nodes: optional corner nodes (3, nz+1, ny+1, nx+1) of a periodic grid of
        trilinear hexahedra (then dim must be 3, ne must match the nodes, lo / hi are
        ignored); without it the grid is the uniform Cartesian box [lo, hi)."""
        import torch
        self.physics = physics if physics is not None else Physics()
        self.dim, self.ne, self.p, self.n = dim, tuple(ne), p, p + 1
        self.scheme, self.precision = scheme, precision
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        if nodes is not None:
            if dim != 3 or tuple(ne) != (nodes.shape[3] - 1, nodes.shape[2] - 1, nodes.shape[1] - 1):
                raise ValueError("a curvilinear grid needs dim = 3 and ne matching the nodes")
            self._ctx = sd_init_curvilinear(nodes, p, scheme, self.physics, precision, stream)
        else:
            self._ctx = sd_init(dim, ne, lo, hi, p, scheme, self.physics, precision, stream)
        lib = load_library()
        self.numel = int(lib.sd_state_size(self._ctx))
        self.nvar = int(lib.sd_nvar(self._ctx))
        self.shape = (self.nvar,) + tuple(reversed(tuple(ne))) + (self.n,) * dim

    @classmethod
    def curvilinear(cls, nodes, p, scheme="compact", physics=None, precision="f32", stream=None):
        """Context on the periodic trilinear-hexahedron grid with corner nodes `nodes`."""
        ne = (nodes.shape[3] - 1, nodes.shape[2] - 1, nodes.shape[1] - 1)
        return cls(3, ne, (0.0,) * 3, (1.0,) * 3, p, scheme, physics, precision, stream, nodes=nodes)

    @property
    def curved(self):
        return bool(load_library().sd_is_curvilinear(self._ctx))

    def set_stream(self, stream):
        _check(load_library().sd_set_stream(self._ctx, _stream_handle(stream)), "sd_set_stream")

    def points(self):
        xi = (ctypes.c_double * self.n)()
        w = (ctypes.c_double * self.n)()
        _check(load_library().sd_points(self._ctx, xi, w), "sd_points")
        return list(xi), list(w)

    def residual(self, U, R=None):
        import torch
        if R is None:
            R = torch.empty_like(U)
        sd_residual(self._ctx, U, R, self.dtype, self.numel)
        return R

    def residual_host(self, U, R):
        sd_residual_host(self._ctx, U, R, self.dtype, self.numel)
        return R

    def rk_step(self, U64, t, dt, rk="ssprk54"):
        sd_rk_step(self._ctx, U64, t, dt, rk, self.numel)

    def set_owned_box(self, lo, hi):
        """Restrict the diagnostics to the elements [lo, hi) per axis (a sub-domain's owned
        block); None removes the restriction."""
        if lo is None:
            _check(load_library().sd_set_owned_box(self._ctx, None, None), "sd_set_owned_box")
            return
        a = (ctypes.c_int * 3)(*lo)
        b = (ctypes.c_int * 3)(*hi)
        _check(load_library().sd_set_owned_box(self._ctx, a, b), "sd_set_owned_box")

    def set_rk_stages(self, mode):
        """Stage arithmetic of rk_step on an FP32 context: "f32" (FP32 stage increments, the
        default) or "f64" (FP64 stage states; allocates three FP64 registers once)."""
        _check(load_library().sd_set_rk_stages(self._ctx, RK_STAGES[mode]), "sd_set_rk_stages")

    def diagnostics(self, U64, t=0.0, raise_nonfinite=True):
        return sd_diagnostics(self._ctx, U64, t, self.numel, raise_nonfinite)

    def profile(self, on=True):
        _check(load_library().sd_profile_enable(self._ctx, int(bool(on))), "sd_profile_enable")

    def profile_read(self):
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        cnt = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        _check(load_library().sd_profile_read(self._ctx, ms, cnt), "sd_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def launch_count(self):
        return int(load_library().sd_launch_count(self._ctx))

    # ---- closure data path (Navier-Stokes)
    def set_flux_tau(self, tau):
        """tau: CUDA float32 tensor (nelem, 15) or None: extra per-element flux."""
        self._tau = tau
        _check(load_library().sd_set_flux_tau(self._ctx, None if tau is None else _ptr(tau)),
               "sd_set_flux_tau")

    def closure_data(self, U, features=True, means=True):
        """Features (nelem, 64) float32 and/or flux means (nelem, 15) float64 of state U."""
        import torch
        E = self.numel // (self.nvar * self.n ** self.dim)
        X = torch.empty(E, 64, dtype=torch.float32, device="cuda") if features else None
        Mn = torch.empty(E, 15, dtype=torch.float64, device="cuda") if means else None
        _check(load_library().sd_closure_data(self._ctx, _dev_ptr(U, self.dtype, self.numel, "U"),
                                              None if X is None else _ptr(X),
                                              None if Mn is None else _ptr(Mn)), "sd_closure_data")
        return X, Mn

    def closure_enable(self, net, mu_x, sig_x, mu_t, sig_t):
        """Attach a trained MLP (sd.MLP) with its standardisation statistics."""
        self._closure_refs = (net, mu_x, sig_x, mu_t, sig_t)
        _check(load_library().sd_closure_enable(self._ctx, _ptr(net.Wb), _ptr(net.P), _ptr(mu_x),
                                                _ptr(sig_x), _ptr(mu_t), _ptr(sig_t)),
               "sd_closure_enable")

    def closure_disable(self):
        _check(load_library().sd_closure_enable(self._ctx, None, None, None, None, None, None),
               "sd_closure_enable")
        self._closure_refs = None

    def close(self):
        if getattr(self, "_ctx", None) is not None:
            sd_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- MLP closure network
MLP_IN, MLP_HID, MLP_OUT = 64, 128, 15


def mlp_layout():
    """Offsets of the packed parameter vector (W1, b1, W2, b2, W3 with a zero 16th row,
    b3 with a zero 16th entry)."""
    off = {}
    o = 0
    for name, size in (("W1", 128 * 64), ("b1", 128), ("W2", 128 * 128), ("b2", 128),
                       ("W3", 16 * 128), ("b3", 16)):
        off[name] = (o, size)
        o += size
    return off, o


class MLP:
    """Device state of the 64-128-128-15 closure network: FP32 master parameters, Adam
    moments, the BF16 weight copy the kernels read, gradient buffers."""

    def __init__(self, params=None, max_rows=4096, stream=None):
        import torch
        lib = load_library()
        self.n = int(lib.sd_mlp_param_count())
        off, total = mlp_layout()
        assert total == self.n
        self.off = off
        self.P = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        if params is not None:
            self.set_params(params)
        self.m1 = torch.zeros_like(self.P)
        self.m2 = torch.zeros_like(self.P)
        self.grad = torch.zeros_like(self.P)
        self.Wb = torch.zeros(self.n, dtype=torch.bfloat16, device="cuda")
        self.max_rows = 0
        self.step = 0
        self.stream = stream
        self._ensure(max_rows)
        self.cast()

    def _s(self):
        return _stream_handle(self.stream)

    def _ensure(self, M):
        import torch
        if M <= self.max_rows:
            return
        self.max_rows = M
        nb = (M + 63) // 64
        self.H = torch.empty(2 * M * 128, dtype=torch.bfloat16, device="cuda")
        self.Y = torch.empty(M * MLP_OUT, dtype=torch.float32, device="cuda")
        self.dY = torch.empty_like(self.Y)
        self.part = torch.empty(nb * self.n, dtype=torch.float32, device="cuda")
        self.lpart = torch.empty(64, dtype=torch.float64, device="cuda")
        self.loss = torch.empty(1, dtype=torch.float64, device="cuda")

    def set_params(self, params):
        """params: list of (W, b) numpy arrays as in oracle.mlp (W of shape (out, in))."""
        import numpy as np
        import torch
        flat = np.zeros(self.n, dtype=np.float32)
        for (W, b), wn, bn in zip(params, ("W1", "W2", "W3"), ("b1", "b2", "b3")):
            o, _ = self.off[wn]
            flat[o:o + W.size] = np.asarray(W, dtype=np.float32).reshape(-1)
            o, _ = self.off[bn]
            flat[o:o + b.size] = np.asarray(b, dtype=np.float32)
        self.P.copy_(torch.from_numpy(flat))

    def get_params(self):
        import numpy as np
        flat = self.P.cpu().numpy()
        out = []
        for wn, bn, shp in (("W1", "b1", (128, 64)), ("W2", "b2", (128, 128)), ("W3", "b3", (15, 128))):
            o, _ = self.off[wn]
            W = flat[o:o + shp[0] * shp[1]].reshape(shp).copy()
            o, _ = self.off[bn]
            out.append((W, flat[o:o + shp[0]].copy()))
        return out

    def cast(self):
        _check(load_library().sd_mlp_cast(_ptr(self.P), _ptr(self.Wb), self._s()), "sd_mlp_cast")

    def forward(self, Xb):
        """Xb: CUDA bfloat16 tensor (M, 64). Returns Y (M, 15) float32 (a view of the
        internal buffer) and keeps the activation cache for backward()."""
        M = int(Xb.shape[0])
        self._ensure(M)
        self.M = M
        self.Xb = Xb.contiguous()
        _check(load_library().sd_mlp_forward(_ptr(self.Xb), M, _ptr(self.Wb), _ptr(self.P),
                                             _ptr(self.Y), _ptr(self.H), self._s()), "sd_mlp_forward")
        return self.Y[:M * MLP_OUT].view(M, MLP_OUT)

    def loss_backward(self, T):
        """MSE loss against T (M, 15) float32 and the parameter gradient (self.grad)."""
        M = self.M
        T = T.contiguous()
        lib = load_library()
        _check(lib.sd_mlp_loss(_ptr(self.Y), _ptr(T), M, _ptr(self.dY), _ptr(self.lpart),
                               _ptr(self.loss), self._s()), "sd_mlp_loss")
        _check(lib.sd_mlp_backward(_ptr(self.Xb), _ptr(self.H), _ptr(self.dY), M, _ptr(self.Wb),
                                   _ptr(self.part), _ptr(self.grad), self._s()), "sd_mlp_backward")
        return self.loss

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        _check(load_library().sd_mlp_adam(_ptr(self.P), _ptr(self.m1), _ptr(self.m2), _ptr(self.grad),
                                          _ptr(self.Wb), self.step, lr, b1, b2, eps, self._s()),
               "sd_mlp_adam")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class DevicePointer:
    """A device array owned by a context (a Runge-Kutta stage input), usable wherever a
    tensor's data_ptr() is read."""

    def __init__(self, ptr):
        self.ptr = int(ptr or 0)

    def data_ptr(self):
        return self.ptr


# ---------------------------------------------------------------- sub-domain primitives
def _idx_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA int32 tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _elem_values(ctx):
    return ctx.nvar * ctx.n ** ctx.dim


def _state_dtype(ctx, U):
    import torch
    dt = getattr(U, "dtype", None)
    if dt is None:
        return ctx.dtype                 # a context-owned stage input: the residual precision
    if dt not in (torch.float32, torch.float64) or not U.is_cuda or not U.is_contiguous() or \
            U.numel() != ctx.numel:
        raise ValueError("U must be a contiguous CUDA float32/float64 state of %d values" % ctx.numel)
    return dt


def pack_elements(ctx, U, elems):
    """Whole elements `elems` (local indices, CUDA int32) of the state U (a tensor of either
    precision, or a context-owned stage input) gathered into a new buffer
    [nvar][len(elems)][n^dim] (sd_pack_elements)."""
    import torch
    dt = _state_dtype(ctx, U)
    buf = torch.empty(len(elems) * _elem_values(ctx), dtype=dt, device="cuda")
    _check(load_library().sd_pack_elements(ctx._ctx, ctypes.c_void_p(U.data_ptr()), buf.element_size(),
                                           _idx_ptr(elems, "elems"), len(elems), _ptr(buf)), "sd_pack_elements")
    return buf


def unpack_elements(ctx, buf, elems, U):
    """The inverse of pack_elements: buf written into elements `elems` of U."""
    dt = _state_dtype(ctx, U)
    if buf.numel() != len(elems) * _elem_values(ctx) or buf.dtype != dt:
        raise ValueError("buffer does not match the element list")
    _check(load_library().sd_unpack_elements(ctx._ctx, _ptr(buf), buf.element_size(), _idx_ptr(elems, "elems"),
                                             len(elems), ctypes.c_void_p(U.data_ptr())), "sd_unpack_elements")


def pack_face_gradients(ctx, elems, faces):
    """Face blocks (elems[k], faces[k]) of the context's interface-gradient buffer."""
    import torch
    g = int(load_library().sd_face_gradient_size(ctx._ctx))
    buf = torch.empty(len(elems) * g, dtype=ctx.dtype, device="cuda")
    _check(load_library().sd_pack_face_gradients(ctx._ctx, _idx_ptr(elems, "elems"), _idx_ptr(faces, "faces"),
                                                 len(elems), _ptr(buf)), "sd_pack_face_gradients")
    return buf


def unpack_face_gradients(ctx, buf, elems, faces):
    g = int(load_library().sd_face_gradient_size(ctx._ctx))
    if buf.numel() != len(elems) * g or buf.dtype != ctx.dtype:
        raise ValueError("buffer does not match the face list")
    _check(load_library().sd_unpack_face_gradients(ctx._ctx, _ptr(buf), _idx_ptr(elems, "elems"),
                                                   _idx_ptr(faces, "faces"), len(elems)),
           "sd_unpack_face_gradients")


def residual_begin(ctx, U):
    """Traces and own interface gradients of U (the first half of sd_residual)."""
    _check(load_library().sd_residual_begin(ctx._ctx, _dev_ptr(U, ctx.dtype, ctx.numel, "U")),
           "sd_residual_begin")


def residual_end(ctx, U, R):
    """Interface fluxes and divergence (the second half of sd_residual)."""
    _check(load_library().sd_residual_end(ctx._ctx, _dev_ptr(U, ctx.dtype, ctx.numel, "U"),
                                          _dev_ptr(R, ctx.dtype, ctx.numel, "R")), "sd_residual_end")


def rk_prepare(ctx, U64):
    """First stage input of a Runge-Kutta step of U64 (sd_rk_prepare); returns it."""
    import torch
    out = ctypes.c_void_p()
    _check(load_library().sd_rk_prepare(ctx._ctx, _dev_ptr(U64, torch.float64, ctx.numel, "U64"),
                                        ctypes.byref(out)), "sd_rk_prepare")
    return DevicePointer(out.value)


def rk_stage(ctx, U64, k, dt, rk="ssprk54"):
    """Stage k of the step (sd_rk_stage); returns the next stage input (None after the last)."""
    import torch
    out = ctypes.c_void_p()
    _check(load_library().sd_rk_stage(ctx._ctx, _dev_ptr(U64, torch.float64, ctx.numel, "U64"), int(k),
                                      float(dt), RK[rk], ctypes.byref(out)), "sd_rk_stage")
    return DevicePointer(out.value) if out.value else None


def filter_matrix(pf, pc, r):
    """Host copy (numpy) of the 1D fine -> coarse L2 projection of sd_filter_matrix."""
    import numpy as np
    P = np.zeros(((pc + 1), r * (pf + 1)), dtype=np.float64)
    _check(load_library().sd_filter_matrix(pf, pc, r, P.ctypes.data_as(ctypes.c_void_p)),
           "sd_filter_matrix")
    return P


def filter_project(Uf, ne_coarse, r, pf, pc, Pdev=None, stream=None):
    """Box filter of the fine FP64 CUDA state Uf onto the nested coarse grid (FP64 out)."""
    import numpy as np
    import torch
    if Pdev is None:
        Pdev = torch.from_numpy(filter_matrix(pf, pc, r)).cuda()
    nv = int(Uf.shape[0])
    Ec = int(np.prod(ne_coarse))
    Uc = torch.empty((nv,) + tuple(reversed(tuple(ne_coarse))) + (pc + 1,) * 3, dtype=torch.float64,
                     device="cuda")
    nec = (ctypes.c_int * 3)(*ne_coarse)
    _check(load_library().sd_filter_project(_ptr(Uf), _ptr(Uc), _ptr(Pdev), nv, nec, r, pf + 1, pc + 1,
                                            _stream_handle(stream)), "sd_filter_project")
    del Ec
    return Uc


def closure_targets(fine_means, coarse_means, ne_coarse, r, stream=None):
    import torch
    tau = torch.empty(coarse_means.shape[0], 15, dtype=torch.float32, device="cuda")
    nec = (ctypes.c_int * 3)(*ne_coarse)
    _check(load_library().sd_closure_targets(_ptr(fine_means), _ptr(coarse_means), _ptr(tau), nec, r,
                                             _stream_handle(stream)), "sd_closure_targets")
    return tau


def colstats(A, stream=None):
    import torch
    rows, cols = A.shape
    mu = torch.empty(cols, dtype=torch.float32, device="cuda")
    sg = torch.empty(cols, dtype=torch.float32, device="cuda")
    _check(load_library().sd_colstats(_ptr(A), rows, cols, _ptr(mu), _ptr(sg), _stream_handle(stream)),
           "sd_colstats")
    return mu, sg


def standardise(A, mu, sigma, bf16=False, stream=None):
    import torch
    rows, cols = A.shape
    out = torch.empty(rows, cols, dtype=torch.bfloat16 if bf16 else torch.float32, device="cuda")
    _check(load_library().sd_standardise(_ptr(A), rows, cols, _ptr(mu), _ptr(sigma),
                                         _ptr(out) if bf16 else None, None if bf16 else _ptr(out),
                                         _stream_handle(stream)), "sd_standardise")
    return out
