"""Python binding of libld (include/ld.h): argument marshalling only.

Every function named ``ld_*`` here calls the C function of the same name
through ctypes with raw device pointers taken from torch tensors; all
arithmetic of the lattice-Boltzmann step runs in the library's CUDA kernels.
PyTorch supplies device memory (the workspace, checkpoints, inputs and
outputs) and the CUDA stream. There is no CPU fallback: if libld.so cannot be
built or loaded, every call raises.

``LdSim`` bundles a context with its torch-owned workspace for convenience.
"""

from __future__ import annotations

import contextlib
import ctypes
import threading

import torch

from . import build as _build

LD_FP64, LD_FP32, LD_FP16DEV, LD_BF16DEV = 0, 1, 2, 3
LD_KERNEL_AUTO, LD_KERNEL_GENERIC, LD_KERNEL_FUSED, LD_KERNEL_FUSED_STAGED = 0, 1, 2, 3
LD_OK, LD_EINVAL, LD_ECUDA, LD_ENONFINITE, LD_ESTATE = 0, -1, -2, -3, -4

PRECISIONS = {"fp64": LD_FP64, "fp32": LD_FP32, "fp16dev": LD_FP16DEV, "bf16dev": LD_BF16DEV}
KERNELS = {"auto": LD_KERNEL_AUTO, "generic": LD_KERNEL_GENERIC, "fused": LD_KERNEL_FUSED,
           "fused_staged": LD_KERNEL_FUSED_STAGED}
STORE_BYTES = {LD_FP64: 8, LD_FP32: 4, LD_FP16DEV: 2, LD_BF16DEV: 2}
LD_STENCIL_7, LD_STENCIL_19 = 0, 1
STENCILS = {7: LD_STENCIL_7, 19: LD_STENCIL_19}
LD_FORCE_POTENTIAL, LD_FORCE_STRESS = 0, 1
FORCES = {"potential": LD_FORCE_POTENTIAL, "stress": LD_FORCE_STRESS}
LD_COLLISION_BGK, LD_COLLISION_TRT = 0, 1
COLLISIONS = {"bgk": LD_COLLISION_BGK, "trt": LD_COLLISION_TRT}
LD_ROUND_NEAREST, LD_ROUND_STOCHASTIC = 0, 1
ROUNDINGS = {"nearest": LD_ROUND_NEAREST, "stochastic": LD_ROUND_STOCHASTIC}
Q = 19


class LdParams(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("B", ctypes.c_double), ("kappa", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
                ("rho0", ctypes.c_double), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("stencil", ctypes.c_int), ("force", ctypes.c_int), ("collision", ctypes.c_int),
                ("magic", ctypes.c_double), ("rounding", ctypes.c_int), ("seed", ctypes.c_uint64)]


class LcParams(ctypes.Structure):
    _fields_ = [("A0", ctypes.c_double), ("gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("xi", ctypes.c_double), ("tau_f", ctypes.c_double),
                ("rho0", ctypes.c_double), ("precision", ctypes.c_int), ("kernel", ctypes.c_int)]


class LdError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where} failed ({code}): {message}")
        self.code = code


_lock = threading.Lock()
_lib = None

# Signatures of every exported entry point (include/ld.h).
_VP = ctypes.c_void_p
_SIGNATURES = {
    "ld_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(LdParams)]),
    "ld_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(LdParams), _VP,
                                 ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "ld_destroy": (ctypes.c_int, [_VP]),
    "ld_set_stream": (ctypes.c_int, [_VP, _VP]),
    "ld_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(LdParams)]),
    "ld_init": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ld_init_with_reference": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double]),
    "ld_field_sum": (ctypes.c_int, [_VP, ctypes.c_longlong, _VP, _VP]),
    "ld_planes_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int]),
    "ld_pack_planes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP]),
    "ld_unpack_planes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP]),
    "ld_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "ld_step_kernel": (ctypes.c_int, [_VP]),
    "ld_moments": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ld_check": (ctypes.c_int, [_VP]),
    "ld_test_bounded_wait": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "ld_get_distributions": (ctypes.c_int, [_VP, _VP, _VP]),
    "ld_set_distributions": (ctypes.c_int, [_VP, _VP, _VP]),
    "ld_propagate": (ctypes.c_int, [_VP, ctypes.c_int]),
    "ld_state_bytes": (ctypes.c_size_t, [_VP]),
    "ld_save_state": (ctypes.c_int, [_VP, _VP]),
    "ld_load_state": (ctypes.c_int, [_VP, _VP]),
    "ld_fields_bytes": (ctypes.c_size_t, [_VP]),
    "ld_step_between": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ld_adjoint_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "ld_adjoint_attach": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "ld_adjoint_seed": (ctypes.c_int, [_VP, _VP]),
    "ld_adjoint_step": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ld_adjoint_init": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "ld_adjoint_get": (ctypes.c_int, [_VP, _VP, _VP]),
    "ld_adjoint_set": (ctypes.c_int, [_VP, _VP, _VP]),
    "ld_totals_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "ld_probe_fp64_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "lc_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(LcParams)]),
    "lc_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(LcParams), _VP,
                                 ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "lc_init": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "lc_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lc_step_kernel": (ctypes.c_int, [_VP]),
    "lc_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "lc_destroy": (ctypes.c_int, [_VP]),
    "ld_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ld_last_error": (ctypes.c_char_p, [_VP]),
}


def _load(path):
    handle = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(handle, name)
        fn.restype = res
        fn.argtypes = args
    return handle


def lib():
    """Load libld.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(_build.build())
        return _lib


@contextlib.contextmanager
def debug_library():
    """Within the block every call goes to the bounds-checked debug build
    (libld_debug.so, built on first use): its step kernels report a site
    index outside the lattice through ld_check instead of faulting. Contexts
    created inside the block belong to it."""
    global _lib
    release = lib()
    with _lock:
        _lib = _load(_build.build(debug=True))
    try:
        yield _lib
    finally:
        with _lock:
            _lib = release


def _ptr(t):
    """Device pointer of a tensor (or None)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _call(name, ctx, *args):
    rc = getattr(lib(), name)(ctx, *args)
    if rc != LD_OK:
        msg = lib().ld_last_error(ctx).decode(errors="replace")
        raise LdError(rc, name, msg)
    return rc


def make_params(A=-0.0625, B=0.0625, kappa=0.04, Gamma=0.5, tau_f=1.0, tau_g=1.0, rho0=1.0,
                precision="fp32", kernel="auto", stencil=7, force="potential", collision="bgk",
                magic=0.1875, rounding="nearest", seed=0) -> LdParams:
    """ld_params; stencil is 7 (7-point Laplacian, central difference) or 19
    (the 19-point isotropic forms); force is "potential" (-phi grad mu) or
    "stress" (-div P); collision is "bgk" or "trt" (with the magic parameter
    (tau_f - 1/2)(tau- - 1/2)); rounding of the 16-bit storage forms is
    "nearest" or "stochastic" (with a 64-bit seed)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    kern = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    frc = FORCES[force] if isinstance(force, str) else int(force)
    col = COLLISIONS[collision] if isinstance(collision, str) else int(collision)
    rnd = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    return LdParams(A, B, kappa, Gamma, tau_f, tau_g, rho0, prec, kern, STENCILS[int(stencil)], frc, col, magic,
                    rnd, int(seed) & 0xFFFFFFFFFFFFFFFF)


# ---------------------------------------------------------------------------
# Same-named wrappers of the C entry points.

def ld_workspace_bytes(nx, ny, nz, params: LdParams) -> int:
    return int(lib().ld_workspace_bytes(nx, ny, nz, ctypes.byref(params)))


def ld_create(nx, ny, nz, params: LdParams, workspace: torch.Tensor, stream=None):
    out = ctypes.c_void_p()
    ws = _ptr(workspace)
    nbytes = workspace.numel() * workspace.element_size()
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream(workspace.device).cuda_stream)
    rc = lib().ld_create(nx, ny, nz, ctypes.byref(params), ws, nbytes, s, ctypes.byref(out))
    if rc != LD_OK:
        raise LdError(rc, "ld_create", lib().ld_last_error(None).decode(errors="replace"))
    return out


def ld_destroy(ctx):
    return lib().ld_destroy(ctx)


def ld_set_stream(ctx, stream: int):
    return _call("ld_set_stream", ctx, ctypes.c_void_p(stream))


def ld_set_params(ctx, params: LdParams):
    return _call("ld_set_params", ctx, ctypes.byref(params))


def ld_init(ctx, phi, rho=None, u=None):
    return _call("ld_init", ctx, _ptr(phi), _ptr(rho), _ptr(u))


def ld_init_with_reference(ctx, phi, rho=None, u=None, phi_mean=0.0):
    return _call("ld_init_with_reference", ctx, _ptr(phi), _ptr(rho), _ptr(u), float(phi_mean))


def ld_field_sum(ctx, x, out):
    return _call("ld_field_sum", ctx, ctypes.c_longlong(x.numel()), _ptr(x), _ptr(out))


def ld_planes_bytes(ctx, nplanes: int) -> int:
    return int(lib().ld_planes_bytes(ctx, int(nplanes)))


def ld_pack_planes(ctx, z0: int, nplanes: int, buf):
    return _call("ld_pack_planes", ctx, int(z0), int(nplanes), _ptr(buf))


def ld_unpack_planes(ctx, z0: int, nplanes: int, buf):
    return _call("ld_unpack_planes", ctx, int(z0), int(nplanes), _ptr(buf))


def ld_step_kernel(ctx) -> str:
    """Name of the step kernel the context runs (AUTO resolved)."""
    code = lib().ld_step_kernel(ctx)
    names = {v: k for k, v in KERNELS.items()}
    if code not in names:
        raise LdError(code, "ld_step_kernel", "invalid context")
    return names[code]


def ld_step(ctx, nsteps: int):
    return _call("ld_step", ctx, int(nsteps))


def ld_moments(ctx, rho=None, u=None, phi=None, grad_phi=None, totals=None):
    return _call("ld_moments", ctx, _ptr(rho), _ptr(u), _ptr(phi), _ptr(grad_phi), _ptr(totals))


def ld_check(ctx):
    return _call("ld_check", ctx)


def ld_test_bounded_wait(ctx, max_polls: int, probe: bool):
    return _call("ld_test_bounded_wait", ctx, int(max_polls), int(bool(probe)))


def ld_get_distributions(ctx, f=None, g=None):
    return _call("ld_get_distributions", ctx, _ptr(f), _ptr(g))


def ld_set_distributions(ctx, f, g):
    return _call("ld_set_distributions", ctx, _ptr(f), _ptr(g))


def ld_propagate(ctx, reverse: bool = False):
    return _call("ld_propagate", ctx, int(bool(reverse)))


def ld_state_bytes(ctx) -> int:
    return int(lib().ld_state_bytes(ctx))


def ld_save_state(ctx, buf):
    return _call("ld_save_state", ctx, _ptr(buf))


def ld_load_state(ctx, buf):
    return _call("ld_load_state", ctx, _ptr(buf))


def ld_fields_bytes(ctx) -> int:
    return int(lib().ld_fields_bytes(ctx))


def ld_step_between(ctx, src_state, dst_state, fields_out=None):
    return _call("ld_step_between", ctx, _ptr(src_state), _ptr(dst_state), _ptr(fields_out))


def ld_adjoint_workspace_bytes(ctx) -> int:
    return int(lib().ld_adjoint_workspace_bytes(ctx))


def ld_adjoint_attach(ctx, workspace):
    return _call("ld_adjoint_attach", ctx, _ptr(workspace), workspace.numel() * workspace.element_size())


def ld_adjoint_seed(ctx, phibar):
    return _call("ld_adjoint_seed", ctx, _ptr(phibar))


def ld_adjoint_step(ctx, state_t, grad_params=None, fields_t=None):
    return _call("ld_adjoint_step", ctx, _ptr(state_t), _ptr(fields_t), _ptr(grad_params))


def ld_adjoint_init(ctx, phi0, grad_phi0, u0=None, grad_params=None):
    return _call("ld_adjoint_init", ctx, _ptr(phi0), _ptr(u0), _ptr(grad_phi0), _ptr(grad_params))


def ld_adjoint_get(ctx, fbar=None, gbar=None):
    return _call("ld_adjoint_get", ctx, _ptr(fbar), _ptr(gbar))


def ld_adjoint_set(ctx, fbar, gbar):
    return _call("ld_adjoint_set", ctx, _ptr(fbar), _ptr(gbar))


def ld_totals_static(nx, ny, nz, f, g, totals, stream=None):
    """Allocation-free FP64 totals of double[19][N] distributions (see ld.h).

    The library can check only the size limit of its static scratch, not the
    extent of the buffers it is given, so the tensors are checked here before
    any launch: f and g float64 with at least 19 nx ny nz elements, totals
    float64 with at least 5, all three on one CUDA device. The call runs with
    that device current."""
    n = int(nx) * int(ny) * int(nz)
    for name, t, need in (("f", f, Q * n), ("g", g, Q * n), ("totals", totals, 5)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"ld_totals_static: {name} must be a torch.Tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"ld_totals_static: {name} must be float64, got {t.dtype}")
        if t.numel() < need:
            raise ValueError(f"ld_totals_static: {name} holds {t.numel()} values, {need} needed")
    if not (f.device == g.device == totals.device):
        raise ValueError("ld_totals_static: f, g and totals must be on one device")
    with torch.cuda.device(f.device):
        s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream(f.device).cuda_stream)
        rc = lib().ld_totals_static(nx, ny, nz, _ptr(f), _ptr(g), _ptr(totals), s)
    if rc != LD_OK:
        raise LdError(rc, "ld_totals_static", lib().ld_last_error(None).decode(errors="replace"))
    return rc


def ld_probe_fp64_rate(op: int, blocks: int, iters: int, sink, stream=None):
    """Launch the FP64 throughput probe (see ld.h); the caller times it."""
    if sink.dtype != torch.float64 or sink.numel() < blocks:
        raise ValueError("ld_probe_fp64_rate: sink must be float64 with at least `blocks` values")
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream(sink.device).cuda_stream)
    rc = lib().ld_probe_fp64_rate(int(op), int(blocks), int(iters), _ptr(sink), s)
    if rc != LD_OK:
        raise LdError(rc, "ld_probe_fp64_rate", lib().ld_last_error(None).decode(errors="replace"))
    return rc


# ---------------------------------------------------------------------------
# Liquid crystal (see ld.h): same-named wrappers and LcSim.

def _lc_call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != LD_OK:
        raise LdError(rc, name, lib().ld_last_error(None).decode(errors="replace"))
    return rc


def make_lc_params(A0=0.01, gamma=3.0, kappa=0.01, Gamma=0.3, xi=0.7, tau_f=1.0, rho0=1.0,
                   precision="fp32", kernel="auto") -> LcParams:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    kern = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return LcParams(A0, gamma, kappa, Gamma, xi, tau_f, rho0, prec, kern)


def lc_workspace_bytes(nx, ny, nz, params: LcParams) -> int:
    return int(lib().lc_workspace_bytes(nx, ny, nz, ctypes.byref(params)))


def lc_create(nx, ny, nz, params: LcParams, workspace, stream=None):
    out = ctypes.c_void_p()
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream(workspace.device).cuda_stream)
    _lc_call("lc_create", nx, ny, nz, ctypes.byref(params), _ptr(workspace),
             workspace.numel() * workspace.element_size(), s, ctypes.byref(out))
    return out


def lc_init(ctx, q, rho=None, u=None):
    return _lc_call("lc_init", ctx, _ptr(q), _ptr(rho), _ptr(u))


def lc_step(ctx, nsteps: int):
    return _lc_call("lc_step", ctx, int(nsteps))


def lc_step_kernel(ctx) -> str:
    """The step kernel of a liquid-crystal context: "generic" or "fused"."""
    k = int(lib().lc_step_kernel(ctx))
    return {v: n for n, v in KERNELS.items()}[k]


def lc_fields(ctx, q=None, rho=None, u=None, h=None, f=None):
    return _lc_call("lc_fields", ctx, _ptr(q), _ptr(rho), _ptr(u), _ptr(h), _ptr(f))


def lc_destroy(ctx):
    return lib().lc_destroy(ctx)


class LcSim:
    """A liquid-crystal lattice with its torch-owned workspace. Q is given
    and returned as float64 CUDA tensors (5, nz, ny, nx) of the components
    xx, xy, xz, yy, yz."""

    def __init__(self, nx, ny, nz, precision="fp32", device="cuda", stream=None, **model):
        self.shape = (nz, ny, nx)
        self.device = torch.device(device)
        self.params = make_lc_params(precision=precision, **model)
        nbytes = lc_workspace_bytes(nx, ny, nz, self.params)
        if nbytes == 0:
            raise LdError(LD_EINVAL, "lc_workspace_bytes", "invalid lattice size or parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lc_create(nx, ny, nz, self.params, self.workspace, stream)

    def close(self):
        if getattr(self, "ctx", None):
            lc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, q, rho=None, u=None):
        conv = lambda t: None if t is None else torch.as_tensor(t, dtype=torch.float64,  # noqa: E731
                                                                 device=self.device).contiguous()
        self._inputs = (conv(q), conv(rho), conv(u))
        lc_init(self.ctx, *self._inputs)

    def step(self, nsteps=1):
        lc_step(self.ctx, nsteps)

    @property
    def kernel(self) -> str:
        return lc_step_kernel(self.ctx)

    def fields(self):
        mk = lambda *lead: torch.empty(*lead, *self.shape, dtype=torch.float64, device=self.device)  # noqa: E731
        out = dict(q=mk(5), rho=mk(), u=mk(3), h=mk(5), f=mk(Q))
        lc_fields(self.ctx, out["q"], out["rho"], out["u"], out["h"], out["f"])
        return out


def ld_strerror(code: int) -> str:
    return lib().ld_strerror(code).decode()


def ld_last_error(ctx=None) -> str:
    return lib().ld_last_error(ctx).decode(errors="replace")


# ---------------------------------------------------------------------------
class LdSim:
    """A lattice with its torch-owned workspace and a library context.

    Fields are torch float64 CUDA tensors shaped (nz, ny, nx) (vectors
    (3, nz, ny, nx), distributions (19, nz, ny, nx)), site order x fastest.
    """

    def __init__(self, nx, ny, nz, precision="fp32", kernel="auto", device="cuda", stream=None, **model):
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self.device = torch.device(device)
        self.params = make_params(precision=precision, kernel=kernel, **model)
        nbytes = ld_workspace_bytes(nx, ny, nz, self.params)
        if nbytes == 0:
            raise LdError(LD_EINVAL, "ld_workspace_bytes", "invalid lattice size or parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = ld_create(nx, ny, nz, self.params, self.workspace, stream)

    def close(self):
        if getattr(self, "ctx", None):
            ld_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, *lead):
        return torch.empty(*lead, *self.shape, dtype=torch.float64, device=self.device)

    def set_params(self, **model):
        p = self.params
        kw = {f[0]: getattr(p, f[0]) for f in LdParams._fields_}
        if "stencil" in model:
            model = dict(model, stencil=STENCILS[int(model["stencil"])])
        if isinstance(model.get("force"), str):
            model = dict(model, force=FORCES[model["force"]])
        if isinstance(model.get("collision"), str):
            model = dict(model, collision=COLLISIONS[model["collision"]])
        if isinstance(model.get("rounding"), str):
            model = dict(model, rounding=ROUNDINGS[model["rounding"]])
        kw.update(model)
        params = LdParams(*[kw[f[0]] for f in LdParams._fields_])
        ld_set_params(self.ctx, params)  # raises, keeping the old parameters, if refused
        self.params = params

    def init(self, phi, rho=None, u=None):
        phi = torch.as_tensor(phi, dtype=torch.float64, device=self.device).contiguous()
        rho = None if rho is None else torch.as_tensor(rho, dtype=torch.float64, device=self.device).contiguous()
        u = None if u is None else torch.as_tensor(u, dtype=torch.float64, device=self.device).contiguous()
        self._inputs = (phi, rho, u)  # kept alive until the stream has consumed them
        ld_init(self.ctx, phi, rho, u)

    def step(self, nsteps=1):
        ld_step(self.ctx, nsteps)

    def moments(self, grad_phi=False):
        out = dict(rho=self._field(), u=self._field(3), phi=self._field(),
                   totals=torch.empty(5, dtype=torch.float64, device=self.device))
        if grad_phi:
            out["grad_phi"] = self._field(3)
        ld_moments(self.ctx, out["rho"], out["u"], out["phi"], out.get("grad_phi"), out["totals"])
        return out

    def totals(self):
        t = torch.empty(5, dtype=torch.float64, device=self.device)
        ld_moments(self.ctx, totals=t)
        return t

    def check(self):
        ld_check(self.ctx)

    def distributions(self):
        f, g = self._field(Q), self._field(Q)
        ld_get_distributions(self.ctx, f, g)
        return f, g

    def set_distributions(self, f, g):
        f = torch.as_tensor(f, dtype=torch.float64, device=self.device).contiguous()
        g = torch.as_tensor(g, dtype=torch.float64, device=self.device).contiguous()
        self._inputs = (f, g)
        ld_set_distributions(self.ctx, f, g)

    def propagate(self, reverse=False):
        ld_propagate(self.ctx, reverse)

    def save_state(self, buf=None):
        if buf is None:
            buf = torch.empty(ld_state_bytes(self.ctx), dtype=torch.uint8, device=self.device)
        ld_save_state(self.ctx, buf)
        return buf

    def load_state(self, buf):
        ld_load_state(self.ctx, buf)
