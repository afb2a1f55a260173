"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a and loads, exports every entry point include/ld.h declares, the
binding defines a same-named wrapper for each, and the pure host calls
(workspace sizing, error strings, argument rejection) behave as declared."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ld.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b((?:ld|lc)_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def ld():
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ld_create", "ld_init", "ld_step", "ld_moments", "ld_destroy", "ld_workspace_bytes",
                     "ld_propagate", "ld_save_state", "ld_load_state", "ld_strerror", "ld_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(ld):
    lib = ld.lib()
    for name in declared_functions():
        assert hasattr(lib, name), f"libld.so does not export {name}"


def test_binding_wraps_every_declared_symbol(ld):
    for name in declared_functions():
        assert callable(getattr(ld, name, None)), f"binding lacks {name}"


def test_workspace_bytes(ld):
    n = 64 * 32 * 16
    for prec, s in ((ld.LD_FP64, 8), (ld.LD_FP32, 4), (ld.LD_FP16DEV, 2), (ld.LD_BF16DEV, 2)):
        p = ld.make_params(precision=prec)
        b = ld.ld_workspace_bytes(64, 32, 16, p)
        # two ping-pong buffers of f and g (2 x 38 values per site) dominate
        assert b >= 2 * 38 * n * s
        assert b < 2 * 38 * n * s + 4 * n * 8 + (1 << 20)
        assert b % 256 == 0


def test_workspace_bytes_rejects_bad_arguments(ld):
    p = ld.make_params()
    assert ld.ld_workspace_bytes(3, 8, 8, p) == 0
    assert ld.ld_workspace_bytes(8, 8, 0, p) == 0
    assert ld.ld_workspace_bytes(8, 8, 8, ld.make_params(tau_f=0.5)) == 0
    assert ld.ld_workspace_bytes(8, 8, 8, ld.make_params(tau_g=0.2)) == 0
    assert ld.ld_workspace_bytes(8, 8, 8, ld.make_params(precision=7)) == 0


def test_error_strings(ld):
    assert ld.ld_strerror(ld.LD_OK) == "success"
    assert ld.ld_strerror(ld.LD_EINVAL) == "invalid argument"
    assert ld.ld_strerror(ld.LD_ENONFINITE).startswith("non-finite")
    assert ld.ld_strerror(12345) == "unknown error code"


def test_create_rejects_null_workspace_and_bad_dims(ld):
    lib = ld.lib()
    out = ctypes.c_void_p()
    p = ld.make_params()
    rc = lib.ld_create(8, 8, 8, ctypes.byref(p), None, 1 << 30, None, ctypes.byref(out))
    assert rc == ld.LD_EINVAL and not out.value
    assert "device pointer" in ld.ld_last_error(None)
    rc = lib.ld_create(2, 8, 8, ctypes.byref(p), None, 1 << 30, None, ctypes.byref(out))
    assert rc == ld.LD_EINVAL
    assert ">= 4" in ld.ld_last_error(None)
    rc = lib.ld_create(8, 8, 8, ctypes.byref(ld.make_params(tau_f=0.4)), None, 0, None, ctypes.byref(out))
    assert rc == ld.LD_EINVAL
    assert "tau" in ld.ld_last_error(None)
    assert lib.ld_destroy(None) == ld.LD_OK


def test_workspace_bytes_validates_the_options(ld):
    """The option fields of ld_params are read at their places in the
    struct and combined as the header states: pure host logic."""
    ws = ld.ld_workspace_bytes
    base = ws(32, 8, 8, ld.make_params(precision="fp32"))
    assert base > 0
    # 19-point stencils: every kernel
    assert ws(32, 8, 8, ld.make_params(precision="fp32", stencil=19)) == base
    assert ws(32, 8, 8, ld.make_params(precision="fp32", stencil=19, kernel="fused_staged")) == base
    # the stress force: generic kernel only, six stress fields in the workspace
    stress = ws(32, 8, 8, ld.make_params(precision="fp32", force="stress"))
    assert stress >= base + 6 * 32 * 8 * 8 * 4
    for kernel in ("fused", "fused_staged"):
        assert ws(32, 8, 8, ld.make_params(precision="fp32", force="stress", kernel=kernel)) == 0
    assert ws(32, 8, 8, ld.make_params(precision="fp32", force=7)) == 0
    # TRT: generic kernel only, positive magic parameter
    assert ws(32, 8, 8, ld.make_params(precision="fp32", collision="trt")) == base
    assert ws(32, 8, 8, ld.make_params(precision="fp32", collision="trt", kernel="fused")) == 0
    assert ws(32, 8, 8, ld.make_params(precision="fp32", collision="trt", magic=0.0)) == 0
    assert ws(32, 8, 8, ld.make_params(precision="fp32", collision=3)) == 0
    # stochastic rounding: the 16-bit forms only, on every kernel
    for prec in ("fp16dev", "bf16dev"):
        nearest = ws(32, 8, 8, ld.make_params(precision=prec))
        assert ws(32, 8, 8, ld.make_params(precision=prec, rounding="stochastic", seed=2**64 - 1)) == nearest
        assert ws(32, 8, 8, ld.make_params(precision=prec, rounding="stochastic", kernel="fused_staged")) == nearest
    for prec in ("fp64", "fp32"):
        assert ws(32, 8, 8, ld.make_params(precision=prec, rounding="stochastic")) == 0
    assert ws(32, 8, 8, ld.make_params(precision="fp16dev", rounding=2)) == 0
    assert ws(32, 8, 8, ld.make_params(precision="fp32", kernel=4)) == 0


def test_static_totals_wrapper_checks_buffers_before_any_launch(ld):
    """The library can check only the size limit of its static scratch, so
    the binding refuses buffers of the wrong type or extent on the host,
    before a pointer reaches the library (these CPU tensors never do)."""
    import torch

    n = 16 * 16 * 16
    f = torch.zeros(19 * n, dtype=torch.float64)
    out = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ValueError, match="needed"):
        ld.ld_totals_static(16, 16, 16, f[:-1], f, out)  # one value short, well under the size limit
    with pytest.raises(ValueError, match="needed"):
        ld.ld_totals_static(16, 16, 16, f, f, out[:4])
    with pytest.raises(ValueError, match="float64"):
        ld.ld_totals_static(16, 16, 16, f.float(), f, out)
    with pytest.raises(TypeError):
        ld.ld_totals_static(16, 16, 16, f.numpy(), f, out)


def test_lc_workspace_bytes_validates_its_arguments(ld):
    ws = ld.lc_workspace_bytes
    p = ld.make_lc_params(precision="fp32")
    b = ws(8, 8, 8, p)
    n = 8 * 8 * 8
    # f ping-pong, Q ping-pong, H, sigma, u: (2*19 + 2*5 + 5 + 9 + 3) values per site
    assert b >= 65 * n * 4 and b % 256 == 0
    assert ws(8, 8, 8, ld.make_lc_params(precision="fp64")) >= 65 * n * 8
    assert ws(2, 8, 8, p) == 0
    assert ws(8, 8, 8, ld.make_lc_params(precision="fp16dev")) == 0
    assert ws(8, 8, 8, ld.make_lc_params(tau_f=0.5)) == 0
    # step kernels: auto, generic and fused only
    assert ws(8, 8, 8, ld.make_lc_params(kernel="fused")) == b
    assert ws(8, 8, 8, ld.make_lc_params(kernel="fused_staged")) == 0
    assert ws(8, 8, 8, ld.make_lc_params(kernel=7)) == 0
