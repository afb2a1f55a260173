"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

FP64: relative L2 <= 1e-12 per field (rho, u, phi) and per distribution
after 10 and 100 steps, for the generic kernel on ragged lattices and the
fused kernel on tiled ones. Propagation and its transpose: bit-exact in every
storage precision. Reduced precisions: errors against the oracle bounded by
the rounding of their storage (derivations next to each tolerance).
"""

import numpy as np
import pytest
import torch

import oracle
from oracle_floors import oracle_u_floor
from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_run(ld, phi, steps, precision="fp64", kernel="auto", prm=None, rho=None, u=None):
    nz, ny, nx = phi.shape
    model = {} if prm is None else dict(zip(oracle.PARAM_NAMES, map(float, prm)))
    if "stencil" in model:  # the oracle's 0/1 selectors -> the library's names
        model["stencil"] = 19 if model["stencil"] else 7
    if "force" in model:
        model["force"] = "stress" if model["force"] else "potential"
    if "collision" in model:
        model["collision"] = "trt" if model["collision"] else "bgk"
    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel=kernel, **model)
    sim.init(torch.from_numpy(phi).cuda(),
             None if rho is None else torch.from_numpy(rho).cuda(),
             None if u is None else torch.from_numpy(u).cuda())
    sim.step(steps)
    m = sim.moments(grad_phi=True)
    f, g = sim.distributions()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in m.items()}
    out["f"], out["g"] = f.cpu().numpy(), g.cpu().numpy()
    sim.close()
    return out


def oracle_run(phi, steps, prm=None, rho=None, u=None):
    prm = oracle.param_vector() if prm is None else prm
    f, g = oracle.init(phi, prm, rho=rho, u=u)
    f, g = oracle.step(f, g, prm, steps)
    m = oracle.macros(f, g, prm)
    m["f"], m["g"] = f, g
    return m


def assert_parity(gpu, ref, tol, fields=("rho", "u", "phi", "grad_phi", "f", "g"), u_tol=None):
    for k in fields:
        err = rel_l2(gpu[k], ref[k])
        t = u_tol if (k == "u" and u_tol is not None) else tol
        assert err <= t, f"{k}: relative L2 {err:.3e} > {t:.1e}"
    # rho is dominated by its mean: compare the deviation too
    drho = rel_l2(gpu["rho"] - 1.0, ref["rho"] - 1.0)
    assert drho <= max(tol * 1e3, 1e-9), f"rho-1: {drho:.3e}"


# --------------------------------------------------------------------------
@pytest.mark.parametrize("steps", [10, 100])
def test_fp64_generic_16cube(ld, steps):
    """The 16^3 spinodal start (configuration 1): 1e-12 on every field; u is
    held to max(1e-12, 4 x its own rounding floor)."""
    phi = inputs.spinodal_phi(16, 16, 16, seed=1)
    u_tol = max(FP64_TOL, 4.0 * oracle_u_floor(phi, steps))
    assert_parity(gpu_run(ld, phi, steps), oracle_run(phi, steps), FP64_TOL, u_tol=u_tol)


@pytest.mark.parametrize("shape", [(4, 4, 4), (7, 6, 5), (5, 9, 33), (12, 4, 20)])
def test_fp64_generic_ragged(ld, shape):
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=7, amplitude=0.3)
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.2)
    assert_parity(gpu_run(ld, phi, 12, kernel="generic", prm=prm), oracle_run(phi, 12, prm=prm), FP64_TOL)


@pytest.mark.parametrize("shape", [(4, 8, 32), (8, 16, 64), (12, 24, 32)])
def test_fp64_fused(ld, shape):
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=3, amplitude=0.3)
    prm = oracle.param_vector(tau_f=0.9, tau_g=1.1)
    assert_parity(gpu_run(ld, phi, 20, kernel="fused", prm=prm), oracle_run(phi, 20, prm=prm), FP64_TOL)


@pytest.mark.parametrize("kernel,shape", [("generic", (7, 6, 5)), ("generic", (5, 9, 33)),
                                          ("fused", (4, 8, 32)), ("fused", (12, 24, 32))])
def test_fp64_isotropic_stencils(ld, kernel, shape):
    """The 19-point isotropic Laplacian and gradient (LD_STENCIL_19): the
    same 1e-12 bar against the oracle, on ragged lattices (generic) and tiled
    ones whose rings wrap (fused; nz = 4 and ny = 8 make every diagonal
    neighbour a periodic image)."""
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=17, amplitude=0.3)
    prm = oracle.param_vector(tau_f=0.9, tau_g=1.1, stencil=19)
    assert_parity(gpu_run(ld, phi, 20, kernel=kernel, prm=prm), oracle_run(phi, 20, prm=prm), FP64_TOL)


@pytest.mark.parametrize("kernel", ["generic", "fused"])
def test_fp32_isotropic_stencils(ld, kernel):
    """FP32 storage with the 19-point stencils: phi within the FP32 bound of
    the oracle run with the same stencils, and measurably different from the
    7-point run (the selection reaches the kernels)."""
    nz, ny, nx = 32, 32, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=2)
    prm = oracle.param_vector(stencil=19)
    g = gpu_run(ld, phi, 100, precision="fp32", kernel=kernel, prm=prm)
    r = oracle_run(phi, 100, prm=prm)
    assert rel_l2(g["phi"], r["phi"]) <= 1e-5
    assert rel_l2(g["grad_phi"], r["grad_phi"]) <= 1e-4
    r7 = oracle_run(phi, 100)
    assert rel_l2(r7["phi"], r["phi"]) > 1e-4


@pytest.mark.parametrize("stencil", [7, 19])
@pytest.mark.parametrize("shape", [(7, 6, 5), (5, 9, 33), (8, 8, 32)])
def test_fp64_stress_force(ld, shape, stencil):
    """F = -div P (LD_FORCE_STRESS) on the generic launches: 1e-12 against
    the oracle, on ragged and tiled lattices, with either stencil pair."""
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=19, amplitude=0.4)
    prm = oracle.param_vector(tau_f=0.9, tau_g=1.1, kappa=0.06, stencil=stencil, force="stress")
    assert_parity(gpu_run(ld, phi, 20, prm=prm), oracle_run(phi, 20, prm=prm), FP64_TOL)


def test_stress_force_conserves_momentum_on_the_gpu(ld):
    """With F = -div P total momentum is conserved to rounding (FP64), where
    -phi grad mu changes it at every step."""
    nz, ny, nx = 16, 16, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=23, amplitude=0.5)
    drift = {}
    for force in ("stress", "potential"):
        sim = ld.LdSim(nx, ny, nz, precision="fp64", force=force, kappa=0.06)
        sim.init(torch.from_numpy(phi).cuda())
        j0 = sim.totals().cpu().numpy()[2:]
        sim.step(200)
        j1 = sim.totals().cpu().numpy()[2:]
        drift[force] = float(np.abs(j1 - j0).max())
        sim.close()
    assert drift["stress"] < 1e-11
    assert drift["potential"] > 1e3 * drift["stress"]


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16dev", 1e-2)])
def test_reduced_precision_stress_force(ld, precision, tol):
    nz, ny, nx = 32, 32, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=2)
    prm = oracle.param_vector(force="stress")
    g = gpu_run(ld, phi, 100, precision=precision, prm=prm)
    r = oracle_run(phi, 100, prm=prm)
    assert rel_l2(g["phi"], r["phi"]) <= tol


def test_stress_force_refusals(ld):
    """The stress form runs on the generic launches and has no adjoint."""
    for kernel in ("fused", "fused_staged"):
        with pytest.raises(ld.LdError) as e:
            ld.LdSim(32, 8, 4, precision="fp32", kernel=kernel, force="stress")
        assert e.value.code == ld.LD_EINVAL
    sim = ld.LdSim(32, 8, 4, precision="fp32", force="stress")
    assert ld.ld_adjoint_workspace_bytes(sim.ctx) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(ld.LdError) as e:
        ld.ld_adjoint_attach(sim.ctx, ws)
    assert e.value.code == ld.LD_EINVAL
    with pytest.raises(ld.LdError):
        sim.set_params(force="potential")
    sim.close()


@pytest.mark.parametrize("shape", [(7, 6, 5), (5, 9, 33), (8, 8, 32)])
@pytest.mark.parametrize("magic", [0.1875, 1.0])
def test_fp64_trt_collision(ld, shape, magic):
    """The two-relaxation-time collision (LD_COLLISION_TRT) on the generic
    launches: 1e-12 against the oracle, with nonzero flow and density so that
    every even and odd part is exercised."""
    nz, ny, nx = shape
    rng = np.random.default_rng(29)
    phi = inputs.spinodal_phi(nx, ny, nz, seed=29, amplitude=0.4)
    rho = 1.0 + 0.02 * rng.standard_normal((nz, ny, nx))
    u = 0.03 * rng.standard_normal((3, nz, ny, nx))
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.1, collision="trt", magic=magic)
    assert_parity(gpu_run(ld, phi, 20, prm=prm, rho=rho, u=u), oracle_run(phi, 20, prm=prm, rho=rho, u=u), FP64_TOL)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16dev", 1e-2)])
def test_reduced_precision_trt(ld, precision, tol):
    nz, ny, nx = 32, 32, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=2)
    prm = oracle.param_vector(collision="trt", tau_f=0.8)
    g = gpu_run(ld, phi, 100, precision=precision, prm=prm)
    r = oracle_run(phi, 100, prm=prm)
    assert rel_l2(g["phi"], r["phi"]) <= tol
    assert rel_l2(g["rho"], r["rho"]) <= tol


def test_trt_refusals(ld):
    for kernel in ("fused", "fused_staged"):
        with pytest.raises(ld.LdError) as e:
            ld.LdSim(32, 8, 4, precision="fp32", kernel=kernel, collision="trt")
        assert e.value.code == ld.LD_EINVAL
    with pytest.raises(ld.LdError):
        ld.LdSim(8, 8, 8, precision="fp32", collision="trt", magic=0.0)
    sim = ld.LdSim(8, 8, 8, precision="fp32", collision="trt")
    assert ld.ld_adjoint_workspace_bytes(sim.ctx) == 0
    with pytest.raises(ld.LdError):
        sim.set_params(collision="bgk")
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("stencil", [7, 19])
def test_staged_and_register_fused_kernels_agree(ld, precision, stencil):
    """The staged kernel runs the register kernel's arithmetic on the same
    values (it changes only how they reach the threads), so the two agree
    far inside the storage bound, with either stencil pair."""
    nz, ny, nx = 12, 24, 96
    phi = inputs.spinodal_phi(nx, ny, nz, seed=19, amplitude=0.3)
    prm = oracle.param_vector(stencil=stencil)
    a = gpu_run(ld, phi, 15, precision=precision, kernel="fused", prm=prm)
    b = gpu_run(ld, phi, 15, precision=precision, kernel="fused_staged", prm=prm)
    same = {"fp32": 1e-6, "fp16dev": 2e-3, "bf16dev": 2e-2}[precision]
    assert rel_l2(b["phi"], a["phi"]) <= same
    assert rel_l2(b["f"], a["f"]) <= same
    assert rel_l2(b["g"], a["g"]) <= same


def test_fp64_fused_with_flow_and_density(ld):
    """Nonzero initial rho and u exercise every term of both equilibria."""
    nz, ny, nx = 8, 8, 32
    rng = np.random.default_rng(9)
    phi = inputs.spinodal_phi(nx, ny, nz, seed=9, amplitude=0.5)
    rho = 1.0 + 0.02 * rng.standard_normal((nz, ny, nx))
    u = 0.03 * rng.standard_normal((3, nz, ny, nx))
    g = gpu_run(ld, phi, 10, kernel="fused", rho=rho, u=u)
    r = oracle_run(phi, 10, rho=rho, u=u)
    assert_parity(g, r, FP64_TOL)


def test_fp64_droplet_fused(ld):
    n = 32
    phi = inputs.droplet_phi(n, n, n, 8.0, 1.0, 1.1313708498984760)
    assert_parity(gpu_run(ld, phi, 50), oracle_run(phi, 50), FP64_TOL)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("shape", [(5, 6, 7), (4, 8, 32)])
def test_propagate_bit_exact(ld, precision, shape):
    """Propagation moves raw stored values: decode(propagate(x)) equals
    propagate(decode(x)) bit for bit, and reverse undoes forward."""
    nz, ny, nx = shape
    rng = np.random.default_rng(11)
    sim = ld.LdSim(nx, ny, nz, precision=precision)
    c, w = oracle.lattice()
    f0 = w[:, None, None, None] * (1.0 + 0.1 * rng.standard_normal((19,) + shape))
    g0 = w[:, None, None, None] * 0.3 * rng.standard_normal((19,) + shape)
    sim.set_distributions(torch.from_numpy(f0).cuda(), torch.from_numpy(g0).cuda())
    f_dec, g_dec = (t.cpu().numpy() for t in sim.distributions())
    sim.propagate()
    f1, g1 = (t.cpu().numpy() for t in sim.distributions())
    assert np.array_equal(f1, oracle.propagate(f_dec))
    assert np.array_equal(g1, oracle.propagate(g_dec))
    sim.propagate(reverse=True)
    sim.propagate(reverse=True)
    f2, g2 = (t.cpu().numpy() for t in sim.distributions())
    assert np.array_equal(f2, oracle.propagate(f_dec, reverse=True))
    assert np.array_equal(g2, oracle.propagate(g_dec, reverse=True))
    sim.propagate()
    f3, g3 = (t.cpu().numpy() for t in sim.distributions())
    assert np.array_equal(f3, f_dec) and np.array_equal(g3, g_dec)
    sim.close()


# --------------------------------------------------------------------------
def test_conservation_fp64_gpu(ld):
    nz, ny, nx = 16, 16, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=5, amplitude=0.3)
    sim = ld.LdSim(nx, ny, nz, precision="fp64")
    sim.init(torch.from_numpy(phi).cuda())
    t0 = sim.totals().cpu().numpy()
    m = sim.moments()
    for _ in range(5):
        sim.step(20)
    t1 = sim.totals().cpu().numpy()
    n = nx * ny * nz
    assert abs(t1[0] - t0[0]) < 1e-13 * n
    assert abs(t1[1] - t0[1]) < 1e-13 * n
    sim.close()


def test_totals_match_oracle_and_are_reproducible(ld):
    nz, ny, nx = 8, 16, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=6, amplitude=0.3)
    a = gpu_run(ld, phi, 7)
    b = gpu_run(ld, phi, 7)
    r = oracle_run(phi, 7)
    assert np.array_equal(a["totals"], b["totals"])  # bitwise run to run
    assert np.array_equal(a["f"], b["f"]) and np.array_equal(a["g"], b["g"])
    assert abs(a["totals"][0] - r["totals"][0]) < 1e-12 * nx * ny * nz
    assert abs(a["totals"][1] - r["totals"][1]) < 1e-12 * nx * ny * nz
    assert np.abs(a["totals"][2:] - r["totals"][2:]).max() < 1e-13 * nx * ny * nz


def test_save_load_roundtrip(ld):
    nz, ny, nx = 8, 8, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=8, amplitude=0.3)
    for precision in ("fp32", "fp16dev"):
        sim = ld.LdSim(nx, ny, nz, precision=precision)
        sim.init(torch.from_numpy(phi).cuda())
        sim.step(3)
        buf = sim.save_state()
        sim.step(5)
        fa, ga = sim.distributions()
        sim.load_state(buf)
        sim.step(5)
        fb, gb = sim.distributions()
        assert torch.equal(fa, fb) and torch.equal(ga, gb)
        sim.close()


# --------------------------------------------------------------------------
# Reduced precision against the FP64 oracle.
#
# FP32: every stored value carries a relative rounding of at most 2^-24 per
# step and the arithmetic adds a few ulp; over T steps the independent
# roundings grow like sqrt(T) (the linear dynamics amplify by at most
# exp(omega* T) ~ 1.8 at T = 100), so phi, whose scale is ~0.05, stays
# within a relative L2 of ~100 ulp: 1e-5 is the bound stated for FP32.
#
# FP16/BF16 deviations: the stored deviation h carries a relative rounding
# of 2^-11 (FP16) or 2^-8 (BF16) per step; deviations are O(w_i * |phi|),
# so phi accumulates a random-walk error of ~sqrt(T) * 2^-11 relative
# (FP16) and 2^-8 (BF16): bounds 1e-2 and 1e-1 over 100 steps.


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16dev", 1e-2), ("bf16dev", 1e-1)])
@pytest.mark.parametrize("kernel", ["generic", "fused", "fused_staged"])
def test_reduced_precision_error(ld, precision, tol, kernel):
    nz, ny, nx = 32, 32, 32
    phi = inputs.spinodal_phi(nx, ny, nz, seed=2)
    g = gpu_run(ld, phi, 100, precision=precision, kernel=kernel)
    r = oracle_run(phi, 100)
    err = rel_l2(g["phi"], r["phi"])
    assert err <= tol, f"phi relative L2 {err:.3e}"
    assert rel_l2(g["rho"], r["rho"]) <= tol


# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("shape", [(4, 8, 32), (8, 16, 64), (12, 24, 96), (16, 48, 32)])
def test_staged_kernel_matches_oracle_and_generic(ld, precision, shape):
    """The staged fused kernel on lattices that exercise every periodic edge
    of its copies: one tile across x (nx = 32) or y, edge tiles on both sides,
    z-chunks whose halo planes wrap (nz = 4, 12). Same arithmetic as the
    generic kernel up to FMA contraction; against the FP64 oracle within the
    storage-precision bound."""
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=13, amplitude=0.3)
    steps = 15
    a = gpu_run(ld, phi, steps, precision=precision, kernel="generic")
    b = gpu_run(ld, phi, steps, precision=precision, kernel="fused_staged")
    r = oracle_run(phi, steps)
    tol = {"fp32": 1e-5, "fp16dev": 1e-2, "bf16dev": 1e-1}[precision]
    assert rel_l2(b["phi"], r["phi"]) <= tol
    # rho is stored as f_i ~ w_i rho: its deviation from 1 is not resolved
    # beyond the storage ulp, so rho itself is compared
    assert rel_l2(b["rho"], r["rho"]) <= tol
    # generic and fused perform the same operations; only contraction differs
    same = {"fp32": 1e-6, "fp16dev": 2e-3, "bf16dev": 2e-2}[precision]
    assert rel_l2(b["phi"], a["phi"]) <= same
    assert rel_l2(b["f"], a["f"]) <= same


@pytest.mark.parametrize("stencil", [7, 19])
@pytest.mark.parametrize("shape", [(12, 32, 64), (8, 48, 32)])
def test_fp32_fused_several_y_tiles(ld, shape, stencil):
    """FP32 fused step over four and six y-tiles (the lowest tile's halo and
    the highest one's wrapping periodically), both stencil pairs: the same
    arithmetic as the staged kernel (1e-6, FMA contraction only) and within
    the FP32 bound of the oracle."""
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=23, amplitude=0.3)
    prm = oracle.param_vector(stencil=stencil)
    a = gpu_run(ld, phi, 20, precision="fp32", kernel="fused", prm=prm)
    b = gpu_run(ld, phi, 20, precision="fp32", kernel="fused_staged", prm=prm)
    r = oracle_run(phi, 20, prm=prm)
    assert rel_l2(a["phi"], b["phi"]) <= 1e-6
    assert rel_l2(a["f"], b["f"]) <= 1e-6
    assert rel_l2(a["g"], b["g"]) <= 1e-6
    assert rel_l2(a["phi"], r["phi"]) <= 1e-5


def test_generic_and_fused_agree(ld):
    nz, ny, nx = 8, 16, 64
    phi = inputs.spinodal_phi(nx, ny, nz, seed=12, amplitude=0.4)
    a = gpu_run(ld, phi, 30, precision="fp32", kernel="generic")
    for kernel in ("fused", "fused_staged"):
        b = gpu_run(ld, phi, 30, precision="fp32", kernel=kernel)
        assert rel_l2(b["phi"], a["phi"]) < 1e-6
        assert rel_l2(b["f"], a["f"]) < 1e-6


def test_errors_are_reported_not_raised_on_device(ld):
    sim = ld.LdSim(8, 8, 8, precision="fp32")
    with pytest.raises(ld.LdError) as e:
        sim.step(1)
    assert e.value.code == ld.LD_ESTATE
    with pytest.raises(ld.LdError) as e:
        ld.ld_init(sim.ctx, None)
    assert e.value.code == ld.LD_EINVAL
    phi = torch.zeros(8, 8, 8, dtype=torch.float64, device="cuda")
    sim.init(phi)
    sim.step(2)
    sim.check()
    # a state buffer that is not 16-byte aligned is refused before any launch
    nb = ld.ld_state_bytes(sim.ctx)
    src = torch.empty(nb + 16, dtype=torch.uint8, device="cuda")
    dst = torch.empty(nb, dtype=torch.uint8, device="cuda")
    ld.ld_save_state(sim.ctx, src)
    with pytest.raises(ld.LdError) as e:
        ld.ld_step_between(sim.ctx, src[4:], dst)
    assert e.value.code == ld.LD_EINVAL
    f, g = sim.distributions()
    f[3, 1, 2, 3] = float("nan")
    sim.set_distributions(f, g)
    with pytest.raises(ld.LdError) as e:
        sim.check()
    assert e.value.code == ld.LD_ENONFINITE
    with pytest.raises(ld.LdError):
        ld.ld_set_params(sim.ctx, ld.make_params(precision="fp64"))
    sim.close()
