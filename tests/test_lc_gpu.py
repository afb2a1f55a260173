"""Parity of the liquid-crystal step (lc_* calls of the C ABI) with the FP64
oracle (oracle/lc_oracle.cpp), and its invariants on the GPU.

FP64: Q, f, rho and u after 10 coupled steps within relative L2 1e-12 of the
oracle, on ragged lattices and from a start with flow, density variations and
nematic order far from equilibrium (every term of H, the stress, the
co-rotation and the upwind advection is active). FP32: within 1e-5 after 50
steps (FP32 rounding, 2^-24 per operation, accumulated over the steps).
Both step kernels: the three per-site launches (any lattice) and the fused
z-marching launch + Q update (nx % 32 == 0, ny % 8 == 0), which in FP64 gives
the same bits as the per-site launches (the same operations in the same
order), over several z-chunks and periodic wraps of every tile.
Invariants: total mass and momentum conserved (the force is the divergence
of a stress); a uniform bulk equilibrium Q = q0 (n n - I/3), at rest, is a
fixed point.
"""

import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


MODEL = dict(A0=0.01, gamma=3.0, kappa=0.01, Gamma=0.3, xi=0.7, tau_f=0.9, rho0=1.0)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def start(shape, seed):
    rng = np.random.default_rng(seed)
    q = 0.15 * rng.standard_normal((5,) + shape)
    rho = 1.0 + 0.02 * rng.standard_normal(shape)
    u = 0.02 * rng.standard_normal((3,) + shape)
    return q, rho, u


def gpu_run(ld, shape, q, rho, u, steps, precision, kernel="auto", expect=None):
    nz, ny, nx = shape
    sim = ld.LcSim(nx, ny, nz, precision=precision, kernel=kernel, **MODEL)
    if expect is not None:
        assert sim.kernel == expect
    sim.init(torch.from_numpy(q), torch.from_numpy(rho), torch.from_numpy(u))
    sim.step(steps)
    out = {k: v.cpu().numpy() for k, v in sim.fields().items()}
    sim.close()
    return out


def oracle_run(shape, q, rho, u, steps):
    prm = oracle.lc_param_vector(**MODEL)
    f = oracle.lc_init(shape, prm, rho=rho, u=u)
    f, q = oracle.lc_step(f, q, prm, steps)
    m = oracle.lc_macros(f, q, prm)
    return dict(q=q, f=f, rho=m["rho"], u=m["u"])


@pytest.mark.parametrize("shape", [(5, 6, 7), (8, 8, 16), (12, 10, 9)])
def test_fp64_matches_the_oracle(ld, shape):
    q, rho, u = start(shape, seed=sum(shape))
    g = gpu_run(ld, shape, q, rho, u, 10, "fp64")
    r = oracle_run(shape, q, rho, u, 10)
    for k in ("q", "f", "rho", "u"):
        assert rel(g[k], r[k]) <= 1e-12, (k, rel(g[k], r[k]))


# (nz, ny, nx): one tile in x and y (the halo wraps onto the tile itself),
# several tiles, and an nz the z-chunks divide unevenly into.
@pytest.mark.parametrize("shape", [(3, 8, 32), (6, 16, 64), (9, 24, 32)])
def test_fused_fp64_matches_the_oracle(ld, shape):
    q, rho, u = start(shape, seed=7 + sum(shape))
    g = gpu_run(ld, shape, q, rho, u, 10, "fp64", kernel="fused", expect="fused")
    r = oracle_run(shape, q, rho, u, 10)
    for k in ("q", "f", "rho", "u"):
        assert rel(g[k], r[k]) <= 1e-12, (k, rel(g[k], r[k]))


# 64 x 64 x 128: 32 tile columns, so the fused launch marches 16 planes per
# CTA (the small lattices above take one) and its rings turn over.
@pytest.mark.parametrize("shape", [(12, 16, 64), (64, 64, 128)])
def test_fused_fp64_is_bitwise_the_per_site_step(ld, shape):
    q, rho, u = start(shape, seed=21)
    a = gpu_run(ld, shape, q, rho, u, 5, "fp64", kernel="fused", expect="fused")
    b = gpu_run(ld, shape, q, rho, u, 5, "fp64", kernel="generic", expect="generic")
    for k in ("q", "f", "rho", "u", "h"):
        assert np.array_equal(a[k], b[k]), k
    if shape[0] == 64:
        r = oracle_run(shape, q, rho, u, 5)
        for k in ("q", "f", "rho", "u"):
            assert rel(a[k], r[k]) <= 1e-12, (k, rel(a[k], r[k]))


def test_fused_fp32_tracks_the_per_site_step(ld):
    """FP32 over 16-plane chunks (128 x 64 x 128): the two kernels round the
    same operations, up to the compiler's FMA contraction in each."""
    shape = (128, 64, 128)
    q, rho, u = start(shape, seed=5)
    a = gpu_run(ld, shape, q, rho, u, 20, "fp32", kernel="fused", expect="fused")
    b = gpu_run(ld, shape, q, rho, u, 20, "fp32", kernel="generic", expect="generic")
    for k in ("q", "f", "rho"):
        assert rel(a[k], b[k]) <= 1e-6, (k, rel(a[k], b[k]))


def test_kernel_choice(ld):
    assert ld.LcSim(32, 8, 4, precision="fp32").kernel == "fused"
    assert ld.LcSim(32, 8, 4, precision="fp64").kernel == "generic"
    assert ld.LcSim(30, 8, 4, precision="fp32").kernel == "generic"
    with pytest.raises(ld.LdError):
        ld.LcSim(30, 8, 4, precision="fp32", kernel="fused")


@pytest.mark.parametrize("kernel", ["fused", "generic"])
def test_fp32_within_its_rounding(ld, kernel):
    shape = (16, 16, 32)
    q, rho, u = start(shape, seed=3)
    g = gpu_run(ld, shape, q, rho, u, 50, "fp32", kernel=kernel, expect=kernel)
    r = oracle_run(shape, q, rho, u, 50)
    for k in ("q", "f", "rho"):
        assert rel(g[k], r[k]) <= 1e-5, (k, rel(g[k], r[k]))


@pytest.mark.parametrize("shape", [(8, 12, 16), (8, 8, 32)])
def test_mass_and_momentum_are_conserved(ld, shape):
    q, rho, u = start(shape, seed=9)
    c, _ = oracle.lattice()

    def totals(f):
        return f.sum(), np.einsum("ia,i...->a...", c, f).reshape(3, -1).sum(axis=1)

    f0 = oracle.lc_init(shape, oracle.lc_param_vector(**MODEL), rho=rho, u=u)
    m0, p0 = totals(f0)
    kernel = "fused" if shape[2] % 32 == 0 and shape[1] % 8 == 0 else "generic"
    g = gpu_run(ld, shape, q, rho, u, 100, "fp64", kernel=kernel, expect=kernel)
    m1, p1 = totals(g["f"])
    assert abs(m1 - m0) < 1e-11 * f0.size
    assert np.abs(p1 - p0).max() < 1e-12 * f0.size


def test_bulk_equilibrium_is_a_fixed_point(ld):
    shape = (4, 4, 4)
    gamma = MODEL["gamma"]
    S = 0.25 + 0.75 * math.sqrt(1.0 - 8.0 / (3.0 * gamma))
    n = np.array([1.0, -2.0, 0.5])
    n /= np.linalg.norm(n)
    Q = S * (np.outer(n, n) - np.eye(3) / 3)
    q = np.broadcast_to(np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])[:, None, None, None],
                        (5,) + shape).copy()
    g = gpu_run(ld, shape, q, np.ones(shape), np.zeros((3,) + shape), 20, "fp64")
    assert np.abs(g["q"] - q).max() < 1e-15
    assert np.abs(g["u"]).max() < 1e-15
