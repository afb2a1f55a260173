"""Checks at the benchmark's full size and in its launch configuration.

Sampled parity at 384^3 (the spinodal benchmark lattice, fused kernel) and
at 512 x 512 x 448 (large enough for the kernel's 64-bit offsets):
after n steps the macroscopic fields at a site depend only on the initial
state within L-infinity distance 3n + 2 of it (each step reads phi within 2
sites for mu and grad mu, and propagation moves values by 1; the output
moments read phi within 2). A periodic sub-box of 24^3 around a sampled site
therefore reproduces the full lattice's values there exactly for n = 2, so
the oracle runs that sub-box and the two are compared site by site.

Properties at any size: total mass and total phi are conserved by the step.

Droplet (configuration 3 geometry at a smaller scale): Laplace pressure jump
and mass drift per storage precision.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def _sampled_parity(ld, nx, ny, nz, samples, seed, kernel="auto"):
    """Run 2 FP32 steps on the full lattice and compare the moments at the
    sampled sites with the oracle on periodic 24^3 boxes around them."""
    steps, box = 2, 24
    phi0 = inputs.spinodal_phi(nx, ny, nz, seed=seed)
    sim = ld.LdSim(nx, ny, nz, precision="fp32", kernel=kernel)  # auto: the benchmark's kernel
    sim.init(torch.from_numpy(phi0).cuda())
    sim.step(steps)
    m = sim.moments()
    totals = m["totals"].cpu().numpy()
    prm = oracle.param_vector()
    h = box // 2
    for (z, y, x) in samples:
        zi = (np.arange(z - h, z + h) % nz)[:, None, None]
        yi = (np.arange(y - h, y + h) % ny)[None, :, None]
        xi = (np.arange(x - h, x + h) % nx)[None, None, :]
        sub = phi0[zi, yi, xi]
        f, g = oracle.init(sub, prm)
        f, g = oracle.step(f, g, prm, steps)
        r = oracle.macros(f, g, prm)
        ref_rho, ref_phi = r["rho"][h, h, h], r["phi"][h, h, h]
        ref_u = r["u"][:, h, h, h]
        got_rho = float(m["rho"][z, y, x])
        got_phi = float(m["phi"][z, y, x])
        got_u = m["u"][:, z, y, x].cpu().numpy()
        # FP32 storage: rho to a few ulp of 1, phi and u to FP32 rounding of
        # the O(w_i) values they are summed from
        assert abs(got_rho - ref_rho) < 5e-7
        assert abs(got_phi - ref_phi) < 5e-7
        assert np.abs(got_u - ref_u).max() < 5e-7
    del m
    # conservation over the whole lattice
    n = nx * ny * nz
    sim.init(torch.from_numpy(phi0).cuda())
    t0 = sim.totals().cpu().numpy()
    assert abs(totals[0] - t0[0]) < 1e-6 * n
    assert abs(totals[1] - t0[1]) < 1e-6 * n
    sim.close()


def test_sampled_parity_384cube(ld):
    n = 384
    rng = np.random.default_rng(99)
    samples = [(0, 0, 0), (n - 1, n - 1, n - 1), (191, 7, 383)] + [tuple(rng.integers(0, n, 3)) for _ in range(5)]
    _sampled_parity(ld, n, n, n, samples, seed=5)


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["fused", "generic"])
def test_sampled_parity_64bit_offsets(ld, kernel):
    """512 x 512 x 448 sites: 19 x npad exceeds 2^31, so the step runs the
    kernel instances with 64-bit element offsets (35 GB of FP32 state)."""
    nx, ny, nz = 512, 512, 448
    samples = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (447, 3, 260), (200, 511, 0)]
    _sampled_parity(ld, nx, ny, nz, samples, seed=6, kernel=kernel)


def _droplet(ld, prec, n, R, steps):
    A, B, kappa = -0.0625, 0.0625, 0.04
    xi = math.sqrt(-2 * kappa / A)
    phi0 = inputs.droplet_phi(n, n, n, R, 1.0, xi)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
    pb = lambda p: A * p * p / 2 + 3 * B * p ** 4 / 4  # noqa: E731
    sim = ld.LdSim(n, n, n, precision=prec)
    sim.init(torch.from_numpy(phi0).cuda())
    t0 = sim.totals().cpu().numpy()
    sim.step(steps)
    m = sim.moments()
    p = m["phi"].cpu().numpy()
    t1 = m["totals"].cpu().numpy()
    sim.close()
    pin = p[r < R / 2].mean()
    pout = p[r > R + 8 * xi].mean()
    V = ((p - pout) / (pin - pout)).sum()
    reff = (3 * V / (4 * math.pi)) ** (1 / 3)
    return dict(dp=pb(pin) - pb(pout), reff=reff, phi=p, mass_drift=abs(t1[0] - t0[0]) / t0[0])


@pytest.mark.slow
def test_droplet_laplace_law(ld):
    """Droplets of radius 12 and 16 in a 64^3 box, relaxed for 20000 steps:
    about six relaxation times of the slowest bulk mode of phi,
    L^2 / (4 pi^2 D) with D = Gamma (tau_g - 1/2)(A + 3B) ~ 0.031. The pressure
    jump p_b(phi_in) - p_b(phi_out), p_b = A phi^2/2 + 3B phi^4/4, follows the
    Laplace law dp = 2 sigma / R_eff up to a curvature correction that falls
    with R: the tension dp R_eff / 2 moves towards the continuum
    sigma = sqrt(-8 kappa A^3 / (9 B^2)) as R grows and is within 10 % of it at
    R = 16."""
    n, steps = 64, 20000
    A, B, kappa = -0.0625, 0.0625, 0.04
    sigma = math.sqrt(-8 * kappa * A ** 3 / (9 * B * B))
    d12 = _droplet(ld, "fp32", n, 12.0, steps)
    d16 = _droplet(ld, "fp32", n, 16.0, steps)
    s12 = d12["dp"] * d12["reff"] / 2
    s16 = d16["dp"] * d16["reff"] / 2
    assert abs(s16 - sigma) < abs(s12 - sigma), (s12, s16, sigma)
    assert abs(s16 / sigma - 1.0) < 0.10, (s12, s16, sigma)
    # FP32 storage: a step can move total mass by at most the rounding of the
    # 19 stored values per site, 19 * 2^-25 relative; the drift measured over
    # the run must stay 100 times below that worst case.
    assert d16["mass_drift"] < steps * 19 * 2.0 ** -25 / 100


@pytest.mark.slow
def test_droplet_precisions(ld):
    """A droplet of radius 24 in a 128^3 box, 2000 steps: the FP16/BF16
    deviation forms stay close to FP32 and keep the droplet's size. Each step
    rounds the stored deviations to 2^-p of their size (p = 11 for FP16, 8 for
    BF16), and in the droplet the g deviations are as large as phi itself, so
    phi may wander from FP32 by about 2^-p sqrt(steps) in relative L2."""
    n, steps, R = 128, 2000, 24.0
    ref = _droplet(ld, "fp32", n, R, steps)
    assert ref["mass_drift"] < steps * 19 * 2.0 ** -25 / 100
    for prec, p in (("fp16dev", 11), ("bf16dev", 8)):
        tol = 2.0 ** -p * math.sqrt(steps)
        d = _droplet(ld, prec, n, R, steps)
        e = np.linalg.norm(d["phi"] - ref["phi"]) / np.linalg.norm(ref["phi"])
        assert e < tol, (prec, e)
        assert abs(d["reff"] - ref["reff"]) < 0.5
