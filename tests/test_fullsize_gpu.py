"""Checks at the benchmark's full size and in its launch configuration.

Sub-box parity at 384^3 (the spinodal benchmark lattice, fused kernel, FP32,
FP16-deviation and BF16-deviation storage) and at 512 x 512 x 448 (large enough for the
kernels' 64-bit offsets): after n steps the macroscopic fields at a site
depend only on the initial state within L-infinity distance 3n + 2 of it
(each step reads phi within 2 sites for mu and grad mu, and propagation moves
values by 1; the output moments read phi within 2). A periodic box of edge
2h around a sampled centre therefore reproduces the full lattice's values
exactly on the inner cube of half-width r wherever r + 3n + 2 <= h - 1. The
oracle runs that box, and the inner cube (24^3 sites here) is compared with
the GPU's full-lattice moments element by element.

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


def _bounds(precision, steps, f_dev_max):
    """Per-field bounds against the FP64 oracle on the compared cube.

    FP32 storage: each stored value rounds by at most 2^-24 of itself per
    step and rho, phi and j sum 19 of them, each at most 1/3 (f) in size, so
    after n steps rho, phi and u move by at most n * 19 * 2^-24 / 3 absolute
    (the arithmetic's own rounding is smaller still).
    FP16/BF16 deviations (p = 11, 8 significand bits): each stored f
    deviation rounds by at most 2^-p of its size per step, so rho and u move
    by at most n * 19 * 2^-p * max|f_i - w_i rho0| absolute (f_dev_max is
    the largest deviation of the oracle's final state on the box), plus the
    FP32 arithmetic's share, the FP32 bound above; phi
    stays within 2^-p sqrt(n) relative L2, the random-walk bound used for
    these forms at every configuration."""
    if precision == "fp32":
        a = steps * 19 * 2.0 ** -24 / 3.0
        return {"rho": a, "phi": a, "u": a}
    p = {"fp16dev": 11, "bf16dev": 8}[precision]
    a = steps * 19 * (2.0 ** -p * f_dev_max + 2.0 ** -24 / 3.0)
    return {"rho": a, "u": a, "phi_rel": 2.0 ** -p * math.sqrt(steps)}


def _subbox_parity(ld, nx, ny, nz, centres, seed, kernel="auto", precision="fp32", steps=10, r=12):
    """Run `steps` steps on the full lattice and compare the moments on the
    (2r)^3 cube around each centre with the oracle run on a periodic box of
    edge 2h, h = r + 3 steps + 3."""
    h = r + 3 * steps + 3
    phi0 = inputs.spinodal_phi(nx, ny, nz, seed=seed)
    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel=kernel)  # auto: the benchmark's kernel
    sim.init(torch.from_numpy(phi0).cuda())
    sim.step(steps)
    m = sim.moments()
    totals = m["totals"].cpu().numpy()
    prm = oracle.param_vector()
    w = oracle.lattice()[1]
    for (z, y, x) in centres:
        box = lambda c, n: np.arange(c - h, c + h) % n  # noqa: E731
        sub = phi0[box(z, nz)[:, None, None], box(y, ny)[None, :, None], box(x, nx)[None, None, :]]
        f, g = oracle.init(sub, prm)
        f, g = oracle.step(f, g, prm, steps)
        ref = oracle.macros(f, g, prm)
        inner = slice(h - r, h + r)
        bound = _bounds(precision, steps, float(np.abs(f - w[:, None, None, None]).max()))
        zi = torch.from_numpy(np.arange(z - r, z + r) % nz).cuda()
        yi = torch.from_numpy(np.arange(y - r, y + r) % ny).cuda()
        xi = torch.from_numpy(np.arange(x - r, x + r) % nx).cuda()
        pick = lambda t: t.index_select(-3, zi).index_select(-2, yi).index_select(-1, xi).cpu().numpy()  # noqa: E731
        got = {"rho": pick(m["rho"]), "phi": pick(m["phi"]), "u": pick(m["u"])}
        want = {"rho": ref["rho"][inner, inner, inner], "phi": ref["phi"][inner, inner, inner],
                "u": ref["u"][:, inner, inner, inner]}
        where = f"{precision} {nx}x{ny}x{nz} centre {(z, y, x)}"
        for k in ("rho", "phi", "u"):
            if k in bound:
                err = float(np.abs(got[k] - want[k]).max())
                assert err <= bound[k], f"{where}: {k} max abs error {err:.3e} > {bound[k]:.2e}"
        if "phi_rel" in bound:
            err = float(np.linalg.norm(got["phi"] - want["phi"]) / np.linalg.norm(want["phi"]))
            assert err <= bound["phi_rel"], f"{where}: phi relative L2 {err:.3e} > {bound['phi_rel']:.2e}"
    del m
    # conservation over the whole lattice
    n = nx * ny * nz
    sim.init(torch.from_numpy(phi0).cuda())
    t0 = sim.totals().cpu().numpy()
    tol = 1e-6 * n if precision == "fp32" else 1e-3 * n
    assert abs(totals[0] - t0[0]) < tol
    assert abs(totals[1] - t0[1]) < tol
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
def test_subbox_parity_384cube(ld, precision):
    """The benchmark lattice and kernel, 10 steps, four 24^3 cubes (one on
    the lattice's corner, so every periodic seam is inside a compared cube).
    BF16-dev runs the pair kernel's psi pass on four-site quads."""
    n = 384
    rng = np.random.default_rng(99)
    centres = [(0, 0, 0), (191, 7, 383)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(2)]
    _subbox_parity(ld, n, n, n, centres, seed=5, precision=precision)


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["fused", "generic"])
def test_subbox_parity_64bit_offsets(ld, kernel):
    """512 x 512 x 448 sites: 19 x npad exceeds 2^31, so the step runs the
    kernel instances with 64-bit element offsets (35 GB of FP32 state)."""
    nx, ny, nz = 512, 512, 448
    centres = [(0, 0, 0), (447, 3, 260), (200, 511, 0)]
    _subbox_parity(ld, nx, ny, nz, centres, seed=6, kernel=kernel, steps=4)


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
