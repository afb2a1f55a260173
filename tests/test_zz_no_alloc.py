"""ld_totals_static: the FP64 conservation totals without any allocation.

Callers that cannot allocate device memory or hand the library a workspace
(a monitoring or checkpoint hook that must leave a running simulation's
device-memory footprint unchanged, code running inside another library's
allocator callback) use this entry point; its partial sums live in a fixed
static device array inside the library. Here its result is checked against
the workspace-based totals of ld_moments and against sums that numpy forms
on the host from the same distributions, on two calls in a row with
different data; a repeat call on the same data gives identical bits; and
sizes beyond its limit are rejected.

This file is collected last on purpose (name order), so that a run stopping
at the first failure has already run every other test.
"""

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


def host_totals(f, g):
    """[sum rho, sum phi, sum jx, sum jy, sum jz] by numpy (pairwise sums in
    float64), with the velocity set of the oracle, and the sum of absolute
    values that bounds the rounding of any summation order."""
    c = oracle.lattice()[0].astype(np.float64)
    f2 = f.reshape(19, -1)
    g2 = g.reshape(19, -1)
    per_dir = f2.sum(axis=1)
    t = np.array([per_dir.sum(), g2.sum(), c[:, 0] @ per_dir, c[:, 1] @ per_dir, c[:, 2] @ per_dir])
    scale = np.array([np.abs(f2).sum(), np.abs(g2).sum()] + [np.abs(f2).sum()] * 3)
    return t, scale


def check_against_host(ld, nx, ny, nz, f_dev, g_dev, out):
    out.fill_(float("nan"))
    ld.ld_totals_static(nx, ny, nz, f_dev, g_dev, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want, scale = host_totals(f_dev.cpu().numpy(), g_dev.cpu().numpy())
    # any two summation orders of these values differ by at most a few
    # hundred roundings of the largest partial sum: 1e-12 of the absolute sum
    assert np.all(np.abs(got - want) <= 1e-12 * scale), (got, want)
    return got


def test_static_totals_match_workspace_and_host_totals(ld):
    # 40,000 sites: three blocks of the static reduction, the last one ragged
    nz, ny, nx = 20, 40, 50
    n = nx * ny * nz
    sim = ld.LdSim(nx, ny, nz, precision="fp64")
    sim.init(torch.from_numpy(inputs.spinodal_phi(nx, ny, nz, seed=31, amplitude=0.3)).cuda())
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(7)
        f, g = sim.distributions()
        ref = sim.totals()
        a = check_against_host(ld, nx, ny, nz, f, g, out)
        b = ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: {a}"
        # same tolerances as the workspace totals against the oracle
        assert abs(a[0] - b[0]) <= 1e-12 * n, f"call {call}: mass {a[0]} vs {b[0]}"
        assert abs(a[1] - b[1]) <= 1e-12 * n, f"call {call}: phi {a[1]} vs {b[1]}"
        assert np.abs(a[2:] - b[2:]).max() <= 1e-13 * n, f"call {call}: momentum {a[2:]} vs {b[2:]}"
    sim.close()


@pytest.mark.parametrize("shape", [(16, 16, 16), (168, 168, 168)])
def test_static_totals_block_counts(ld, shape):
    """16^3: exactly one block of the static reduction. 168^3 (4.7M sites):
    290 blocks, more than the final pass's 256 threads, so its strided loop
    runs twice. Two calls in a row on different data, then a repeat of the
    second: identical bits."""
    nz, ny, nx = shape
    n = nx * ny * nz
    rng = np.random.default_rng(nx)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    w = oracle.lattice()[1][:, None]
    last = None
    for call in range(2):
        f = torch.from_numpy(w * (1.0 + 0.1 * rng.standard_normal((19, n)))).cuda()
        g = torch.from_numpy(0.05 * rng.standard_normal((19, n))).cuda()
        last = (f, g, check_against_host(ld, nx, ny, nz, f, g, out))
    f, g, first = last
    out.fill_(0.0)
    ld.ld_totals_static(nx, ny, nz, f, g, out)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tobytes() == first.tobytes()


def test_static_totals_rejects_sizes_beyond_its_scratch(ld):
    """The library refuses lattices beyond its static scratch before any
    launch. The Python wrapper would already refuse these short buffers, so
    the C entry point is called directly: the library reads nothing."""
    small = torch.zeros(19 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = ld.lib().ld_totals_static(1024, 1024, 128, ld._ptr(small), ld._ptr(small), ld._ptr(out),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == ld.LD_EINVAL
    assert "static scratch" in ld.ld_last_error(None)
    with pytest.raises(ValueError):
        ld.ld_totals_static(16, 16, 16, small, small, out)  # too short: refused by the wrapper
