"""ld_totals_static: the FP64 conservation totals without any allocation.

Callers that cannot allocate device memory or hand the library a workspace
(a monitoring or checkpoint hook that must leave a running simulation's
device-memory footprint unchanged, code running inside another library's
allocator callback) use this entry point; its partial sums live in a fixed
static device array inside the library. Here its result is checked against
the workspace-based totals of ld_moments, on two calls in a row with
different data, and sizes beyond its limit are rejected.

This file is collected last on purpose (name order), so that a run stopping
at the first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def test_static_totals_match_workspace_totals(ld):
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
        out.fill_(float("nan"))
        ld.ld_totals_static(nx, ny, nz, f, g, out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: {a}"
        # same tolerances as the workspace totals against the oracle
        assert abs(a[0] - b[0]) <= 1e-12 * n, f"call {call}: mass {a[0]} vs {b[0]}"
        assert abs(a[1] - b[1]) <= 1e-12 * n, f"call {call}: phi {a[1]} vs {b[1]}"
        assert np.abs(a[2:] - b[2:]).max() <= 1e-13 * n, f"call {call}: momentum {a[2:]} vs {b[2:]}"
    sim.close()


def test_static_totals_rejects_sizes_beyond_its_scratch(ld):
    f = torch.zeros(19, 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(ld.LdError) as e:
        ld.ld_totals_static(1024, 1024, 128, f, f, out)
    assert e.value.code == ld.LD_EINVAL
    assert "static scratch" in str(e.value)
