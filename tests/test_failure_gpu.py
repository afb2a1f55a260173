"""Failure detection without a GPU fault.

The staged step kernel's barrier waits are bounded: a wait that runs out
records a status bit that ld_check reports as LD_ECUDA, and the kernel
returns. ld_test_bounded_wait makes every thread of the kernel wait once
per step on a barrier that nothing arrives on (no copy is tracked by it),
with a small poll limit: the wait runs out, the step itself completes, and
the host reads the status. Nothing here faults, traps or hangs the GPU.
"""

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


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_bounded_wait_runs_out_and_is_reported(ld, precision):
    nz, ny, nx = 8, 16, 64
    phi = torch.from_numpy(inputs.spinodal_phi(nx, ny, nz, seed=51, amplitude=0.3)).cuda()
    ref = ld.LdSim(nx, ny, nz, precision=precision, kernel="fused_staged")
    ref.init(phi)
    ref.step(3)
    ref.check()
    f_ref, g_ref = ref.distributions()
    ref.close()

    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel="fused_staged")
    sim.init(phi)
    ld.ld_test_bounded_wait(sim.ctx, 64, True)
    sim.step(3)  # every launch returns: its probe wait gives up after 64 polls
    with pytest.raises(ld.LdError) as e:
        sim.check()
    assert e.value.code == ld.LD_ECUDA
    assert "gave up waiting" in str(e.value)
    # the probe tracks no copy, so the steps themselves completed
    f, g = sim.distributions()
    torch.cuda.synchronize()
    assert torch.equal(f, f_ref) and torch.equal(g, g_ref)
    # the context stays usable: probe off, ld_init clears the record
    ld.ld_test_bounded_wait(sim.ctx, 1 << 24, False)
    sim.init(phi)
    sim.step(3)
    sim.check()
    f, g = sim.distributions()
    torch.cuda.synchronize()
    assert torch.equal(f, f_ref) and torch.equal(g, g_ref)
    sim.close()


def test_bounded_wait_setting_is_checked(ld):
    sim = ld.LdSim(32, 8, 8, precision="fp32", kernel="fused_staged")
    with pytest.raises(ld.LdError) as e:
        ld.ld_test_bounded_wait(sim.ctx, 0, False)
    assert e.value.code == ld.LD_EINVAL
    sim.close()


def test_nonfinite_state_is_reported(ld):
    """A NaN written into the state on the host side is found by ld_check."""
    nz, ny, nx = 8, 8, 32
    sim = ld.LdSim(nx, ny, nz, precision="fp32", kernel="fused_staged")
    sim.init(torch.zeros(nz, ny, nx, dtype=torch.float64, device="cuda"))
    f, g = sim.distributions()
    f[3, 2, 1, 0] = float("nan")
    sim.set_distributions(f, g)
    sim.step(1)
    with pytest.raises(ld.LdError) as e:
        sim.check()
    assert e.value.code == ld.LD_ENONFINITE
    sim.close()
