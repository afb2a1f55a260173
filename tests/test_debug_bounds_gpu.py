"""The bounds-checked debug build of the library (libld_debug.so, compiled
with -DLD_DEBUG_BOUNDS), on the small ragged and tiled lattices of the
parity tests. Its step kernels check the site index of every global load and
store against the lattice and report one outside it through ld_check (a
status bit, no trap). Here every kernel and precision runs clean: no index
leaves the lattice, ld_check passes, and the results are those of the
release build (FP64 bit for bit; FP32 and the 16-bit forms within the
contraction differences two compilations may have)."""

import numpy as np
import pytest
import torch

from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4), "generic", "fp64"), ((7, 6, 5), "generic", "fp64"), ((5, 9, 33), "generic", "fp32"),
         ((12, 4, 20), "generic", "fp16dev"), ((4, 8, 32), "fused", "fp64"), ((12, 24, 32), "fused", "fp32"),
         ((4, 8, 32), "fused", "fp16dev"), ((8, 16, 64), "fused_staged", "fp32"),
         ((12, 24, 96), "fused_staged", "bf16dev")]


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def _run(ld, shape, kernel, precision):
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=71, amplitude=0.3)
    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel=kernel, tau_f=0.9, tau_g=1.1)
    sim.init(torch.from_numpy(phi).cuda())
    sim.step(9)
    sim.check()  # raises LD_ECUDA if an index left the lattice
    f, g = sim.distributions()
    torch.cuda.synchronize()
    out = f.cpu().numpy(), g.cpu().numpy()
    sim.close()
    return out


@pytest.mark.parametrize("shape,kernel,precision", CASES)
def test_debug_build_runs_clean_and_matches_release(ld, shape, kernel, precision):
    release = _run(ld, shape, kernel, precision)
    with ld.debug_library():
        debug = _run(ld, shape, kernel, precision)
    tol = {"fp64": 0.0, "fp32": 1e-6, "fp16dev": 2e-3, "bf16dev": 2e-2}[precision]
    for a, b in zip(debug, release):
        if tol == 0.0:
            assert np.array_equal(a, b)
        else:
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
