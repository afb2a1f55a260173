"""The liquid-crystal step at the bench's size and launch configuration
(256^3, the fused FP32 form; and the FP64 generic form), checked against the
FP64 oracle on sampled sub-boxes.

Light cone: one step reads Q within one site for H and the upwind
advection, u within one site for W, and u at a site needs F, so sigma
within one site and Q within two; f after propagation comes from a
neighbour's collision, which needs F there. So after n steps Q and f at a
site depend only on the starting Q and f within L-infinity distance 3n. A
periodic box of edge 2h around a centre reproduces the full lattice's values
exactly on the inner cube of half-width r wherever r + 3n <= h - 1. The
oracle runs that box from the same start, and the inner cube is compared
with the GPU's full-lattice state.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 256
STEPS = 3
H = 16                  # the oracle's box: edge 2H = 32
R = H - 1 - 3 * STEPS   # inner half-width: 6, a 12^3 cube
MODEL = dict(A0=0.01, gamma=3.0, kappa=0.01, Gamma=0.3, xi=0.7, tau_f=1.0, rho0=1.0)


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


@pytest.fixture(scope="module")
def start():
    return inputs.random_q(N, N, N, seed=5)  # the bench's liquid-crystal start


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("precision,kernel,tol", [("fp32", "fused", 1e-5), ("fp64", "generic", 1e-12)])
def test_subbox_parity_256cube(ld, start, precision, kernel, tol):
    sim = ld.LcSim(N, N, N, precision=precision, kernel=kernel, **MODEL)
    assert sim.kernel == kernel
    sim.init(torch.from_numpy(start).cuda())
    sim.step(STEPS)
    out = sim.fields()
    prm = oracle.lc_param_vector(**MODEL)
    for c in ((128, 128, 128), (3, 250, 17)):  # (z, y, x); the second box wraps in y and z
        box = [(np.arange(ci - H, ci + H) % N) for ci in c]
        ix = np.ix_(*box)
        q_box = start[(slice(None),) + ix]
        f0 = oracle.lc_init(q_box.shape[1:], prm, rho=np.ones(q_box.shape[1:]), u=np.zeros((3,) + q_box.shape[1:]))
        f_ref, q_ref = oracle.lc_step(f0, q_box, prm, STEPS)
        inner = [np.arange(ci - R, ci + R + 1) % N for ci in c]
        inner_t = [torch.from_numpy(a).cuda() for a in inner]
        sel = lambda t: t[:, inner_t[0]][:, :, inner_t[1]][:, :, :, inner_t[2]].cpu().numpy()  # noqa: E731
        s = slice(H - R, H + R + 1)
        for name, ref in (("q", q_ref[:, s, s, s]), ("f", f_ref[:, s, s, s])):
            got = sel(out[name])
            assert rel(got, ref) <= tol, (name, c, rel(got, ref))
    sim.close()
