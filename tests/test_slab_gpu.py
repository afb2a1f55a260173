"""The z-slab domain decomposition on one GPU (paper Sec. 2.1.1: sub-domains
with halo regions filled from their neighbours).

Each slab is its own library context; halos are refreshed through
ld_pack_planes / ld_unpack_planes between steps. Every site of a slab's own
planes then runs the same arithmetic on the same inputs as in the whole
lattice, so the decomposed run equals the single-lattice run bit for bit,
in every storage precision (the 16-bit forms take the whole lattice's
deviation reference through ld_init_with_reference).
"""

import numpy as np
import pytest
import torch

from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld, slab

    ld.lib()
    return ld, slab


def _single(ld, phi, steps, precision, kernel):
    nz, ny, nx = phi.shape
    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel=kernel)
    sim.init(torch.from_numpy(phi).cuda())
    sim.step(steps)
    f, g = sim.distributions()
    m = sim.moments()
    torch.cuda.synchronize()
    out = (f.cpu().numpy(), g.cpu().numpy(), m["phi"].cpu().numpy(), ld.ld_step_kernel(sim.ctx))
    sim.close()
    return out


@pytest.mark.parametrize("precision,kernel", [("fp64", "auto"), ("fp32", "auto"), ("fp32", "fused_staged"),
                                              ("fp16dev", "auto"), ("fp32", "generic")])
@pytest.mark.parametrize("nslabs,steps_per_exchange", [(2, 1), (3, 1), (1, 1), (2, 2)])
def test_slabs_equal_the_single_lattice_bitwise(mods, precision, kernel, nslabs, steps_per_exchange):
    ld, slab = mods
    nz, ny, nx = 48, 16, 32
    steps = 7
    phi = inputs.spinodal_phi(nx, ny, nz, seed=61, amplitude=0.3)
    f1, g1, p1, k1 = _single(ld, phi, steps, precision, kernel)
    lat = slab.SlabLattice(nx, ny, nz, nslabs, precision=precision, kernel=kernel,
                           steps_per_exchange=steps_per_exchange)
    assert ld.ld_step_kernel(lat.slabs[0].ctx) == k1  # the same kernel on every part
    lat.init(torch.from_numpy(phi).cuda())
    lat.step(steps)
    f, g = lat.distributions()
    p = lat.moments()["phi"]
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), f1)
    assert np.array_equal(g.cpu().numpy(), g1)
    assert np.array_equal(p.cpu().numpy(), p1)
    lat.close()


def test_pack_and_unpack_wrap_periodically(mods):
    """Planes z0 .. z0 + n - 1 taken modulo nz, in both directions."""
    ld, _ = mods
    nz, ny, nx = 12, 8, 32
    a = ld.LdSim(nx, ny, nz, precision="fp32")
    b = ld.LdSim(nx, ny, nz, precision="fp32")
    a.init(torch.from_numpy(inputs.spinodal_phi(nx, ny, nz, seed=62)).cuda())
    b.init(torch.zeros(nz, ny, nx, dtype=torch.float64, device="cuda"))
    buf = torch.empty(ld.ld_planes_bytes(a.ctx, 5), dtype=torch.uint8, device="cuda")
    ld.ld_pack_planes(a.ctx, 10, 5, buf)  # planes 10, 11, 0, 1, 2
    ld.ld_unpack_planes(b.ctx, -3, 5, buf)  # into 9, 10, 11, 0, 1
    fa, ga = a.distributions()
    fb, gb = b.distributions()
    torch.cuda.synchronize()
    src = [10, 11, 0, 1, 2]
    dst = [9, 10, 11, 0, 1]
    assert torch.equal(fb[:, dst], fa[:, src]) and torch.equal(gb[:, dst], ga[:, src])
    with pytest.raises(ld.LdError) as e:
        ld.ld_pack_planes(a.ctx, 0, nz + 1, buf)
    assert e.value.code == ld.LD_EINVAL
    a.close()
    b.close()
