"""Stochastic rounding of the 16-bit storage forms (LD_ROUND_STOCHASTIC) on
the GPU, through the C ABI, against the numpy checker oracle/rounding.py
and the FP64 oracle.

The decision of each store is a function of the FP32 deviation h and its
16-bit key only. The GPU's h differs from the oracle's FP64 value by its
FP32 arithmetic, bounded here by delta = 32 FP32 units of the largest value
of that direction. Stochastic rounding with a fixed key is non-decreasing in
h, so where the checker's results at h - delta and h + delta agree, the GPU
must have stored exactly that value: a wrong key (counter, bit field, site,
array or step) or a wrong rule flips about a third of those decisions
(2p(1 - p) averaged over the position p of h in its cell).
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import rounding as R
from paper_1609_01479_gb300 import inputs

pytestmark = pytest.mark.gpu

FMT = {"fp16dev": "fp16", "bf16dev": "bf16"}
SEED = 0x5EED0F5A17C0FFEE


@pytest.fixture(scope="module")
def ld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01479_gb300 import ld as mod

    mod.lib()
    return mod


def _start(nx, ny, nz, seed=41):
    """A state far from equilibrium deviations of zero: rho 1 +- 5 %,
    |u| ~ 0.04, phi +- 0.5."""
    rng = np.random.default_rng(seed)
    phi = inputs.spinodal_phi(nx, ny, nz, seed=seed, amplitude=0.5)
    rho = 1.0 + 0.05 * (2 * rng.random((nz, ny, nx)) - 1)
    u = 0.04 * (2 * rng.random((3, nz, ny, nx)) - 1)
    return phi, rho, u


def _pushed(keys, shape):
    """Keys indexed by source site -> keys at the destination x + c_i."""
    c, _ = oracle.lattice()
    nz, ny, nx = shape
    k = keys.reshape(19, nz, ny, nx)
    return np.stack([np.roll(k[i], shift=(int(c[i][2]), int(c[i][1]), int(c[i][0])), axis=(0, 1, 2))
                     for i in range(19)])


def _check_decisions(stored, exact, ref, keys, fmt):
    """stored, exact: (19, nz, ny, nx) doubles (decoded GPU values, FP64
    oracle values); ref: (19,) float32 references; keys at the
    destinations. Returns the fraction of decisions that were checked."""
    h_gpu = (stored - ref[:, None, None, None].astype(np.float64)).astype(np.float32)
    h = exact - ref[:, None, None, None].astype(np.float64)
    delta = 32 * 2.0 ** -24 * np.abs(exact).reshape(19, -1).max(axis=1)[:, None, None, None]
    lo = R.decode(R.stochastic_round((h - delta).astype(np.float32), keys, fmt), fmt)
    hi = R.decode(R.stochastic_round((h + delta).astype(np.float32), keys, fmt), fmt)
    sure = lo == hi
    bad = sure & (h_gpu != lo)
    assert not bad.any(), f"{int(bad.sum())} of {int(sure.sum())} decided stores differ"
    # the others lie between the two bracketing results
    assert np.all((h_gpu >= np.minimum(lo, hi)) & (h_gpu <= np.maximum(lo, hi)))
    return float(sure.mean())


@pytest.mark.parametrize("precision", ["fp16dev", "bf16dev"])
@pytest.mark.parametrize("kernel", ["fused", "fused_staged", "generic"])
@pytest.mark.parametrize("t", [0, 3])
def test_stochastic_stores_match_the_checker(ld, precision, kernel, t):
    """One step at step counter t from a known state: every store the FP32
    noise cannot flip equals the checker's stochastic rounding of the FP64
    oracle's value with key (seed, t, array, direction, source site). A
    wrong key would flip about a third of the decided stores."""
    nx, ny, nz = 32, 16, 12
    n = nx * ny * nz
    fmt = FMT[precision]
    phi, rho, u = _start(nx, ny, nz)
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.3)
    f0, g0 = oracle.init(phi, prm, rho=rho, u=u)
    sim = ld.LdSim(nx, ny, nz, precision=precision, kernel=kernel, tau_f=0.8, tau_g=1.3,
                   rounding="stochastic", seed=SEED)
    # no ld_init: references w_i rho0 for f and 0 for g, step counter 0
    sim.set_distributions(torch.from_numpy(f0), torch.from_numpy(g0))
    sim.step(t)
    fa, ga = (a.cpu().numpy() for a in sim.distributions())
    sim.step(1)
    fb, gb = (a.cpu().numpy() for a in sim.distributions())
    sim.close()
    fx, gx = oracle.step(fa, ga, prm, 1)
    _, w = oracle.lattice()
    ref_f = np.array([np.float32(wi * 1.0) for wi in w], dtype=np.float32)
    ref_g = np.zeros(19, dtype=np.float32)
    shape = (nz, ny, nx)
    frac_f = _check_decisions(fb, fx, ref_f, _pushed(R.keys(SEED, t, 0, n), shape), fmt)
    frac_g = _check_decisions(gb, gx, ref_g, _pushed(R.keys(SEED, t, 1, n), shape), fmt)
    # Small deviations sit in cells narrower than the FP32 noise bound and
    # are not decided here; the rest (about 50-95 % of some 10^5 stores) are.
    assert frac_f > 0.3 and frac_g > 0.3, (frac_f, frac_g)


def test_stochastic_differs_from_nearest_where_it_should(ld):
    """From the same state, about a quarter of the stores of a stochastic
    step land on the other neighbour than round-to-nearest (E|SR - RN| is
    1/4 unit for a uniform position in the cell)."""
    nx, ny, nz = 32, 16, 12
    phi, rho, u = _start(nx, ny, nz)
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.3)
    f0, g0 = oracle.init(phi, prm, rho=rho, u=u)
    out = {}
    for rounding in ("nearest", "stochastic"):
        sim = ld.LdSim(nx, ny, nz, precision="bf16dev", tau_f=0.8, tau_g=1.3, rounding=rounding, seed=SEED)
        sim.set_distributions(torch.from_numpy(f0), torch.from_numpy(g0))
        sim.step(1)
        out[rounding] = np.concatenate([a.cpu().numpy().ravel() for a in sim.distributions()])
        sim.close()
    other = (out["nearest"] != out["stochastic"]).mean()
    assert 0.15 < other < 0.35, other


def test_stochastic_runs_are_reproducible_and_seeded(ld):
    """A fixed seed gives bitwise-equal runs; another seed another run;
    ld_init sets the step counter back to 0."""
    nx, ny, nz = 32, 8, 8
    phi = torch.from_numpy(inputs.spinodal_phi(nx, ny, nz, seed=4, amplitude=0.3)).cuda()

    def run(seed, steps, restart=0):
        sim = ld.LdSim(nx, ny, nz, precision="fp16dev", rounding="stochastic", seed=seed)
        sim.init(phi)
        if restart:
            sim.step(restart)
            sim.init(phi)
        sim.step(steps)
        f, g = sim.distributions()
        out = torch.cat([f.flatten(), g.flatten()]).cpu().numpy()
        sim.close()
        return out

    a, b, c = run(11, 5), run(11, 5), run(12, 5)
    assert np.array_equal(a, b)
    assert (a != c).mean() > 0.05
    assert np.array_equal(run(11, 5, restart=3), a)


def test_stochastic_rounding_refusals(ld):
    """Stochastic rounding is for the 16-bit forms, not ld_step_between or
    the adjoint, and fixed at creation."""
    for precision in ("fp64", "fp32"):
        with pytest.raises(ld.LdError) as e:
            ld.LdSim(32, 8, 4, precision=precision, rounding="stochastic")
        assert e.value.code == ld.LD_EINVAL
    sim = ld.LdSim(32, 8, 4, precision="bf16dev", rounding="stochastic", seed=1)
    sim.init(torch.zeros(4, 8, 32, dtype=torch.float64, device="cuda"))
    assert ld.ld_adjoint_workspace_bytes(sim.ctx) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(ld.LdError) as e:
        ld.ld_adjoint_attach(sim.ctx, ws)
    assert e.value.code == ld.LD_EINVAL
    a, b = sim.save_state(), sim.save_state()
    with pytest.raises(ld.LdError) as e:
        ld.ld_step_between(sim.ctx, a, b)
    assert e.value.code == ld.LD_EINVAL
    with pytest.raises(ld.LdError):
        sim.set_params(rounding="nearest")
    sim.set_params(seed=2)  # the seed may change
    sim.close()
