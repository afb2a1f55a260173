"""Pins of the stochastic-rounding checker (oracle/rounding.py) to facts
that do not come from it: exact rational bounds of rounding toward zero,
the defining expectation of stochastic rounding (averaged over every
16-bit key it returns h exactly), numpy's own round-to-nearest, and an
independent SplitMix64 (the seeded-input generator's).
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle import rounding as R
from paper_1609_01479_gb300 import inputs


def _samples(fmt, n=400, seed=3):
    """float32 values across the format's normal and subnormal ranges, both signs."""
    rng = np.random.default_rng(seed)
    lo_exp, hi_exp = (-26, 14) if fmt == "fp16" else (-135, 40)
    e = rng.integers(lo_exp, hi_exp, n)
    m = rng.random(n) + 1.0
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    h = (sign * m * np.exp2(e.astype(np.float64))).astype(np.float32)
    return h[np.isfinite(h) & (h != 0)]


@pytest.mark.parametrize("fmt", R.FORMATS)
def test_round_toward_zero_brackets_exactly(fmt):
    """|RZ(h)| <= |h| < |RZ(h) + 1 unit|, same sign, in exact rationals: a
    wrong direction or an off-by-one in the bit step fails."""
    h = _samples(fmt)
    lo = R.round_toward_zero(h, fmt)
    lof = R.decode(lo, fmt)
    hif = R.decode((lo + np.uint16(1)).astype(np.uint16), fmt)
    for hv, a, b in zip(h, lof, hif):
        H, A, B = Fraction(float(hv)), Fraction(float(a)), Fraction(float(b))
        assert abs(A) <= abs(H) < abs(B), (hv, a, b)
        assert A == 0 or (A > 0) == (H > 0)


@pytest.mark.parametrize("fmt", R.FORMATS)
def test_round_nearest_matches_numpy_or_half_ulp(fmt):
    """Round to nearest: fp16 against numpy's own conversion of the float32
    value; bf16 against the exact half-unit bound with ties to an even
    pattern."""
    h = _samples(fmt)
    rn = R.round_nearest(h, fmt)
    if fmt == "fp16":
        assert np.array_equal(rn, h.astype(np.float16).view(np.uint16))
        return
    lo = R.round_toward_zero(h, fmt)
    for hv, r, l in zip(h, rn, lo):
        lof, hif = Fraction(float(R.decode(np.uint16(l), fmt))), Fraction(float(R.decode(np.uint16(l + 1), fmt)))
        H = Fraction(float(hv))
        dl, dh = abs(H - lof), abs(hif - H)
        want = l if dl < dh else (l + 1 if dh < dl else (l if l % 2 == 0 else l + 1))
        assert int(r) == int(want)


@pytest.mark.parametrize("fmt", R.FORMATS)
def test_stochastic_rounding_is_exact_in_expectation(fmt):
    """Averaged over all 65536 keys, SR(h) = h exactly whenever h has at
    most 16 bits below the format's last place (every bf16 case, fp16's
    normal range); otherwise within 2^-16 of a unit. Every result is lo or
    hi. A flipped comparison, a wrong scale or a swapped lo/hi fails."""
    h = _samples(fmt, n=60)
    k = np.arange(65536, dtype=np.uint32)
    for hv in h:
        out = R.stochastic_round(np.full(65536, hv, dtype=np.float32), k, fmt)
        lo = R.round_toward_zero(np.float32(hv), fmt)
        assert set(np.unique(out).tolist()) <= {int(lo), int(lo) + 1}
        vals = R.decode(out, fmt)
        mean = sum(Fraction(float(v)) * int((vals == v).sum()) for v in np.unique(vals)) / 65536
        H = Fraction(float(hv))
        unit = abs(Fraction(float(R.decode(np.uint16(lo + 1), fmt))) - Fraction(float(R.decode(np.uint16(lo), fmt))))
        frac_bits = (abs(H) - abs(Fraction(float(R.decode(np.uint16(lo), fmt))))) / unit * 65536
        if frac_bits.denominator == 1:
            assert mean == H, (hv, float(mean))
        else:
            assert abs(mean - H) < unit / 65536


@pytest.mark.parametrize("fmt", R.FORMATS)
def test_stochastic_rounding_keeps_exact_values_and_is_odd(fmt):
    """Representable values are returned unchanged for every key, and
    SR(-h; k) = -SR(h; k)."""
    rng = np.random.default_rng(5)
    k = rng.integers(0, 65536, 2000).astype(np.uint32)
    exact = R.decode(R.round_nearest(_samples(fmt, 2000, 9)[:2000], fmt), fmt)
    exact = exact[np.isfinite(exact)]
    out = R.stochastic_round(exact, k[:exact.size], fmt)
    assert np.array_equal(R.decode(out, fmt), exact)
    h = _samples(fmt, 2000, 11)
    pos = R.stochastic_round(h, k[:h.size], fmt)
    neg = R.stochastic_round(-h, k[:h.size], fmt)
    assert np.array_equal(pos ^ np.uint16(0x8000), neg)


def test_splitmix64_matches_the_input_generator():
    """The checker's SplitMix64 against the seeded-input module's, written
    separately (that one advances its state by gamma, then mixes): the same
    outputs, and the counter layout (word of counter c = output after c + 1
    advances from the seed)."""
    rng = np.random.default_rng(1)
    states = rng.integers(0, 2**63, 1000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    with np.errstate(over="ignore"):
        assert np.array_equal(R.splitmix64_output(states + R.GAMMA), inputs.splitmix64(states))
    seed, t, n = 0x1234ABCD5678, 3, 50
    w = R.words(seed, t, 1, n)
    with np.errstate(over="ignore"):
        c = np.uint64(((2 * t + 1) * 5 + 2) * n) + np.arange(n, dtype=np.uint64)
        assert np.array_equal(w[2], inputs.splitmix64(np.uint64(seed) + c * R.GAMMA))


def test_keys_are_uniform_and_distinct_per_stream():
    """Keys of one step are uniform over 16 bits (chi-square over 256 bins
    of the top byte) and the f and g streams and successive steps differ."""
    kf = R.keys(7, 0, 0, 40000)
    kg = R.keys(7, 0, 1, 40000)
    k1 = R.keys(7, 1, 0, 40000)
    hist = np.bincount((kf.ravel() >> 8).astype(np.int64), minlength=256)
    expected = kf.size / 256
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 400  # 255 degrees of freedom: mean 255, sd 22.6
    assert (kf == kg).mean() < 1e-3 and (kf == k1).mean() < 1e-3


def test_bf16_round_nearest_matches_torch():
    """bf16 round-to-nearest-even against PyTorch's own float32 -> bfloat16
    conversion (a third implementation), on random values across the range,
    exact ties (half a unit above a pattern, odd and even) and subnormals."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    bits = rng.integers(0, 2**32, 200000, dtype=np.uint64).astype(np.uint32)
    h = bits.view(np.float32)
    h = h[np.isfinite(h)]
    base = rng.integers(0, 2**15, 4000, dtype=np.uint32) << np.uint32(16)
    ties = (base | np.uint32(0x8000)).view(np.float32)               # exactly half a unit
    sub = (rng.integers(1, 2**23, 4000, dtype=np.uint32)).view(np.float32)  # float32 subnormals
    ties = ties[np.isfinite(ties)]  # NaN patterns are not a rounding question
    for x in (h, ties, sub, -ties, -sub):
        ours = R.round_nearest(x, "bf16")
        theirs = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        assert np.array_equal(ours, theirs)
