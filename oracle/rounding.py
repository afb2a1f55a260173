"""Stochastic rounding of the 16-bit storage forms, as plain numpy: the
checker for the library's LD_ROUND_STOCHASTIC stores.

Test infrastructure only (tests, smoke() and the bench's CPU leg use it);
the library never imports it and shares no code with it.

The paper fixes no storage precision or rounding; the 16-bit deviation
forms and their rounding are readings. Stochastic rounding here is the
standard "mode 1" (Connolly, Higham & Mary, SIAM J. Sci. Comput. 43 (2021)
A566): a value between two neighbours of the target format rounds up with
probability equal to its distance from the lower one, in units of their
spacing. Its random integers come from SplitMix64 (Steele, Lea & Flood,
OOPSLA 2014) used as a counter-based generator.

Definitions (both fixed by the library's header, restated here from those
publications):
  * h: the FP32 deviation x - ref that a store rounds.
  * lo = h rounded toward zero to the format, hi = the next value of the
    format away from zero (magnitude one unit in the last place larger).
  * the stored value is hi when k (|hi| - |lo|) < 65536 (|h| - |lo|), else
    lo, for the 16-bit random integer k; exact values and the largest finite
    magnitude are kept.
  * SplitMix64: state s advances by gamma = 0x9E3779B97F4A7C15 (mod 2^64);
    the output of state z is z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
    z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
  * the word of step t, array a (0 f, 1 g), quarter q of the directions and
    site s is the output of state seed + (c + 1) gamma with
    c = ((2t + a) 5 + q) N + s; direction i takes bits 16 (i % 4) .. +15 of
    the word of quarter i // 4.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)
Q = 19
FORMATS = ("fp16", "bf16")


def splitmix64_output(state):
    """The SplitMix64 output function of (an array of) 64-bit states."""
    z = np.asarray(state, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _MIX1
        z ^= z >> np.uint64(27)
        z *= _MIX2
        z ^= z >> np.uint64(31)
    return z


def words(seed, t, a, n):
    """The five random words (5, n) of step t, array a, for sites 0..n-1."""
    s = np.arange(n, dtype=np.uint64)
    out = np.empty((5, n), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for q in range(5):
            c = np.uint64(((2 * t + a) * 5 + q) * n) + s
            out[q] = splitmix64_output(np.uint64(seed) + (c + np.uint64(1)) * GAMMA)
    return out


def keys(seed, t, a, n):
    """The 16-bit random integers (19, n) of step t and array a: direction i
    of site s takes bits 16 (i % 4) .. 16 (i % 4) + 15 of word i // 4."""
    w = words(seed, t, a, n)
    return np.stack([(w[i // 4] >> np.uint64(16 * (i % 4))) & np.uint64(0xFFFF) for i in range(Q)]).astype(np.uint32)


def _max_finite_bits(fmt):
    return 0x7BFF if fmt == "fp16" else 0x7F7F


def decode(bits, fmt):
    """Values (float32) of 16-bit patterns of the format."""
    bits = np.asarray(bits, dtype=np.uint16)
    if fmt == "fp16":
        return bits.view(np.float16).astype(np.float32)
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)


def round_nearest(h, fmt):
    """Round-to-nearest-even 16-bit patterns of float32 values."""
    h = np.asarray(h, dtype=np.float32)
    if fmt == "fp16":
        return h.astype(np.float16).view(np.uint16)
    u = h.view(np.uint32).astype(np.uint64)
    # add half an ulp of the target, plus one if the kept part is odd (ties to even)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    out = r.astype(np.uint16)
    return np.where(np.isnan(h), np.uint16(0x7FFF), out)


def round_toward_zero(h, fmt):
    """16-bit patterns of float32 values rounded toward zero."""
    h = np.asarray(h, dtype=np.float32)
    if fmt == "bf16":
        out = (h.view(np.uint32) >> np.uint32(16)).astype(np.uint16)
        return np.where(np.isnan(h), np.uint16(0x7FFF), out)
    # nearest first, then one step toward zero where it went past h
    b = h.astype(np.float16).view(np.uint16).copy()
    back = b.view(np.float16).astype(np.float32)
    over = (np.abs(back) > np.abs(h)) & ~np.isnan(h)
    b[over] -= np.uint16(1)  # sign-magnitude: one unit less in magnitude
    return b


def stochastic_round(h, k, fmt):
    """16-bit patterns of float32 deviations h rounded stochastically with
    the 16-bit integers k (same shape)."""
    h = np.asarray(h, dtype=np.float32)
    k = np.asarray(k)
    lo = round_toward_zero(h, fmt)
    lof = decode(lo, fmt)
    keep = (lof == h) | ((lo & np.uint16(0x7FFF)) == np.uint16(_max_finite_bits(fmt))) | np.isnan(h)
    hi = (lo + np.uint16(1)).astype(np.uint16)
    hif = decode(hi, fmt)
    with np.errstate(invalid="ignore", over="ignore"):
        gap = np.abs(hif) - np.abs(lof)  # float32, a power of two
        d = np.abs(h) - np.abs(lof)      # float32, exact
        up = k.astype(np.float32) * gap < d * np.float32(65536.0)
    return np.where(keep, lo, np.where(up, hi, lo)).astype(np.uint16)
