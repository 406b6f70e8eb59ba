"""Pins of the oracle's (B16) conversion and split (Sec. I, II-A, II-F, II-G).

Nothing here compares the oracle with itself: expected values come from
hand-worked golden files, from torch's own float32->bfloat16 conversion (an
independent library routine), from a brute-force nearest-neighbour search,
and from the exactness and bin-bound invariants the paper states.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import bfx_inputs as bi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            toks = line.split()
            vals = []
            for t in toks:
                if t.startswith("0x"):
                    vals.append(int(t, 16))
                else:
                    break
            rows.append(vals)
    return rows


def _bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def _f32(bits):
    return np.asarray(bits, dtype=np.uint32).view(np.float32)


def _exact(bits16):
    """Exact rational value of a bfloat16 bit pattern (via its FP32 widening)."""
    v = float(np.uint32(int(bits16) << 16).view(np.float32))
    return Fraction(v)


# --------------------------------------------------------------- (B16)
def test_rne_golden(orc):
    rows = _read_golden("bf16_rne.txt")
    assert len(rows) >= 20
    x = _f32([r[0] for r in rows])
    got = orc.bf16_rne(x)
    for (inp, exp), g in zip(rows, got):
        assert int(g) == exp, f"{inp:#010x}: got {int(g):#06x}, expected {exp:#06x}"


def test_rne_matches_torch_bfloat16(orc):
    """torch's CPU float32 -> bfloat16 cast is an independent RNE implementation."""
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2**32, size=2_000_000, dtype=np.uint64).astype(np.uint32)
    # force many exact ties and near-ties
    bits[::4] = (bits[::4] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    bits[1::8] = (bits[1::8] & np.uint32(0xFFFF0000)) | np.uint32(0x7FFF)
    bits[2::8] = (bits[2::8] & np.uint32(0xFFFF0000)) | np.uint32(0x8001)
    x = _f32(bits)
    finite = np.isfinite(x)
    ours = orc.bf16_rne(x)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours[finite], ref[finite])
    # NaN stays NaN (torch canonicalises the payload; ours keeps sign and top bits)
    nan = np.isnan(x)
    ours_f = (ours[nan].astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isnan(ours_f))


def test_rne_bruteforce_nearest(orc):
    """Pick the nearest bfloat16 among all candidates by exact distance; ties to even."""
    rng = np.random.default_rng(12)
    bits = rng.integers(0x00000000, 0x7F7F0000, size=3000, dtype=np.uint64).astype(np.uint32)
    bits[::3] = (bits[::3] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    sign = rng.integers(0, 2, size=bits.size).astype(np.uint32) << np.uint32(31)
    bits = bits | sign
    got = orc.bf16_rne(_f32(bits))
    for b, g in zip(bits, got):
        xv = Fraction(float(_f32(b)))
        top = int(b) >> 16
        cands = [c & 0xFFFF for c in (top - 1, top, top + 1, top + 2) if 0 <= (c & 0x7FFF) <= 0x7F7F]
        cands = [c for c in cands if (c >> 15) == (top >> 15) or (c & 0x7FFF) == 0]
        dist = {c: abs(_exact(c) - xv) for c in cands}
        best = min(dist.values())
        winners = [c for c, d in dist.items() if d == best]
        if len(winners) > 1:
            winners = [c for c in winners if c % 2 == 0]
        assert int(g) in winners, (hex(int(b)), hex(int(g)), [hex(w) for w in winners])


# --------------------------------------------------------------- split
def test_split_golden(orc):
    rows = _read_golden("split.txt")
    x = _f32([r[0] for r in rows])
    hi, mid, lo = orc.split(x, 3)
    for r, h, m, l in zip(rows, hi, mid, lo):
        assert (int(h), int(m), int(l)) == tuple(r[1:4]), hex(r[0])


def _stratified_bits(low_per_high=48, seed=0):
    """Every sign/exponent/top-7-mantissa pattern with a set of low halves."""
    rng = np.random.default_rng(seed)
    high = np.arange(1 << 16, dtype=np.uint32) << np.uint32(16)
    fixed = np.array([0x0000, 0x0001, 0x7FFF, 0x8000, 0x8001, 0xFFFF, 0x5555, 0xAAAA], np.uint32)
    rand = rng.integers(0, 1 << 16, size=low_per_high - fixed.size, dtype=np.uint32)
    low = np.concatenate([fixed, rand]).astype(np.uint32)
    return (high[:, None] | low[None, :]).ravel()


def test_split_exact_sum_in_domain(orc):
    """hi + mid + lo == a exactly for finite |a| >= 2^-110 (Sec. II-A, II-F)."""
    bits = _stratified_bits()
    x = _f32(bits)
    fin = np.isfinite(x)
    x, bits = x[fin], bits[fin]
    hi, mid, lo = (orc.bf16_to_f32(p).astype(np.float64) for p in orc.split(x, 3))
    ax = np.abs(x.astype(np.float64))
    dom = (ax >= 2.0**-110) | (ax == 0)
    s = hi + mid + lo  # three terms spanning < 53 bits: exact in FP64
    bad = dom & (s != x.astype(np.float64))
    assert not bad.any(), hex(int(bits[np.argmax(bad)]))
    assert dom.sum() > 0.8 * dom.size


def test_split_domain_edge_is_minus_110(orc):
    """Sec. II-F: exponent -110 is the lowest at which the split is exact for every value."""
    rng = np.random.default_rng(3)

    def frac_exact(e):
        m = rng.integers(0, 1 << 23, size=200_000, dtype=np.uint32)
        bits = (np.uint32(e + 127) << np.uint32(23)) | m
        x = _f32(bits)
        pieces = [orc.bf16_to_f32(p).astype(np.float64) for p in orc.split(x, 3)]
        return np.mean(sum(pieces) == x.astype(np.float64))

    assert frac_exact(-110) == 1.0
    assert frac_exact(-109) == 1.0
    assert frac_exact(-111) < 0.75


def test_split_full_binades_exhaustive(orc):
    """Every pattern of the binades [1,2), [2^-110, 2^-109) and the top binade."""
    for e in (0, -110, 127):
        bits = (np.uint32(e + 127) << np.uint32(23)) | np.arange(1 << 23, dtype=np.uint32)
        for sgn in (0, 1):
            b = bits | np.uint32(sgn << 31)
            x = _f32(b)
            pieces = [orc.bf16_to_f32(p).astype(np.float64) for p in orc.split(x, 3)]
            assert np.array_equal(pieces[0] + pieces[1] + pieces[2], x.astype(np.float64)), e


def test_split_bin_bounds(orc):
    """|b1| <= 2^-8 |b0| and |b2| <= 2^-8 |b1| (Sec. II-G), hence |b2| <= 2^-16 |b0|."""
    bits = _stratified_bits(low_per_high=24, seed=1)
    x = _f32(bits)
    mag = bits & np.uint32(0x7FFFFFFF)
    rne = mag < 0x7F7F8000  # below the values whose hi is truncated (reading R3)
    trunc = (mag >= 0x7F7F8000) & (mag < 0x7F800000)
    hi, mid, lo = (np.abs(orc.bf16_to_f32(p).astype(np.float64)) for p in orc.split(x, 3))
    assert np.all(mid[rne] <= 2.0**-8 * hi[rne])
    assert np.all(lo[rne] <= 2.0**-8 * mid[rne])
    assert np.all(lo[rne] <= 2.0**-16 * hi[rne])
    # truncated hi: the remainder is below one bfloat16 ulp of hi, 2^-7 |hi|
    assert trunc.sum() > 0
    assert np.all(mid[trunc] <= 2.0**-7 * hi[trunc])
    assert np.all(lo[trunc] <= 2.0**-8 * mid[trunc])


def test_pair_split_is_prefix_of_triple(orc):
    x = bi.wide_range(100_000, 5, -30, 30)
    h2, m2 = orc.split(x, 2)
    h3, m3, _ = orc.split(x, 3)
    assert np.array_equal(h2, h3) and np.array_equal(m2, m3)
    (h1,) = orc.split(x, 1)
    assert np.array_equal(h1, h3)


def test_split_already_bfloat16_has_zero_tail(orc):
    """A value that is already a bfloat16 is its own hi; mid = lo = 0."""
    rng = np.random.default_rng(4)
    top = rng.integers(0, 0x7F7F, size=50_000, dtype=np.uint32)
    x = _f32(top << np.uint32(16))
    hi, mid, lo = orc.split(x, 3)
    assert np.array_equal(hi.astype(np.uint32), top)
    assert not mid.any() and not lo.any()


def test_split_statistics_768(orc):
    """Sec. II-G: on uniform data mean |a1| ~ |a0|/768 and |a2| ~ |a0|/768^2.

    The paper's derivation is a heuristic estimate; measured with RNE it comes
    out within a few percent (truncation instead would give about 1/370).
    """
    x = bi.uniform_pm1(2_000_000, 21)
    hi, mid, lo = (np.abs(orc.bf16_to_f32(p).astype(np.float64)) for p in orc.split(x, 3))
    r1 = 1.0 / np.mean(mid / hi)
    r2 = 1.0 / np.mean(lo / hi)
    assert abs(r1 / 768 - 1) < 0.06, r1
    assert abs(r2 / 768**2 - 1) < 0.06, r2


def test_split_error_term_statistic(orc):
    """Sec. II-G: E = a1 b2 + a2 b1 + a2 b2 averages about 4.412e-9 |a0 b0|."""
    x = bi.uniform_pm1(2_000_000, 22)
    y = bi.uniform_pm1(2_000_000, 23)
    a0, a1, a2 = (orc.bf16_to_f32(p).astype(np.float64) for p in orc.split(x, 3))
    b0, b1, b2 = (orc.bf16_to_f32(p).astype(np.float64) for p in orc.split(y, 3))
    c = np.mean((np.abs(a1 * b2) + np.abs(a2 * b1) + np.abs(a2 * b2)) / np.abs(a0 * b0))
    assert abs(c / 4.412e-9 - 1) < 0.15, c
    # worst case of Sec. II-G: |E| <= (513/512) 2^-23 |a0 b0|
    E = np.abs(a1 * b2 + a2 * b1 + a2 * b2)
    assert np.all(E <= (513 / 512) * 2.0**-23 * np.abs(a0 * b0))


def test_split_bits_range_matches_split(orc):
    start = 0x3F000000
    p_range = orc.split_bits_range(start, 1 << 16, 3)
    x = _f32(np.arange(start, start + (1 << 16), dtype=np.uint64).astype(np.uint32))
    p_arr = orc.split(x, 3)
    for a, b in zip(p_range, p_arr):
        assert np.array_equal(a, b)
