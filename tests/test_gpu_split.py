"""Device split (Sec. II-A) against the oracle: bit-exact, every FP32 pattern."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _to_u16(t):
    return t.cpu().numpy().view(np.uint16)


@pytest.mark.slow
def test_split_exhaustive_all_fp32_patterns(bfx, orc):
    """All 2^32 inputs, chunk by chunk: hi, mid, lo bit-identical to the oracle."""
    chunk = 1 << 27
    x = torch.empty(chunk, dtype=torch.int32, device="cuda")
    pieces = [torch.empty((1, chunk), dtype=torch.int16, device="cuda") for _ in range(3)]
    base = torch.arange(chunk, dtype=torch.int64, device="cuda")
    for start in range(0, 1 << 32, chunk):
        v = base + start  # the bit patterns start .. start+chunk-1 as signed 32-bit ints
        x.copy_(torch.where(v >= 2**31, v - 2**32, v).to(torch.int32))
        bfx.split(x.view(torch.float32).view(1, chunk), 3, out=pieces)
        got = [_to_u16(p).ravel() for p in pieces]
        exp = orc.split_bits_range(start, chunk, 3)
        for g, e, name in zip(got, exp, ("hi", "mid", "lo")):
            if not np.array_equal(g, e):
                i = int(np.argmax(g != e))
                pytest.fail(f"{name} differs at input {start + i:#010x}: {g[i]:#06x} vs {e[i]:#06x}")


@pytest.mark.parametrize("rows,cols,ldx,npieces", [
    (37, 53, 53, 3),     # scalar path, ragged
    (64, 256, 256, 3),   # vectorised path
    (64, 256, 264, 2),   # padded rows
    (1, 8, 8, 1),
    (300, 96, 100, 3),   # ld not a multiple of 8: scalar path
])
def test_split_matrix_layouts(bfx, orc, rows, cols, ldx, npieces):
    full = bi.wide_range((rows, ldx), 7, -40, 40)
    x = torch.from_numpy(full).cuda()[:, :cols]
    got = bfx.split(x, npieces)
    exp = orc.split(full[:, :cols], npieces)
    for g, e in zip(got, exp):
        assert np.array_equal(_to_u16(g), e)


@pytest.mark.parametrize("rows,cols", [(37, 53), (64, 64), (130, 257), (1, 1), (256, 8)])
def test_split_transpose(bfx, orc, rows, cols):
    xa = bi.wide_range((rows, cols), 8, -20, 20)
    x = torch.from_numpy(xa).cuda()
    got = bfx.split_transpose(x, 3)
    exp = orc.split(xa.T.copy(), 3)
    for g, e in zip(got, exp):
        assert np.array_equal(_to_u16(g), e)


def test_split_special_values(bfx, orc):
    xa = bi.special_values_f32().reshape(1, -1).copy()
    got = bfx.split(torch.from_numpy(xa).cuda(), 3)
    for g, e in zip(got, orc.split(xa, 3)):
        assert np.array_equal(_to_u16(g), e)


def test_split_empty(bfx):
    x = torch.empty((0, 5), dtype=torch.float32, device="cuda")
    assert [p.shape for p in bfx.split(x, 3)] == [(0, 5)] * 3


@pytest.mark.parametrize("ma,ka,kb,nb,npa,npb", [
    (256, 512, 512, 384, 3, 3),   # one launch: A contiguous, B's planes 16-byte aligned
    (1000, 64, 64, 777, 2, 3),    # one launch, ragged B tiles
    (33, 40, 40, 129, 3, 2),      # one launch, small
    (37, 53, 53, 70, 3, 3),       # A's width not a multiple of 8: two launches
    (0, 16, 16, 20, 3, 3),        # empty A
])
def test_split_pair_equals_split_and_transpose(bfx, ma, ka, kb, nb, npa, npb):
    """split_pair gives the pieces of split(A) and split_transpose(B) bit for
    bit, in the combined launch and in the two-launch fallback (wide-range
    values, so every piece is populated)."""
    A = torch.from_numpy(bi.wide_range((ma, ka), ma + ka)).cuda()
    B = torch.from_numpy(bi.wide_range((kb, nb), kb + nb)).cuda()
    pa, pb = bfx.split_pair(A, B, npa, npb)
    if ma:
        ea = bfx.split(A, npa)
        for g, e in zip(pa, ea):
            assert torch.equal(g, e)
    eb = bfx.split_transpose(B, npb)
    for g, e in zip(pb, eb):
        assert torch.equal(g, e)
