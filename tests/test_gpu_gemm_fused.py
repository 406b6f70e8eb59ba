"""The fused split + tensor-core GEMM (split in registers inside the kernel,
the conversion of Sec. V "hidden") against the separate split pass + GEMM:
the same pieces go through the same products in the same order, so the two
must agree bit for bit; and against the FP64 oracle product within the
mode's bound."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi
from _tol import check_bound

pytestmark = pytest.mark.gpu


def _padded(a, ld):
    """Device copy of a with row stride ld (>= a.shape[1], a multiple of 4)."""
    r, c = a.shape
    buf = torch.zeros((r, ld), dtype=torch.float32, device="cuda")
    buf[:, :c] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return buf[:, :c]


SHAPES = [(128, 256, 32), (300, 520, 200), (1, 1, 1), (17, 33, 5), (129, 257, 33),
          (256, 512, 512), (640, 300, 77)]


@pytest.mark.parametrize("mode", [1, 3, 6, 8, 9])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_fused_equals_separate_split(bfx, mode, m, n, k):
    A = bi.wide_range((m, k), 10 + m, -12, 12)
    B = bi.wide_range((k, n), 20 + n, -12, 12)
    Ad = _padded(A, (k + 3) // 4 * 4)
    Bd = _padded(B, (n + 3) // 4 * 4)
    C0 = torch.from_numpy(bi.uniform_pm1((m, n), 7)).cuda()
    for alpha, beta in ((1.0, 0.0), (-0.75, 1.25)):
        Cs = C0.clone()
        Cf = C0.clone()
        bfx.gemm_bf16xN(mode, Ad, Bd, Cs, alpha=alpha, beta=beta)
        bfx.gemm_bf16xN_fused(mode, Ad, Bd, Cf, alpha=alpha, beta=beta)
        assert torch.equal(Cs, Cf), (mode, m, n, k, alpha, beta)


@pytest.mark.parametrize("mode", [3, 6])
def test_fused_within_bound_of_fp64(bfx, orc, mode):
    m, n, k = 384, 768, 512
    A = bi.wide_range((m, k), 31)
    B = bi.wide_range((k, n), 32)
    C = bfx.gemm_bf16xN_fused(mode, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    rows = np.arange(0, m, 7)
    C64, absAB = orc.dgemm_rows(A, B, rows)
    check_bound(C.cpu().numpy()[rows], C64, absAB, mode, k)


def test_fused_special_values_propagate(bfx):
    """Inf and NaN pieces (hi carries the value) give the same result as the
    separate split."""
    sv = bi.special_values_f32()
    k = sv.size + (-sv.size) % 4
    A = np.zeros((8, k), np.float32)
    A[0, : sv.size] = sv
    A[1:, :] = bi.uniform_pm1((7, k), 3)
    B = bi.uniform_pm1((k, 16), 4)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cs = bfx.gemm_bf16xN(6, Ad, Bd)
    Cf = bfx.gemm_bf16xN_fused(6, Ad, Bd)
    assert torch.equal(torch.isnan(Cs), torch.isnan(Cf))
    ok = ~torch.isnan(Cs)
    assert torch.equal(Cs[ok], Cf[ok])


def test_fused_rejects_unaligned_rows(bfx):
    A = torch.zeros((8, 7), device="cuda")
    B = torch.zeros((7, 8), device="cuda")
    with pytest.raises(bfx.BfxError) as e:
        bfx.gemm_bf16xN_fused(6, A, B)  # lda = 7
    assert e.value.code == 4
    with pytest.raises(bfx.BfxError) as e:
        bfx.gemm_bf16xN_fused(0, torch.zeros((8, 8), device="cuda"), torch.zeros((8, 8), device="cuda"))
    assert e.value.code == 1


@pytest.mark.parametrize("mode", [3, 6])
def test_fused_long_k_within_bound(bfx, orc, mode):
    """Beyond K = 512 the separate path accumulates hi*hi in chunks of 256
    (round-to-nearest chunk sums) while the fused kernel keeps one
    accumulator: both stay within the mode's bound of the FP64 product."""
    m, n, k = 256, 512, 1000
    A = bi.wide_range((m, k), 41)
    B = bi.wide_range((k, n), 42)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    rows = np.arange(0, m, 5)
    C64, absAB = orc.dgemm_rows(A, B, rows)
    for C in (bfx.gemm_bf16xN_fused(mode, Ad, Bd), bfx.gemm_bf16xN(mode, Ad, Bd)):
        check_bound(C.cpu().numpy()[rows], C64, absAB, mode, k)
