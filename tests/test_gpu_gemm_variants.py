"""Two GEMM variants of the paper on the tensor cores, against the oracle.

* x5, the asymmetric split of Sec. II-G: A in two bfloat16 pieces, B in
  three, products {00, 01, 10, 02, 11}.
* The "d" collection of Sec. IV-A (bfx_gemm_bf16xN_f64): every product in its
  own FP32 accumulator, the partial products added in FP64 and C kept in FP64.

Both are held to the elementwise bounds of tests/_tol.py against the FP64
product and to the oracle's model of the same variant within the sum of both
bounds; exact special cases (permutation operands) must match bit for bit.
"""
import numpy as np
import pytest
import torch

import bfx_inputs as bi
from _tol import check_bound, tol

pytestmark = pytest.mark.gpu

SHAPES = [
    (128, 64, 32),      # one 64-wide tile of the FP64 variant
    (300, 520, 200),    # several tiles, ragged in m, n and k
    (1, 1, 1),
    (17, 33, 5),        # k below one K-slice
    (129, 257, 1000),
]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sixteen_bit(shape, seed):
    x = bi.uniform_pm1(shape, seed)
    return (x.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("gen", ["uniform", "wide"])
def test_x5_bounds_vs_fp64_and_oracle(bfx, orc, m, n, k, gen):
    if gen == "uniform":
        A, B = bi.uniform_pm1((m, k), 80), bi.uniform_pm1((k, n), 81)
    else:
        A, B = bi.wide_range((m, k), 82), bi.wide_range((k, n), 83)
    C = bfx.gemm_bf16xN(bfx.BFX_X5, _cuda(A), _cuda(B)).cpu().numpy()
    C64, Cabs = orc.dgemm_rows(A, B)
    check_bound(C, C64, Cabs, 5, k)
    Co = orc.gemm(5, A, B)
    assert np.all(np.abs(C.astype(np.float64) - Co) <= 2 * tol(5, k) * Cabs + 1e-38)


def test_x5_permutation_exact(bfx, orc):
    """P B keeps every piece of B (products (0, j)); A Q keeps only A's two
    pieces (products (i, 0)): a third piece of A would show up here."""
    rng = np.random.default_rng(84)
    n = 160
    P = np.zeros((n, n), np.float32)
    perm = rng.permutation(n)
    P[np.arange(n), perm] = 1.0
    B = bi.wide_range((n, 300), 85, -30, 30)
    A = bi.wide_range((200, n), 86, -30, 30)
    C1 = bfx.gemm_bf16xN(bfx.BFX_X5, _cuda(P), _cuda(B)).cpu().numpy()
    assert np.array_equal(C1, B[perm])
    C2 = bfx.gemm_bf16xN(bfx.BFX_X5, _cuda(A), _cuda(P.T.copy())).cpu().numpy()
    assert np.array_equal(C2, orc.gemm(5, A, P.T.copy()))
    assert not np.array_equal(C2, A[:, perm])  # A's third piece is dropped


def test_x5_reaches_fp32_accuracy_only_without_a_third_piece(bfx, orc):
    """Sec. II-G: x5 is held to x6's (FP32-level) bound when A has at most 16
    significant bits, and is far less accurate than x6 otherwise."""
    m, n, k = 256, 320, 512
    B = bi.uniform_pm1((k, n), 88)
    A16 = _sixteen_bit((m, k), 87)
    C64, Cabs = orc.dgemm_rows(A16, B)
    C5 = bfx.gemm_bf16xN(bfx.BFX_X5, _cuda(A16), _cuda(B)).cpu().numpy()
    check_bound(C5, C64, Cabs, 6, k)
    # k = 128: the tensor core's accumulation error (which grows with k, see
    # the x6 accuracy reading) stays below the 2^-16 term being compared
    kr = 128
    A, B = bi.uniform_pm1((m, kr), 89), B[:kr]
    C64, _ = orc.dgemm_rows(A, B)
    e = {md: np.linalg.norm(bfx.gemm_bf16xN(md, _cuda(A), _cuda(B)).cpu().numpy() - C64)
         for md in (3, 5, 6)}
    assert e[5] >= 10 * e[6] and e[5] < e[3], e


def test_x5_presplit_two_and_three_planes(bfx):
    m, n, k = 256, 384, 160
    A = _cuda(bi.uniform_pm1((m, k), 90))
    B = _cuda(bi.uniform_pm1((k, n), 91))
    Ap = torch.zeros((2, m, k), dtype=torch.int16, device="cuda")
    Bp = torch.zeros((3, n, k), dtype=torch.int16, device="cuda")
    bfx.split(A, 2, out=[Ap[i] for i in range(2)])
    bfx.split_transpose(B, 3, out=[Bp[i] for i in range(3)])
    C1 = torch.empty((m, n), device="cuda")
    bfx.gemm_presplit(bfx.BFX_X5, Ap, Bp, k, C1)
    assert torch.equal(C1, bfx.gemm_bf16xN(bfx.BFX_X5, A, B))


def test_x5_rejected_outside_the_gemm(bfx):
    A = torch.eye(64, device="cuda")
    with pytest.raises(bfx.BfxError):
        bfx.gemm_bf16xN_fused(bfx.BFX_X5, A, A)
    with pytest.raises(bfx.BfxError):
        bfx.lu_bf16xN(bfx.BFX_X5, A.clone())


# ---------------------------------------------------------------- FP64 collection
F64_MODES = [1, 3, 5, 6, 8, 9]


@pytest.mark.parametrize("mode", F64_MODES)
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_f64_bounds_vs_fp64_and_oracle(bfx, orc, mode, m, n, k):
    A, B = bi.wide_range((m, k), 92), bi.wide_range((k, n), 93)
    C = bfx.gemm_bf16xN_f64(mode, _cuda(A), _cuda(B))
    assert C.dtype == torch.float64
    C = C.cpu().numpy()
    C64, Cabs = orc.dgemm_rows(A, B)
    check_bound(C, C64, Cabs, mode, k)
    Co = orc.gemm_f64out(mode, A, B)
    assert np.all(np.abs(C - Co) <= 2 * tol(mode, k) * Cabs + 1e-300)


@pytest.mark.parametrize("mode", F64_MODES)
def test_f64_permutation_exact(bfx, orc, mode):
    """P B and A Q: the kept pieces, summed exactly in FP64 (no rounding to
    FP32 at the end): x6, x8, x9 return B's rows exactly; every mode equals
    the oracle's FP64 collection bit for bit."""
    rng = np.random.default_rng(94)
    n = 96
    P = np.zeros((n, n), np.float32)
    perm = rng.permutation(n)
    P[np.arange(n), perm] = 1.0
    B = bi.wide_range((n, 200), 95, -30, 30)
    A = bi.wide_range((150, n), 96, -30, 30)
    C1 = bfx.gemm_bf16xN_f64(mode, _cuda(P), _cuda(B)).cpu().numpy()
    assert np.array_equal(C1, orc.gemm_f64out(mode, P, B))
    if mode in (5, 6, 8, 9):
        assert np.array_equal(C1, B[perm].astype(np.float64))
    C2 = bfx.gemm_bf16xN_f64(mode, _cuda(A), _cuda(P.T.copy())).cpu().numpy()
    assert np.array_equal(C2, orc.gemm_f64out(mode, A, P.T.copy()))


def test_f64_strided_output(bfx, orc):
    m, n, k = 150, 140, 90
    A, B = bi.uniform_pm1((m, k), 97), bi.uniform_pm1((k, n), 98)
    Cbig = torch.zeros((m, n + 9), dtype=torch.float64, device="cuda")
    bfx.gemm_bf16xN_f64(6, _cuda(A), _cuda(B), Cbig[:, 1:n + 1])
    C64, Cabs = orc.dgemm_rows(A, B)
    check_bound(Cbig[:, 1:n + 1].cpu().numpy(), C64, Cabs, 6, k)
    assert (Cbig[:, 0] == 0).all() and (Cbig[:, n + 1:] == 0).all()


@pytest.mark.slow
@pytest.mark.parametrize("variant", ["x5", "x6_f64"])
def test_variants_full_size_sampled_rows(bfx, orc, variant):
    """8192^3, the size bench.py times the variants at, wide-range inputs; 32
    random rows against the FP64 oracle."""
    m = n = k = 8192
    A = bi.wide_range((m, k), 60)
    B = bi.wide_range((k, n), 61)
    if variant == "x5":
        C, mode = bfx.gemm_bf16xN(bfx.BFX_X5, _cuda(A), _cuda(B)), 5
    else:
        C, mode = bfx.gemm_bf16xN_f64(6, _cuda(A), _cuda(B)), 6
    rows = np.sort(np.random.default_rng(99).choice(m, 32, replace=False))
    rows[-1] = m - 1
    Cs = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    C64, Cabs = orc.dgemm_rows(A, B, rows)
    check_bound(Cs, C64, Cabs, mode, k)
