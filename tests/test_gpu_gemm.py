"""Tensor-core bf16xN GEMM and the FP32 SIMT baseline against the oracle.

* FP32 SIMT: bit-identical to the oracle's FP32 FMA model (Sec. II-C), which
  accumulates each element with one FMA per k in the same order.
* bf16xN: tensor-core accumulation order and rounding are not the sequential
  FMA of the paper's model, so the result is held to the elementwise bounds of
  tests/_tol.py against the FP64 product, and compared element by element with
  the oracle's FP32 model within the sum of both bounds.  Exact special cases
  (permutation operands) must match bit for bit.
"""
import numpy as np
import pytest
import torch

import bfx_inputs as bi
from _tol import check_bound, tol

pytestmark = pytest.mark.gpu
MODES = [1, 3, 6, 8, 9]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [
    (128, 256, 64),     # exactly one tile
    (300, 520, 200),    # several tiles, ragged in m, n and k
    (1, 1, 1),
    (17, 33, 5),        # k below one K-slice
    (256, 512, 1000),
    (129, 257, 33),
]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_sgemm_simt_bit_exact(bfx, orc, m, n, k):
    A = bi.uniform_pm1((m, k), 1)
    B = bi.wide_range((k, n), 2, -10, 10)
    C = bfx.sgemm_simt(_cuda(A), _cuda(B)).cpu().numpy()
    assert np.array_equal(C, orc.gemm(0, A, B))


def test_sgemm_simt_alpha_beta_and_unaligned(bfx, orc):
    m, n, k = 77, 91, 45
    Af = bi.uniform_pm1((m, k + 3), 3)
    Bf = bi.uniform_pm1((k, n + 1), 4)
    C0 = bi.uniform_pm1((m, n), 5)
    A, B = _cuda(Af)[:, 1:k + 1], _cuda(Bf)[:, :n]  # misaligned A, odd ldb
    Cd = _cuda(C0)
    bfx.sgemm_simt(A, B, Cd, alpha=-1.0, beta=1.0)
    exp = orc.gemm(0, Af[:, 1:k + 1], Bf[:, :n], alpha=-1.0, beta=1.0, C=C0)
    assert np.array_equal(Cd.cpu().numpy(), exp)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("gen", ["uniform", "wide"])
def test_gemm_bounds_vs_fp64(bfx, orc, mode, m, n, k, gen):
    if gen == "uniform":
        A, B = bi.uniform_pm1((m, k), 10), bi.uniform_pm1((k, n), 11)
    else:
        A, B = bi.wide_range((m, k), 12), bi.wide_range((k, n), 13)
    C = bfx.gemm_bf16xN(mode, _cuda(A), _cuda(B)).cpu().numpy()
    C64, Cabs = orc.dgemm_rows(A, B)
    check_bound(C, C64, Cabs, mode, k)
    # element by element against the oracle's FP32 FMA model of the same mode
    Co = orc.gemm(mode, A, B)
    assert np.all(np.abs(C.astype(np.float64) - Co) <= 2 * tol(mode, k) * Cabs + 1e-38)


@pytest.mark.parametrize("mode", MODES)
def test_gemm_permutation_exact(bfx, orc, mode):
    """P B and A Q are exact: the kept pieces of B's rows / A's columns."""
    rng = np.random.default_rng(20)
    n = 160
    perm = rng.permutation(n)
    P = np.zeros((n, n), np.float32)
    P[np.arange(n), perm] = 1.0
    B = bi.wide_range((n, 300), 21, -30, 30)
    A = bi.wide_range((200, n), 22, -30, 30)
    C1 = bfx.gemm_bf16xN(mode, _cuda(P), _cuda(B)).cpu().numpy()
    assert np.array_equal(C1, orc.gemm(mode, P, B))
    C2 = bfx.gemm_bf16xN(mode, _cuda(A), _cuda(P.T.copy())).cpu().numpy()
    assert np.array_equal(C2, orc.gemm(mode, A, P.T.copy()))
    if mode in (6, 8, 9):
        assert np.array_equal(C1, B[perm])


@pytest.mark.parametrize("mode", [3, 6])
def test_gemm_alpha_beta_update_form(bfx, orc, mode):
    """C <- C - A B, the LU trailing update (alpha = -1, beta = 1)."""
    m, n, k = 200, 300, 64
    A, B = bi.uniform_pm1((m, k), 30), bi.uniform_pm1((k, n), 31)
    C0 = bi.uniform_pm1((m, n), 32)
    Cd = _cuda(C0)
    bfx.gemm_bf16xN(mode, _cuda(A), _cuda(B), Cd, alpha=-1.0, beta=1.0)
    C64, Cabs = orc.dgemm_rows(A, B)
    check_bound(Cd.cpu().numpy(), C64, Cabs, mode, k, alpha=-1.0, Cin=C0, beta=1.0)
    # beta = 0 must not read C (NaN there stays out of the result)
    Cn = torch.full((m, n), float("nan"), device="cuda")
    bfx.gemm_bf16xN(mode, _cuda(A), _cuda(B), Cn, alpha=2.0, beta=0.0)
    assert torch.isfinite(Cn).all()


def test_gemm_strided_output_and_inputs(bfx, orc):
    m, n, k = 150, 140, 90
    Af = bi.uniform_pm1((m, k + 5), 40)
    Bf = bi.uniform_pm1((k, n + 7), 41)
    Cbig = torch.zeros((m, n + 9), device="cuda")
    A, B = _cuda(Af)[:, 2:k + 2], _cuda(Bf)[:, 3:n + 3]
    bfx.gemm_bf16xN(6, A, B, Cbig[:, 1:n + 1])
    C64, Cabs = orc.dgemm_rows(Af[:, 2:k + 2], Bf[:, 3:n + 3])
    check_bound(Cbig[:, 1:n + 1].cpu().numpy(), C64, Cabs, 6, k)
    assert (Cbig[:, 0] == 0).all() and (Cbig[:, n + 1:] == 0).all()  # nothing outside C


def test_gemm_empty_and_k0(bfx):
    A = torch.empty((5, 0), device="cuda")
    B = torch.empty((0, 7), device="cuda")
    C = torch.full((5, 7), 3.0, device="cuda")
    bfx.gemm_bf16xN(6, A, B, C, alpha=1.0, beta=2.0)
    assert (C == 6.0).all()
    bfx.gemm_bf16xN(6, torch.empty((0, 4), device="cuda"), torch.empty((4, 3), device="cuda"),
                    torch.empty((0, 3), device="cuda"))


def test_gemm_presplit_matches_split_path(bfx):
    m, n, k = 256, 384, 160
    A = _cuda(bi.uniform_pm1((m, k), 50))
    B = _cuda(bi.uniform_pm1((k, n), 51))
    Ap = torch.zeros((3, m, k), dtype=torch.int16, device="cuda")
    Bp = torch.zeros((3, n, k), dtype=torch.int16, device="cuda")
    bfx.split(A, 3, out=[Ap[i] for i in range(3)])
    bfx.split_transpose(B, 3, out=[Bp[i] for i in range(3)])
    C1 = torch.empty((m, n), device="cuda")
    bfx.gemm_presplit(6, Ap, Bp, k, C1)
    C2 = bfx.gemm_bf16xN(6, A, B)
    assert torch.equal(C1, C2)


@pytest.mark.slow
@pytest.mark.parametrize("mode", [3, 6])
@pytest.mark.parametrize("m,n,k", [(8192, 8192, 8192), (16384, 16384, 256)])
def test_gemm_full_size_sampled_rows(bfx, orc, mode, m, n, k):
    """The benchmark's sizes and launch configuration, wide-range inputs; 48
    random rows checked against the FP64 oracle (rows are independent)."""
    A = bi.wide_range((m, k), 60)
    B = bi.wide_range((k, n), 61)
    C = bfx.gemm_bf16xN(mode, _cuda(A), _cuda(B))
    rows = np.sort(np.random.default_rng(62).choice(m, 48, replace=False))
    rows[-1] = m - 1
    Cs = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    C64, Cabs = orc.dgemm_rows(A, B, rows)
    check_bound(Cs, C64, Cabs, mode, k)


def test_x8_z3_bin_exact(bfx, orc):
    """The construction of the oracle's x8 pin, batched into one GEMM: rows
    [a, -a] times columns [b, b0 + b1] leave only a0 b2 and a1 b2.  x6 is the
    exact a0 b2 (bit-equal to the oracle); x8 adds a1 b2 (the Z3 bin).  The
    tensor core adds its accumulator at the alignment of the largest product
    of each MMA, even when those products cancel, so the later 2^-8-bin MMAs
    (a1 b0 - a1 b0 = 0 here) keep between none and all of the bits of the
    a1 b2 held in the correction accumulator, depending on the magnitudes
    (measured; R23).  Held: (x8 - x6) / (a1 b2) has median 1 (within 10 %)
    and lies within a quarter of 1 for most outputs; a kernel without the
    bin gives 0 everywhere."""
    rng = np.random.default_rng(19)
    a = rng.uniform(-1, 1, 64).astype(np.float32)
    b = (rng.uniform(-1, 1, 48) * 2.0 ** rng.integers(-5, 6, 48)).astype(np.float32)
    bp = orc.split(b, 3)
    c = (orc.bf16_to_f32(bp[0]).astype(np.float64) + orc.bf16_to_f32(bp[1])).astype(np.float32)
    cp = orc.split(c, 3)
    assert np.all((cp[0] == bp[0]) & (cp[1] == bp[1]) & (cp[2] == 0))  # c splits as (b0, b1, 0)
    A = np.stack([a, -a], axis=1)           # 64 x 2
    B = np.stack([b, c], axis=0)            # 2 x 48
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C6 = bfx.gemm_bf16xN(6, Ad, Bd).cpu().numpy()
    C8 = bfx.gemm_bf16xN(8, Ad, Bd).cpu().numpy()
    assert np.array_equal(C6, orc.gemm(6, A, B))
    a1 = orc.bf16_to_f32(orc.split(a, 3)[1]).astype(np.float64)
    b2 = orc.bf16_to_f32(bp[2]).astype(np.float64)
    z3 = np.outer(a1, b2)  # the exact a1 b2 of every output
    nz = z3 != 0
    ratio = (C8.astype(np.float64) - C6)[nz] / z3[nz]
    assert nz.sum() > 1000
    assert abs(np.median(ratio) - 1.0) <= 0.1
    assert np.mean(np.abs(ratio - 1.0) <= 0.25) >= 0.75
