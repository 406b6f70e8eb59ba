"""Pins of the oracle's single-type LU and refinement (Sec. IV-B plain IR
table, reading R26) and of its binary16 rounding.

The LU is checked against independent brute-force restatements: numpy's
float16 scalar arithmetic (which computes each operation in FP32 and rounds
the result to binary16, the reading's definition) and an FP32 loop with the
separately pinned bfloat16 rounding.  The refinement is checked against the
qualitative order of the paper's table.
"""
import numpy as np
import pytest

import bfx_inputs as bi


# ----------------------------------------------------------------- binary16 rounding
def _check_f16(orc, bits):
    x = bits.view(np.float32)
    got = orc.f16_rne(x)
    ref = x.astype(np.float16).view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(got[~nan], ref[~nan])
    g = got[nan]
    assert np.all((g & 0x7C00) == 0x7C00) and np.all((g & 0x3FF) != 0)  # NaN stays NaN
    assert np.array_equal(g >> 15, (bits[nan] >> 31).astype(np.uint16))  # sign kept


def test_f16_rne_matches_ieee_conversion(orc):
    """Every FP32 exponent from 2^-27 to 2^18 (all of binary16's subnormal,
    normal and overflow boundaries) at a stride of 7 patterns, plus a random
    sample of all 2^32 patterns, against numpy's IEEE float32 -> float16."""
    with np.errstate(over="ignore", invalid="ignore"):
        for sign in (0, 1):
            lo = (sign << 31) | (100 << 23)
            hi = (sign << 31) | (146 << 23)
            _check_f16(orc, np.arange(lo, hi, 7, dtype=np.uint64).astype(np.uint32))
        rng = np.random.default_rng(0)
        _check_f16(orc, rng.integers(0, 2**32, 4_000_000, dtype=np.uint64).astype(np.uint32))
        edges = np.array([0x477FE000, 0x477FEFFF, 0x477FF000, 0x33000000, 0x33000001, 0x387FC000,
                          0x387FE000, 0x00000001, 0x7F800000, 0x7FC00000, 0xFF800001], np.uint32)
        _check_f16(orc, edges)


# ----------------------------------------------------------------- single-type LU
def _lu_loop(A, rnd):
    """Textbook right-looking LU with partial pivoting (first max), each
    operation's result passed through rnd."""
    M = [[rnd(v) for v in row] for row in A.astype(np.float32)]
    n = len(M)
    ipiv, info = [], 0
    for k in range(n):
        p, amax = k, abs(M[k][k])
        for i in range(k + 1, n):
            if abs(M[i][k]) > amax:
                p, amax = i, abs(M[i][k])
        ipiv.append(p)
        if amax == 0:
            info = info or k + 1
            continue
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            l = rnd(M[i][k] / M[k][k])
            M[i][k] = l
            for j in range(k + 1, n):
                M[i][j] = rnd(M[i][j] - rnd(l * M[k][j]))
    return np.array(M, np.float32), np.array(ipiv, np.int32), info


def _cases():
    yield bi.uniform_pm1((12, 12), 1)
    yield bi.svd_system(16, 1e3, 2).A32
    yield bi.wide_range((10, 10), 3, -6, 6)
    A = bi.uniform_pm1((9, 9), 4)
    A[:, 3] = 0.0  # an exactly zero pivot column: info = 4, column skipped
    yield A


def test_lu_lowp_fp16_equals_numpy_half_arithmetic(orc):
    for A in _cases():
        ref, ipiv, info = _lu_loop(A.astype(np.float16), lambda v: np.float16(v))
        LU, ip, inf = orc.lu_lowp(orc.LOWP_FP16, A)
        assert np.array_equal(LU, ref) and np.array_equal(ip, ipiv) and inf == info
        assert np.array_equal(LU.astype(np.float16).astype(np.float32), LU)  # binary16 values


def test_lu_lowp_bf16_equals_fp32_loop_with_bf16_rounding(orc):
    def rnd(v):
        return orc.bf16_to_f32(orc.bf16_rne(np.float32(v))).reshape(-1)[0]
    for A in _cases():
        ref, ipiv, info = _lu_loop(A, lambda v: np.float32(rnd(v)))
        LU, ip, inf = orc.lu_lowp(orc.LOWP_BF16, A)
        assert np.array_equal(LU, ref) and np.array_equal(ip, ipiv) and inf == info


def test_lu_lowp_fp32_equals_fp32_loop_and_backward_stable(orc):
    for A in _cases():
        ref, ipiv, info = _lu_loop(A, np.float32)
        LU, ip, inf = orc.lu_lowp(orc.LOWP_FP32, A)
        assert np.array_equal(LU, ref) and np.array_equal(ip, ipiv) and inf == info
    A = bi.svd_system(40, 1e2, 5).A32
    LU, ip, _ = orc.lu_lowp(orc.LOWP_FP32, A)
    n = A.shape[0]
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    PA = A.astype(np.float64).copy()
    for k, p in enumerate(ip):
        PA[[k, p]] = PA[[p, k]]
    assert np.linalg.norm(PA - L @ U, np.inf) <= 4 * n * 2.0**-24 * np.linalg.norm(A, np.inf) * 8


# ----------------------------------------------------------------- refinement
def test_ir_counts_an_overflowing_correction_as_divergence(orc):
    """Factors of a different matrix make the corrections grow by 1e30 a step
    until they overflow: that is divergence, never convergence."""
    n = 4
    A = np.eye(n, dtype=np.float32)
    LU = np.diag(np.full(n, 1e-30, np.float32))
    b = np.ones(n)
    x, iters, conv, _ = orc.solve_ir(A, LU, np.arange(n, dtype=np.int32), b, max_iter=50,
                                     tol=1e-12, tol_b=0.0, stall=float("inf"))
    assert conv[0] == 0 and iters[0] < 50


@pytest.mark.parametrize("kappa", [10.0, 1e3])
def test_single_type_ir_follows_the_tables_order(orc, kappa):
    """Sec. IV-B plain IR table (n = 50): FP32 factors converge every time in
    about three corrections; a single binary16 factorisation needs more, a
    single bfloat16 one more still and fails more often as cond grows."""
    stats = {}
    for typ in (orc.LOWP_FP32, orc.LOWP_FP16, orc.LOWP_BF16):
        conv, its = [], []
        for s in range(16):
            P = bi.svd_system(50, kappa, 500 + s)
            _, it, c, info, _, _ = orc.lowp_lu_solve_ir(typ, P.A32, P.b, tol=kappa * 2.0**-53)
            assert info == 0
            conv.append(c)
            if c:
                its.append(it)
        stats[typ] = (np.mean(conv), np.mean(its) if its else np.inf)
    f32, f16, b16 = stats[orc.LOWP_FP32], stats[orc.LOWP_FP16], stats[orc.LOWP_BF16]
    assert f32[0] == 1.0 and f32[1] <= 4.0, stats
    assert f16[0] >= b16[0] and f16[1] > f32[1], stats
    assert b16[1] > f16[1] or b16[0] < f16[0], stats
    if kappa >= 1e3:
        assert b16[0] < 1.0, stats


def test_ir_counts_a_nan_correction_as_divergence(orc):
    """A NaN in the correction (factors with a NaN entry) must stop the
    refinement unconverged: a max over |d| that skips NaN would read 0."""
    n = 4
    A = np.eye(n, dtype=np.float32)
    LU = np.eye(n, dtype=np.float32)
    LU[2, 1] = np.nan
    x, iters, conv, _ = orc.solve_ir(A, LU, np.arange(n, dtype=np.int32), np.ones(n), max_iter=50,
                                     tol=1e-12, tol_b=0.0, stall=float("inf"))
    assert conv[0] == 0 and iters[0] == 1
