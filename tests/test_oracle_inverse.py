"""Pins of reading R27: the GMRES preconditioner M^-1 = U^-1 L^-1 P applied
through explicit FP64 inverses of the FP32 factors (the preconditioner of
the GMRES remark of Sec. III and of Sec. IV-B, evaluated as two
matrix-vector products).

The inverses are pinned by closed forms whose every entry is a power of two
(exact in FP64), by the defining identity X T = I within the triangular
inverse's error bound, and GMRES through them by its agreement with GMRES
through substitution (the same operator up to FP64 rounding)."""
import numpy as np
import pytest

import bfx_inputs as bi


def _bidiagonal_factors(n):
    """Packed factors with L = I - N (ones below the diagonal in L^-1) and
    U = 2 I - N^T (U^-1_{i,i+k} = 2^-(k+1))."""
    LU = np.zeros((n, n), dtype=np.float32)
    for i in range(n):
        LU[i, i] = 2.0
        if i > 0:
            LU[i, i - 1] = -1.0
        if i + 1 < n:
            LU[i, i + 1] = -1.0
    return LU


@pytest.mark.parametrize("n", [1, 2, 7, 64, 130])
def test_inverse_closed_forms(orc, n):
    LU = _bidiagonal_factors(n)
    XL = orc.tri_inverse(LU, True)
    XU = orc.tri_inverse(LU, False)
    i, j = np.indices((n, n))
    assert np.array_equal(XL, np.where(j <= i, 1.0, 0.0))
    expect_u = np.where(j >= i, 2.0 ** (-(j - i + 1).astype(np.float64)), 0.0)
    assert np.array_equal(XU, expect_u)


@pytest.mark.parametrize("n", [50, 200])
def test_inverse_identity_within_bound(orc, n):
    """X T = I up to the triangular inverse's error, |X T - I| <= c n u |X||T|,
    for the factors of a random matrix (the LU of record)."""
    A = bi.uniform_pm1((n, n), 70 + n)
    LU, ipiv, info = orc.lu(0, A)
    assert info == 0
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    u = 2.0 ** -53
    for X, T, lower in ((orc.tri_inverse(LU, True), L, True), (orc.tri_inverse(LU, False), U, False)):
        assert np.array_equal(X, np.tril(X) if lower else np.triu(X))
        E = np.abs(X @ T - np.eye(n))
        assert np.all(E <= 4 * n * u * (np.abs(X) @ np.abs(T)) + 1e-300)


def test_inverse_matches_numpy_solve(orc):
    """Column c of X solves T x = e_c: against LAPACK's triangular solve."""
    import scipy.linalg as sla
    n = 120
    LU, _, _ = orc.lu(0, bi.uniform_pm1((n, n), 5))
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    XL = orc.tri_inverse(LU, True)
    XU = orc.tri_inverse(LU, False)
    rl = sla.solve_triangular(L, np.eye(n), lower=True, unit_diagonal=True)
    ru = sla.solve_triangular(U, np.eye(n), lower=False)
    assert np.max(np.abs(XL - rl)) <= 1e-12 * np.max(np.abs(rl))
    assert np.max(np.abs(XU - ru)) <= 1e-12 * np.max(np.abs(ru))


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_gmres_through_inverses_equals_substitution(orc, kappa):
    """The same operator: k GMRES steps through the inverses and through
    substitution agree to kappa times FP64 rounding."""
    n, k = 160, 25
    P = bi.svd_system(n, kappa, 31)
    LU, ipiv, _ = orc.lu(1, P.A32)  # x1 factors: GMRES needs many steps
    rhs = np.random.default_rng(3).standard_normal(n)
    d0, k0, h0 = orc.gmres(P.A32, LU, ipiv, rhs, m=k, tau=0.0)
    d1, k1, h1 = orc.gmres(P.A32, LU, ipiv, rhs, m=k, tau=0.0, inverses=True)
    assert k0 == k1 == k
    assert np.max(np.abs(d1 - d0)) <= 1e3 * kappa * 2.0 ** -53 * np.max(np.abs(d0))
    assert np.max(np.abs(h1 - h0)) <= 1e3 * kappa * 2.0 ** -53 * h0[0]


def test_gmres_ir_through_inverses_reaches_fp64_accuracy(orc):
    """GMRES-IR with the preconditioner through the inverses: converged, and
    the forward error within 10x that of FP64 LU at kappa 1e8 (Sec. IV-B)."""
    n = 120
    P = bi.svd_system(n, 1e8, 7)
    LU, ipiv, _ = orc.lu(6, P.A32)
    x, it, inner, conv, berr = orc.solve_gmres_ir(P.A32, LU, ipiv, P.b, m=n, inverses=True)
    assert conv[0] == 1
    xd, _ = orc.dgesv(P.A32, P.b)
    fe = np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))
    fe64 = np.max(np.abs(xd - P.x_true)) / np.max(np.abs(P.x_true))
    assert fe <= 10 * fe64
