"""Pins of the oracle's GMRES and GMRES-IR (reading R18 of the GMRES remark
of Sec. III and the diagonally dominant table of Sec. IV-B).

GMRES is pinned by what defines it, not by its own arithmetic: the k-th
iterate minimises the preconditioned residual over the k-th Krylov space
(checked against numpy's least squares on an explicitly built Krylov basis),
it terminates with the exact solution after at most n steps, an exact
preconditioner solves in one step, and the Givens residual estimate equals the
true residual.  GMRES-IR is pinned by its purpose: forward error within 10x of
FP64 LU where plain refinement fails, and the table's 100 % convergence on
diagonally dominant matrices."""
import numpy as np
import pytest

import bfx_inputs as bi


def _precond(LU, ipiv):
    """M^-1 v = U^-1 L^-1 P v from the FP32 factors, via numpy (FP64)."""
    n = LU.shape[0]
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    perm = np.arange(n)
    for j, p in enumerate(ipiv):
        perm[[j, p]] = perm[[p, j]]
    return lambda v: np.linalg.solve(U, np.linalg.solve(L, v[perm]))


def _inexact_factors(orc, A, seed, eps=0.2):
    """FP32 LU of a perturbed A: a preconditioner far enough from A that
    GMRES needs several steps."""
    E = np.random.default_rng(seed).uniform(-eps, eps, A.shape).astype(np.float32)
    LU, ipiv, info = orc.lu(0, (A + E).astype(np.float32))
    assert info == 0
    return LU, ipiv


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_gmres_iterate_minimises_residual_over_krylov_space(orc, k):
    n = 30
    A = bi.uniform_pm1((n, n), 11) + np.float32(4.0) * np.eye(n, dtype=np.float32)
    LU, ipiv = _inexact_factors(orc, A, 12)
    rhs = np.random.default_rng(13).standard_normal(n)
    Minv = _precond(LU, ipiv)
    At = np.column_stack([Minv(A.astype(np.float64)[:, j]) for j in range(n)])
    rt = Minv(rhs)
    K = np.empty((n, k))
    K[:, 0] = rt
    for j in range(1, k):
        K[:, j] = At @ K[:, j - 1]
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(At @ Q, rt, rcond=None)
    best = np.linalg.norm(rt - At @ (Q @ y))
    d, kk, hist = orc.gmres(A, LU, ipiv, rhs, m=k, tau=0.0)
    assert kk == k
    true = np.linalg.norm(rt - At @ d)
    assert abs(true - best) <= 1e-10 * np.linalg.norm(rt)
    assert abs(hist[-1] - true) <= 1e-10 * np.linalg.norm(rt)  # Givens estimate = residual
    assert np.all(np.diff(hist) <= 1e-14 * np.linalg.norm(rt))  # never increases
    # the iterate itself is the minimiser (the least-squares problem is well posed)
    assert np.linalg.norm(d - Q @ y) <= 1e-8 * np.linalg.norm(Q @ y)


def test_gmres_finite_termination(orc):
    """In at most n steps GMRES returns the exact solution of A d = rhs."""
    n = 12
    A = bi.uniform_pm1((n, n), 21) + np.float32(3.0) * np.eye(n, dtype=np.float32)
    LU, ipiv = _inexact_factors(orc, A, 22, eps=0.5)
    rhs = np.random.default_rng(23).standard_normal(n)
    d, k, hist = orc.gmres(A, LU, ipiv, rhs, m=n, tau=0.0)
    ref = np.linalg.solve(A.astype(np.float64), rhs)
    assert k <= n
    assert np.linalg.norm(d - ref) <= 1e-9 * np.linalg.norm(ref)


def test_gmres_exact_preconditioner_one_step(orc):
    """A = P^T L U exactly in FP32 (integer L, U; powers of two on the
    diagonals): M^-1 A = I, so one Arnoldi step solves the system."""
    rng = np.random.default_rng(31)
    n = 16
    L = np.tril(rng.integers(-3, 4, (n, n)).astype(np.float64) / 4.0, -1) + np.eye(n)
    U = np.triu(rng.integers(-4, 5, (n, n)).astype(np.float64), 1) + np.diag(
        2.0 ** rng.integers(3, 6, n))
    A = (L @ U).astype(np.float32)
    assert np.array_equal(A.astype(np.float64), L @ U)  # exactly representable
    LU, ipiv, info = orc.lu(0, A)
    assert info == 0
    rhs = rng.standard_normal(n)
    d, k, hist = orc.gmres(A, LU, ipiv, rhs, m=10, tau=1e-12)
    assert k == 1
    ref = np.linalg.solve(A.astype(np.float64), rhs)
    assert np.linalg.norm(d - ref) <= 1e-12 * np.linalg.norm(ref)


def _fe(x, P):
    return np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))


@pytest.mark.parametrize("kappa", [1e8, 1e10, 1e12])
def test_gmres_ir_within_10x_of_fp64_lu_where_ir_fails(orc, kappa):
    """The purpose of GMRES-IR: with the FP32 factors of an ill-conditioned
    A32 plain refinement does not reach FP64 accuracy, GMRES-IR does (forward
    error within 10x of FP64 LU on the same system)."""
    fails, ratios = 0, []
    for s in range(4):
        P = bi.svd_system(96, kappa, 40 + s)
        LU, ipiv, info = orc.lu(6, P.A32)
        assert info == 0
        xd, _ = orc.dgesv(P.A32, P.b)
        fe64 = _fe(xd, P)
        x, it, inner, conv, berr = orc.solve_gmres_ir(P.A32, LU, ipiv, P.b)
        assert conv[0] == 1, (kappa, s, it, inner, berr)
        assert berr[0] <= np.sqrt(96) * 2.0**-53
        ratios.append(_fe(x, P) / (fe64 + 1e-300))
        xi, _, ci, _ = orc.solve_ir(P.A32, LU, ipiv, P.b)
        fails += (ci[0] == 0) or (_fe(xi, P) > 10 * fe64 + 1e-15)
    # Both solvers are backward stable; at kappa 1e12 the forward error (of
    # order kappa * berr) swings by orders of magnitude with how x_true falls
    # on the smallest singular directions, so "within 10x" is read there as
    # the median over the systems (and at most 100x for any one).
    if kappa < 1e12:
        assert max(ratios) <= 10, ratios
    else:
        assert np.median(ratios) <= 10 and max(ratios) <= 100, ratios
    if kappa >= 1e10:
        assert fails >= 1  # plain refinement does fail on these


@pytest.mark.parametrize("n", [10, 50, 100])
def test_e6_diag_dominant_fp32_lu_gmres(orc, n):
    """Sec. IV-B GMRES table, FP32 rows: every test converges in about two
    refinement steps on average (the paper prints 2.0 for n = 10, 50, 100),
    with the paper's tolerance read as cond_inf(A) * 2^-53 on the correction.
    With a single bfloat16 product in the trailing update (mode x1) every test
    still converges but needs more Arnoldi steps (the paper's BF16 rows print
    6.6 - 7 iterations; measured here 5 - 9 Arnoldi steps)."""
    its, inn32, inn1 = [], [], []
    for s in range(25):
        P = bi.diag_dominant_system(n, 500 + s)
        tol = np.linalg.cond(P.A32.astype(np.float64), np.inf) * 2.0**-53
        LU, ipiv, _ = orc.lu(0, P.A32)
        x, it, inner, conv, berr = orc.solve_gmres_ir(P.A32, LU, ipiv, P.b, tol=tol)
        assert conv[0] == 1
        its.append(it[0])
        inn32.append(inner[0])
        LU1, ipiv1, _ = orc.lu(1, P.A32)
        x1, it1, inner1, conv1, _ = orc.solve_gmres_ir(P.A32, LU1, ipiv1, P.b, tol=tol)
        assert conv1[0] == 1
        inn1.append(inner1[0])
        xd, _ = orc.dgesv(P.A32, P.b)
        assert _fe(x, P) <= 10 * _fe(xd, P) + 1e-15
    assert 1.0 <= np.mean(its) <= 3.0
    if n > 10:
        assert np.mean(inn1) > np.mean(inn32)


def test_kappa_1e12_forward_error_distribution(orc):
    """Why "within 10x of FP64 dgesv" is read over a distribution at kappa 1e12
    (reading R22).  Over 24 systems (n = 96, config 3's generator), two FP64
    backward-stable LU solvers, LAPACK's dgesv (scipy) and the oracle's own
    FP64 LU, already differ in forward error by more than 10x on some systems:
    the forward error, of order kappa times the backward error, swings with how
    x_true falls on the smallest singular directions.  The oracle's GMRES-IR
    (x6 factors) is held to the same distributional rule as the device: the
    median ratio to the FP64 LU at most 10, at least 80 % of systems within
    10x, none beyond 100x."""
    import scipy.linalg as sla

    r_gm, r_lapack = [], []
    for s in range(24):
        P = bi.svd_system(96, 1e12, 40 + s)
        LU, ipiv, info = orc.lu(6, P.A32)
        assert info == 0
        xd, _ = orc.dgesv(P.A32, P.b)
        fe64 = _fe(xd, P)
        x, it, inner, conv, berr = orc.solve_gmres_ir(P.A32, LU, ipiv, P.b)
        assert conv[0] == 1
        xl = sla.solve(P.A32.astype(np.float64), P.b)
        r_gm.append(_fe(x, P) / fe64)
        r_lapack.append(_fe(xl, P) / fe64)
    r_gm, r_lapack = np.array(r_gm), np.array(r_lapack)
    assert r_lapack.max() > 10 or r_lapack.min() < 0.1  # FP64 against FP64 swings
    assert np.median(r_gm) <= 10
    assert np.mean(r_gm <= 10) >= 0.8
    assert r_gm.max() <= 100
