"""GMRES-IR on the device (GMRES remark of Sec. III; Sec. IV-B) against the
oracle: the first GMRES correction equals the oracle's for the same FP32
factors (the device's FP32 LU is bit-identical to the oracle's blocked
mirror of its schedule) with the preconditioner applied through the
factors' explicit FP64 inverses on both sides (reading R27), and GMRES-IR
reaches FP64-LU accuracy where plain refinement cannot."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _fe(x, P):
    return np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))


@pytest.mark.parametrize("inverses", [True, False])
@pytest.mark.parametrize("n,nrhs,k", [(5, 1, 3), (96, 1, 8), (200, 3, 12), (333, 16, 5),
                                      (700, 2, 20)])
def test_first_gmres_step_matches_oracle(bfx, orc, n, nrhs, k, inverses):
    """Both forms of the preconditioner: explicit inverses (against the
    oracle's inverses, reading R27) and the row-sliced block substitution
    (against the oracle's substitution)."""
    _first_cycle(bfx, orc, n, nrhs, k, 1e5, inverses=inverses)


@pytest.mark.parametrize("n,nrhs,k,kappa", [(300, 1, 200, 1e4), (260, 3, 140, 1e4),
                                            (1300, 1, 1100, 1e6)])
def test_long_gmres_cycle_matches_oracle(bfx, orc, n, nrhs, k, kappa):
    """Long cycles: past 32 vectors the Gram-Schmidt update runs as chunk
    sums, past 1024 rotations the Givens scan gives each thread several rows.
    Single-product (x1) factors make GMRES converge slowly enough that the
    residual estimate does not underflow the (never met) tolerance before k
    steps, as it does within ~100 steps with FP32 factors."""
    _first_cycle(bfx, orc, n, nrhs, k, kappa, mode=1)


def _first_cycle(bfx, orc, n, nrhs, k, kappa, mode=0, inverses=True):
    """gmres = 2, one refinement step of exactly k Arnoldi steps (tolerance
    never met): x = x0 + d with d the k-th GMRES iterate, column by column.
    Equal up to rounding: the device orthogonalises by two classical
    Gram-Schmidt passes, the oracle by modified Gram-Schmidt, and sums in
    another order (the inverses too: blocked on the device, by columns in
    the oracle), so the tolerance is kappa(A) times FP64 rounding."""
    P = bi.svd_system(n, kappa, 900 + n, nrhs=nrhs)
    A = torch.from_numpy(P.A32).cuda()
    b = torch.from_numpy(P.b).cuda()
    x, res, code = bfx.solve_ir(mode, A, b, max_iter=1, gmres=2, gmres_m=k, gmres_tol=1e-300,
                                escalate=False, gmres_inverses=inverses)
    assert code in (0, 6)
    kk = min(k, n)
    assert res["gmres_steps"] == 1 and res["arnoldi"] == kk, res
    LU, ipiv, info = orc.lu_mirror(mode, P.A32, nb=64)
    xo, it, inner, conv, berr = orc.solve_gmres_ir(P.A32, LU, ipiv, P.b, max_iter=1, m=k,
                                                   tau=0.0, inverses=inverses)
    assert np.all(inner == kk)
    x = x.cpu().numpy()
    scale = np.max(np.abs(xo), axis=0)
    assert np.all(np.max(np.abs(x - xo), axis=0) <= 1e3 * kappa * 2.0**-53 * scale), (
        np.max(np.abs(x - xo), axis=0) / scale)


@pytest.mark.parametrize("kappa", [1e8, 1e10, 1e12])
def test_gmres_ir_within_10x_of_fp64_lu(bfx, orc, kappa):
    """x3 factors, escalation to x6, then GMRES-IR: converged (backward error
    at FP64 level) and forward error within 10x of the oracle's FP64 LU solve;
    at kappa 1e12 read as the median over the systems, at most 100x for any
    (the forward error of either backward-stable solver swings by orders of
    magnitude there)."""
    ratios = []
    for n, seed, nrhs in ((256, 1, 1), (515, 2, 4), (300, 3, 1)):
        P = bi.svd_system(n, kappa, seed, nrhs=nrhs)
        A = torch.from_numpy(P.A32).cuda()
        b = torch.from_numpy(P.b).cuda()
        x, res, code = bfx.solve_ir(3, A, b, nb=64)
        assert code == 0 and res["converged"] == 1, res
        assert res["berr"] <= np.sqrt(n) * 2.0**-53
        xd, _ = orc.dgesv(P.A32, P.b)
        fe, fe64 = _fe(x.cpu().numpy(), P), _fe(xd, P)
        ratios.append(fe / (fe64 + 1e-300))
    if kappa < 1e12:
        assert max(ratios) <= 10, ratios
    else:
        assert np.median(ratios) <= 10 and max(ratios) <= 100, ratios


def test_gmres_ir_without_escalation_on_x3_factors(bfx, orc):
    P = bi.svd_system(300, 1e9, 7, nrhs=2)
    A = torch.from_numpy(P.A32).cuda()
    b = torch.from_numpy(P.b).cuda()
    x, res, code = bfx.solve_ir(3, A, b, escalate=False, gmres=1)
    assert code == 0 and res["converged"] == 1 and res["refactorizations"] == 0
    assert res["gmres_steps"] >= 1 and res["mode_used"] == 3
    xd, _ = orc.dgesv(P.A32, P.b)
    assert _fe(x.cpu().numpy(), P) <= 10 * _fe(xd, P) + 1e-15


def test_plain_refinement_fails_where_gmres_converges(bfx):
    P = bi.svd_system(256, 1e10, 11)
    A = torch.from_numpy(P.A32).cuda()
    b = torch.from_numpy(P.b).cuda()
    _, res0, code0 = bfx.solve_ir(6, A, b, escalate=False, gmres=0)
    _, res1, code1 = bfx.solve_ir(6, A, b, escalate=False, gmres=1)
    assert code0 == 6 and res0["gmres_steps"] == 0
    assert code1 == 0 and res1["gmres_steps"] >= 1


def test_gmres_deterministic(bfx):
    P = bi.svd_system(400, 1e9, 5, nrhs=3)
    A = torch.from_numpy(P.A32).cuda()
    b = torch.from_numpy(P.b).cuda()
    x1, r1, _ = bfx.solve_ir(3, A, b, gmres=2)
    x2, r2, _ = bfx.solve_ir(3, A, b, gmres=2)
    assert torch.equal(x1, x2) and r1 == r2


def test_gmres_diag_dominant_table(bfx, orc):
    """Sec. IV-B GMRES table, FP32 rows (n = 10, 50, 100): every system
    converges, with about two refinement steps at the paper's tolerance read
    as cond_inf(A) 2^-53."""
    for n in (10, 50, 100):
        steps = []
        for s in range(10):
            P = bi.diag_dominant_system(n, 500 + s)
            tol = np.linalg.cond(P.A32.astype(np.float64), np.inf) * 2.0**-53
            A = torch.from_numpy(P.A32).cuda()
            b = torch.from_numpy(P.b).cuda()
            x, res, code = bfx.solve_ir(0, A, b, gmres=2, tol=tol, nb=8)
            assert code == 0 and res["converged"] == 1
            steps.append(res["gmres_steps"])
            xd, _ = orc.dgesv(P.A32, P.b)
            assert _fe(x.cpu().numpy(), P) <= 10 * _fe(xd, P) + 1e-15
        assert np.mean(steps) <= 3.0


def test_gmres_argument_checks(bfx):
    A = torch.eye(4, device="cuda")
    b = torch.ones((4, 1), dtype=torch.float64, device="cuda")
    for kw in ({"gmres": 3}, {"gmres_m": 4097}, {"gmres": -1}):
        with pytest.raises(bfx.BfxError) as e:
            bfx.solve_ir(3, A, b, **kw)
        assert e.value.code == 1
    b17 = torch.ones((4, 17), dtype=torch.float64, device="cuda")
    with pytest.raises(bfx.BfxError) as e:
        bfx.solve_ir(3, A, b17, gmres=1)
    assert e.value.code == 4
    x, res, code = bfx.solve_ir(3, A, b17, gmres=0)
    assert code == 0
