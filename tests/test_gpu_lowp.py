"""The single-type LU with FP64 refinement (the plain IR table of Sec. IV-B)
on the device against the oracle, bit for bit: factors, pivots, info, the
refined solution, the number of corrections and the convergence flag.

Every operation of the factorisation is defined elementwise (an FP32
operation rounded to the type) and every sum of the refinement runs in one
fixed order on both sides, so the results must be identical, not merely
close.
"""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _systems(count, n, kappa, seed):
    probs = [bi.svd_system(n, kappa, seed + s) for s in range(count)]
    A = np.stack([p.A32 for p in probs])
    b = np.stack([p.b[:, 0] for p in probs])
    return probs, A, b


def _run(bfx, typ, A, b, tol, max_iter=50):
    out = bfx.lowp_lu_ir_batched(typ, torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(),
                                 torch.from_numpy(tol).cuda(), max_iter=max_iter, factors=True)
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("typ", [0, 1, 2])
@pytest.mark.parametrize("n,kappa", [(50, 10.0), (50, 1e3), (37, 1e4), (128, 1e2), (1, 1.0), (33, 10.0)])
def test_lowp_bit_exact_vs_oracle(bfx, orc, typ, n, kappa):
    count = 12
    probs, A, b = _systems(count, n, kappa, 700 + n)
    tol = np.full(count, kappa * 2.0**-53)
    x, iters, conv, info, LU, ipiv = _run(bfx, typ, A, b, tol)
    for s in range(count):
        xo, it, c, inf, LUo, ipo = orc.lowp_lu_solve_ir(typ, A[s], b[s], tol=tol[s])
        assert np.array_equal(LU[s], LUo, equal_nan=True), s
        assert np.array_equal(ipiv[s], ipo) and info[s] == inf, s
        assert iters[s] == it and conv[s] == c, (s, iters[s], it, conv[s], c)
        assert np.array_equal(x[s], xo[:, 0], equal_nan=True), s


def test_lowp_zero_pivot_column_and_divergence(bfx, orc):
    """An exactly zero column: info names it, the refinement diverges (NaN or
    Inf) and reports no convergence, as the oracle does."""
    n, count = 24, 3
    _, A, b = _systems(count, n, 10.0, 800)
    A[1, :, 5] = 0.0
    tol = np.full(count, 10.0 * 2.0**-53)
    for typ in (0, 1, 2):
        x, iters, conv, info, LU, ipiv = _run(bfx, typ, A, b, tol)
        assert info[1] == 6 and conv[1] == 0
        for s in range(count):
            xo, it, c, inf, LUo, ipo = orc.lowp_lu_solve_ir(typ, A[s], b[s], tol=tol[s])
            assert info[s] == inf and iters[s] == it and conv[s] == c
            assert np.array_equal(LU[s], LUo, equal_nan=True)


def test_lowp_binary16_overflow_and_max_iter(bfx, orc):
    """Entries beyond binary16's range become infinite in the FP16 factors;
    max_iter = 0 returns the first solve."""
    n, count = 16, 2
    _, A, b = _systems(count, n, 10.0, 810)
    A[0] *= 1e5
    b[0] *= 1e5
    tol = np.full(count, 10.0 * 2.0**-53)
    x, iters, conv, info, LU, ipiv = _run(bfx, 2, A, b, tol)
    for s in range(count):
        xo, it, c, inf, LUo, ipo = orc.lowp_lu_solve_ir(2, A[s], b[s], tol=tol[s])
        assert np.array_equal(LU[s], LUo, equal_nan=True)
        assert iters[s] == it and conv[s] == c and info[s] == inf
    x, iters, conv, info, LU, ipiv = _run(bfx, 0, A, b, tol, max_iter=0)
    assert (iters == 0).all() and (conv == 0).all()
    xo, *_ = orc.lowp_lu_solve_ir(0, A[1], b[1], tol=tol[1], max_iter=0)
    assert np.array_equal(x[1], xo[:, 0])


def test_lowp_argument_errors(bfx):
    A = torch.zeros((1, 129, 129), device="cuda")
    b = torch.zeros((1, 129), dtype=torch.float64, device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(bfx.BfxError):
        bfx.lowp_lu_ir_batched(0, A, b, t)
    with pytest.raises(bfx.BfxError):
        bfx.lowp_lu_ir_batched(3, A[:, :8, :8].contiguous(), b[:, :8].contiguous(), t)
