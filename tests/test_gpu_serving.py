"""Serving runtime: continuous admission under a memory budget; every result
is bit-for-bit the one the same request gets when solved alone."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _alone(bfx, P, mode):
    x, res, code = bfx.solve_ir(mode, torch.from_numpy(P.A32).cuda(), torch.from_numpy(P.b).cuda(),
                                escalate=True, nb=64)
    return x.cpu().numpy(), res, code


def test_mixed_requests_same_as_alone(bfx):
    rng = np.random.default_rng(5)
    ns = [16, 300, 64, 1500, 77, 513, 128, 1024, 33, 700, 256, 90]
    reqs = [bi.svd_system(n, 10 ** rng.uniform(1, 5), 100 + i, nrhs=int(rng.integers(1, 5)))
            for i, n in enumerate(ns)]
    srv = bfx.Server(budget_bytes=2 << 30, max_inflight=6, mode=3)
    tickets = [srv.submit(P.A32, P.b) for P in reqs]
    out = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["peak_running"] >= 2  # requests did overlap
    for P, (x, res) in zip(reqs, out):
        assert res["status"] == 0 and res["converged"] == 1, res
        xa, ra, code = _alone(bfx, P, 3)
        assert code == 0
        assert np.array_equal(x, xa)  # identical alone and in the mix
        assert res["iters"] == ra["iters"]


def test_budget_limits_admission(bfx):
    n = 1024
    reqs = [bi.svd_system(n, 100.0, 200 + i) for i in range(5)]
    r256 = lambda v: (v + 255) // 256 * 256
    p = bfx.IrParams(50, 2.0**-53, -1.0, 0.5, 1, 64, 1, 0, 1e-10)
    per = r256(4 * n * n) + 2 * r256(8 * n) + bfx.solve_ir_workspace_size(3, n, 1, p) + 256
    srv = bfx.Server(budget_bytes=int(2.5 * per), max_inflight=8, mode=3)
    tickets = [srv.submit(P.A32, P.b) for P in reqs]
    res = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r[1]["converged"] == 1 for r in res)
    assert st["peak_used_bytes"] <= st["pool_bytes"]
    assert st["peak_running"] <= 2  # only two fit the budget at once
    assert max(r[1]["queue_s"] for r in res) > 0.0


def test_oversized_request_rejected(bfx):
    srv = bfx.Server(budget_bytes=8 << 20, max_inflight=2, mode=3)
    with pytest.raises(bfx.BfxError) as e:
        srv.submit(np.eye(2048, dtype=np.float32), np.ones(2048))
    assert e.value.code == 2
    srv.close()


def test_many_concurrent_requests_same_as_alone(bfx):
    """32 workers on a Poisson stream of 40 mixed-size requests (most n not a
    multiple of the 64-row solve block): each result equals solving alone.
    Kernels of other requests share the SMs, so any read of shared memory a
    kernel did not write shows up here as a changed or non-finite result."""
    reqs = bi.serving_stream(40, 3)
    systems = [bi.fast_system(r.n, 10.0 ** min(r.log10_kappa, 3), r.seed, nrhs=r.nrhs)
               for r in reqs]
    assert sum(P.n % 64 != 0 for P in systems) >= 30
    srv = bfx.Server(budget_bytes=60 * 10**9, max_inflight=32, mode=3, escalate=False)
    tickets = [srv.submit(P.A32, P.b) for P in systems]
    out = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["peak_running"] >= 8
    for P, (x, res) in zip(systems, out):
        assert np.isfinite(x).all()
        xa, ra, code = bfx.solve_ir(3, torch.from_numpy(P.A32).cuda(), torch.from_numpy(P.b).cuda(),
                                    escalate=False)
        assert np.array_equal(x, xa.cpu().numpy())
        assert res["iters"] == ra["iters"] and res["converged"] == ra["converged"]


def test_mixed_requests_same_as_alone_x6_gmres(bfx, orc):
    """bench.py's serving configuration: bf16x6 factors, escalation, GMRES-IR
    for what plain refinement cannot finish, the Krylov length capped at
    min(n, 1024), the preconditioner by row-sliced block substitution (the
    server's form).  Requests of kappa up to 1e10 go through GMRES-IR; each
    result equals the same request solved alone (same kernels, same order),
    bit for bit, with the same refinement and Arnoldi counts, and lies within
    10x of the oracle's FP64 LU in forward error."""
    rng = np.random.default_rng(11)
    ns = [300, 96, 700, 160, 515, 64, 257, 420]
    lks = [9.5, 2.0, 10.0, 6.0, 9.0, 1.0, 8.0, 4.0]
    reqs = [bi.svd_system(n, 10.0 ** lk, 400 + i, nrhs=int(rng.integers(1, 4)))
            for i, (n, lk) in enumerate(zip(ns, lks))]
    srv = bfx.Server(budget_bytes=4 << 30, max_inflight=8, mode=6, escalate=True, gmres=1)
    tickets = [srv.submit(P.A32, P.b) for P in reqs]
    out = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["peak_running"] >= 2
    assert sum(res["gmres_steps"] > 0 for _, res in out) >= 2  # GMRES-IR ran in the mix
    for P, (x, res) in zip(reqs, out):
        assert res["status"] == 0 and res["converged"] == 1, res
        xa, ra, code = bfx.solve_ir(6, torch.from_numpy(P.A32).cuda(), torch.from_numpy(P.b).cuda(),
                                    escalate=True, nb=64, gmres=1, gmres_m=min(P.n, 1024),
                                    gmres_inverses=False)
        assert code == 0
        assert np.array_equal(x, xa.cpu().numpy())
        for k in ("iters", "gmres_steps", "arnoldi", "refactorizations", "mode_used"):
            assert res[k] == ra[k], k
        xd, _ = orc.dgesv(P.A32, P.b)
        fe = np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))
        fe64 = np.max(np.abs(xd - P.x_true)) / np.max(np.abs(P.x_true))
        assert fe <= 10 * fe64 + 1e-15, (P.n, fe, fe64)


def test_continuous_batching_small_requests(bfx, orc):
    """Continuous batching: small requests (n <= 512) waiting together are
    solved as one batch (grouped tensor-core updates over all of them), large
    ones one per worker.  Each small request's result does not depend on the
    batch it shared: it equals the same request alone through a server (a
    batch of one), bit for bit; large requests equal bfx_solve_ir alone.
    Every result lies within 10x of the oracle's FP64 LU in forward error."""
    rng = np.random.default_rng(21)
    ns = [64, 300, 96, 700, 512, 128, 33, 1100, 257, 200, 480, 150, 75, 1024, 400, 90]
    reqs = [bi.svd_system(n, 10.0 ** rng.uniform(1, 7), 600 + i, nrhs=int(rng.integers(1, 3)))
            for i, n in enumerate(ns)]
    kw = dict(budget_bytes=4 << 30, mode=6, escalate=True, gmres=1, batch_max_n=512)
    srv = bfx.Server(max_inflight=4, **kw)
    tickets = [srv.submit(P.A32, P.b) for P in reqs]
    out = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["batches"] >= 1
    small = [i for i, P in enumerate(reqs) if P.n <= 512]
    alone_srv = bfx.Server(max_inflight=1, **kw)
    for i, (P, (x, res)) in enumerate(zip(reqs, out)):
        assert res["status"] == 0 and res["converged"] == 1, (P.n, res)
        if i in small:
            xa, ra = alone_srv.wait(alone_srv.submit(P.A32, P.b))
            assert np.array_equal(x, xa), P.n
            assert res["iters"] == ra["iters"] and res["gmres_steps"] == ra["gmres_steps"]
        else:
            xa, ra, code = bfx.solve_ir(6, torch.from_numpy(P.A32).cuda(),
                                        torch.from_numpy(P.b).cuda(), escalate=True, nb=64,
                                        gmres=1, gmres_m=min(P.n, 1024))
            assert np.array_equal(x, xa.cpu().numpy())
        xd, _ = orc.dgesv(P.A32, P.b)
        fe = np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))
        fe64 = np.max(np.abs(xd - P.x_true)) / np.max(np.abs(P.x_true))
        assert fe <= 10 * fe64 + 1e-15, (P.n, fe, fe64)
    alone_srv.close()
