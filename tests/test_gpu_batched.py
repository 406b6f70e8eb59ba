"""Batched solves of uneven-size systems (one graph launch) against the oracle
and against the same systems solved one at a time."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _make(ns, kappas, seed):
    return [bi.svd_system(int(n), float(k), seed + i) for i, (n, k) in enumerate(zip(ns, kappas))]


@pytest.mark.parametrize("mode", [3, 6])
def test_batched_matches_oracle_and_single(bfx, orc, mode):
    ns = [1, 7, 64, 65, 100, 128, 129, 200, 257, 33, 300, 64]
    kap = [1e1, 1e2, 1e3, 1e1, 1e2, 1e3, 1e2, 1e1, 1e3, 1e2, 1e2, 1e3]
    probs = _make(ns, kap, 100)
    B = bfx.Batch(mode, ns)
    A, b = B.pack([p.A32 for p in probs], [p.b for p in probs])
    x, status = B.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = B.decode_status(status)
    assert (info == 0).all() and conv.all(), (conv, iters, info, berr)
    xs = B.unpack(x)
    for p, xb in zip(probs, xs):
        xd, _ = orc.dgesv(p.A32, p.b)
        fe = np.max(np.abs(xb - p.x_true)) / np.max(np.abs(p.x_true))
        fe64 = np.max(np.abs(xd - p.x_true)) / np.max(np.abs(p.x_true))
        assert fe <= 10 * fe64 + 1e-15, (p.n, fe, fe64)
        # the same system alone through the single-system entry point
        xs1, res, code = bfx.solve_ir(mode, torch.from_numpy(p.A32).cuda(),
                                      torch.from_numpy(p.b).cuda(), escalate=False)
        assert code == 0
        scale = np.max(np.abs(xs1.cpu().numpy()))
        assert np.max(np.abs(xb - xs1.cpu().numpy())) <= 100 * p.kappa_nominal * 2.0 ** -53 * scale * p.n


def test_batched_singular_system_isolated(bfx):
    ns = [50, 40, 60]
    probs = _make(ns, [10, 10, 10], 7)
    mats = [p.A32.copy() for p in probs]
    mats[1][:, 5] = 0.0
    B = bfx.Batch(6, ns)
    A, b = B.pack(mats, [p.b for p in probs])
    x, status = B.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = B.decode_status(status)
    assert info[1] == 6 and conv[1] == 0
    assert conv[0] == 1 and conv[2] == 1 and info[0] == 0 and info[2] == 0


def test_batched_graph_replay_and_rebind(bfx):
    ns = [90, 33, 150]
    probs = _make(ns, [10, 100, 10], 9)
    B = bfx.Batch(6, ns)
    A, b = B.pack([p.A32 for p in probs], [p.b for p in probs])
    x1, st1 = B.solve(A, b)
    x2, st2 = B.solve(A, b, x=torch.empty_like(x1), status=torch.empty_like(st1))  # new buffers
    x3 = torch.empty_like(x1)
    B.solve(A, b, x=x3, status=st2)
    B.solve(A, b, x=x3, status=st2)  # replay of the same graph
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(x1, x3)


@pytest.mark.parametrize("nb,bn", [(32, 64), (32, 256), (64, 128), (128, 64), (128, 256)])
def test_batched_every_tile_shape(bfx, orc, nb, bn):
    """Each shape the autotuner may pick solves the batch to FP64-LU accuracy;
    nb = 32 / 128 also exercise the narrow and wide block columns."""
    ns = [1, 31, 64, 96, 130, 200, 257, 400, 17]
    kap = [1e1, 1e2, 1e3, 1e2, 1e4, 1e1, 1e3, 1e2, 1e5]
    probs = _make(ns, kap, 300)
    B = bfx.Batch(3, ns, config=(nb, bn))
    assert B.config == (nb, bn)
    A, b = B.pack([p.A32 for p in probs], [p.b for p in probs])
    x, status = B.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = B.decode_status(status)
    assert conv.all() and (info == 0).all()
    for p, xb in zip(probs, B.unpack(x)):
        xd, _ = orc.dgesv(p.A32, p.b)
        fe = np.max(np.abs(xb - p.x_true)) / np.max(np.abs(p.x_true))
        fe64 = np.max(np.abs(xd - p.x_true)) / np.max(np.abs(p.x_true))
        assert fe <= 10 * fe64 + 1e-15, (p.n, fe, fe64)


def test_autotune_picks_the_fastest_and_records_it(bfx):
    rng = np.random.default_rng(4)
    ns = rng.integers(32, 257, size=60)
    probs = [bi.fast_system(int(n), 100.0, 400 + i) for i, n in enumerate(ns)]
    B0 = bfx.Batch(3, ns)
    A, b = B0.pack([p.A32 for p in probs], [p.b for p in probs])
    best, best_ms, table = bfx.batch_autotune(3, ns, A, b, reps=2)
    assert len(table) == 9
    ok = [r for r in table if r[3] == 0]
    assert len(ok) == 9 and all(r[2] > 0 for r in ok)
    assert best_ms == min(r[2] for r in ok)
    assert best in [(r[0], r[1]) for r in ok if r[2] == best_ms]
    # a batch of the same make-up takes the recorded shape
    Bt = bfx.Batch(3, ns, config="tuned")
    assert Bt.config == best
    x, status = Bt.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = Bt.decode_status(status)
    assert conv.all()


def test_batch_config_rejected(bfx):
    with pytest.raises(bfx.BfxError):
        bfx.Batch(3, [10, 20], config=(48, 256))
    with pytest.raises(bfx.BfxError):
        bfx.Batch(3, [10, 20], config=(64, 96))


def test_batched_gmres_ir_converges_where_plain_ir_stops(bfx, orc):
    """Ill-conditioned members (kappa 1e7 .. 3e8) of a batch: plain batched
    refinement leaves some unconverged; with GMRES-IR (the default) every one
    converges to within 10x of the FP64 LU forward error."""
    rng = np.random.default_rng(12)
    ns = [int(v) for v in rng.integers(64, 400, size=24)]
    kap = [float(10 ** v) for v in rng.uniform(7.0, 8.5, size=24)]
    probs = _make(ns, kap, 700)
    mats, rhs = [p.A32 for p in probs], [p.b for p in probs]
    B0 = bfx.Batch(6, ns, max_iter=12, gmres=0)
    A, b = B0.pack(mats, rhs)
    x0, st0 = B0.solve(A, b)
    torch.cuda.synchronize()
    conv0 = B0.decode_status(st0)[0]
    assert conv0.sum() < len(ns)  # plain refinement does not reach all of them
    B = bfx.Batch(6, ns, max_iter=12)
    x, st = B.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = B.decode_status(st)
    gs = B.gmres_steps(st)
    assert conv.all() and (info == 0).all(), (conv, iters, berr)
    assert (gs[conv0 == 0] > 0).all() and (gs[conv0 == 1] == 0).all()
    for p, xb in zip(probs, B.unpack(x)):
        xd, _ = orc.dgesv(p.A32, p.b)
        fe = np.max(np.abs(xb - p.x_true)) / np.max(np.abs(p.x_true))
        fe64 = np.max(np.abs(xd - p.x_true)) / np.max(np.abs(p.x_true))
        assert fe <= 10 * fe64 + 1e-15, (p.n, p.kappa_nominal, fe, fe64)
    # systems plain refinement had already converged are untouched by the GMRES phase
    for i in np.nonzero(conv0)[0]:
        assert np.array_equal(B0.unpack(x0)[i], B.unpack(x)[i])


def test_batched_gmres_multiple_rhs(bfx, orc):
    ns = [150, 90, 220]
    probs = [bi.svd_system(n, 3e7, 900 + i, nrhs=3) for i, n in enumerate(ns)]
    B = bfx.Batch(6, ns, nrhs=3, max_iter=12)
    A, b = B.pack([p.A32 for p in probs], [p.b for p in probs])
    x, st = B.solve(A, b)
    torch.cuda.synchronize()
    conv, iters, info, berr = B.decode_status(st)
    assert conv.all()
    for p, xb in zip(probs, B.unpack(x)):
        xd, _ = orc.dgesv(p.A32, p.b)
        fe = np.max(np.abs(xb - p.x_true)) / np.max(np.abs(p.x_true))
        fe64 = np.max(np.abs(xd - p.x_true)) / np.max(np.abs(p.x_true))
        assert fe <= 10 * fe64 + 1e-15


def test_batched_late_steps_large_systems(bfx, orc):
    """Systems of more than 512 unknowns that need more than five refinement
    steps run the later steps in the 1024-thread latency form, where every
    element of x must receive its correction exactly once: results agree
    with the single-system path and repeat bit for bit."""
    ns = [600, 1000, 130, 777]
    probs = _make(ns, [1e4, 1e4, 1e2, 3e4], 1300)
    B = bfx.Batch(3, ns, max_iter=30, gmres=0)
    A, b = B.pack([p.A32 for p in probs], [p.b for p in probs])
    x1, st1 = B.solve(A, b)
    torch.cuda.synchronize()
    x1 = x1.clone()
    conv, iters, info, berr = B.decode_status(st1)
    assert conv.all() and (info == 0).all(), (conv, iters, berr)
    big = np.array([n > 512 for n in ns])
    assert (iters[big] > 5).all(), iters  # the latency form ran on them
    x2, st2 = B.solve(A, b)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    for p, xb in zip(probs, B.unpack(x1)):
        xd, _ = orc.dgesv(p.A32, p.b)
        fe = np.max(np.abs(xb - p.x_true)) / np.max(np.abs(p.x_true))
        fe64 = np.max(np.abs(xd - p.x_true)) / np.max(np.abs(p.x_true))
        assert fe <= 10 * fe64 + 1e-15, (p.n, fe, fe64)
        xs1, res, code = bfx.solve_ir(3, torch.from_numpy(p.A32).cuda(),
                                      torch.from_numpy(p.b).cuda(), escalate=False)
        assert code == 0
        scale = np.max(np.abs(xs1.cpu().numpy()))
        assert np.max(np.abs(xb - xs1.cpu().numpy())) <= 100 * p.kappa_nominal * 2.0 ** -53 * scale * p.n
