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
