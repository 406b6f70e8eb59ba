"""The asynchronous solve (bfx_solve_ir_async) through the C ABI: the plain
residual-form refinement of Sec. III with every stop decision made on the
device and the result written to device memory.  Two solves are enqueued on
one stream with no host synchronisation between them; each must equal the
synchronous bfx_solve_ir (escalate = 0, gmres = 0) bit for bit, since both
run the same kernels in the same order, and be within 10x of the oracle's
FP64 LU solve in forward error."""
import numpy as np
import pytest
import torch

import bfx_inputs as bi

pytestmark = pytest.mark.gpu


def _fe(x, P):
    return np.max(np.abs(x - P.x_true)) / np.max(np.abs(P.x_true))


@pytest.mark.parametrize("mode", [0, 3, 6])
def test_two_async_solves_on_one_stream_match_sync(bfx, orc, mode):
    probs = [bi.svd_system(300, 1e4, 21, nrhs=3), bi.svd_system(257, 1e2, 22, nrhs=1)]
    dev = [(torch.from_numpy(P.A32).cuda(), torch.from_numpy(P.b).cuda()) for P in probs]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = [bfx.solve_ir_async(mode, A, b, stream=s) for A, b in dev]  # no sync between
    s.synchronize()
    for (x, res), (A, b), P in zip(outs, dev, probs):
        r = bfx.decode_ir_result(res)
        xs, rs, code = bfx.solve_ir(mode, A, b, escalate=False, gmres=0)
        torch.cuda.synchronize()
        assert code == 0 and rs["converged"] == 1
        assert r["info"] == 0 and r["converged"] == 1 and r["mode_used"] == mode
        assert r["iters"] == rs["iters"] and r["berr"] == rs["berr"]
        assert torch.equal(x, xs)
        xd, _ = orc.dgesv(P.A32, P.b)
        assert _fe(x.cpu().numpy(), P) <= 10 * _fe(xd, P) + 1e-15


def test_async_solve_reports_zero_pivot_and_non_convergence(bfx):
    A = torch.eye(8, device="cuda")
    A[3, 3] = 0.0
    b = torch.ones((8, 1), dtype=torch.float64, device="cuda")
    x, res = bfx.solve_ir_async(3, A, b)
    r = bfx.decode_ir_result(res)
    assert r["info"] == 4 and r["converged"] == 0
    # x1 factors cannot refine a kappa 1e8 system: reported on the device
    P = bi.svd_system(200, 1e8, 3)
    A = torch.from_numpy(P.A32).cuda()
    b = torch.from_numpy(P.b).cuda()
    x, res = bfx.solve_ir_async(1, A, b)
    r = bfx.decode_ir_result(res)
    xs, rs, code = bfx.solve_ir(1, A, b, escalate=False, gmres=0)
    assert code == 6 and r["converged"] == 0 and r["info"] == 0
    assert r["iters"] == rs["iters"]
    assert torch.equal(x, xs)


def test_async_solve_rejects_host_decisions(bfx):
    import ctypes

    A = torch.eye(4, device="cuda")
    b = torch.ones((4, 1), dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    res = torch.zeros(bfx._bfx.IR_RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for esc, gm in ((1, 0), (0, 1), (0, 2)):
        p = bfx._bfx.IrParams(50, 2.0 ** -53, -1.0, 0.5, esc, 64, gm, 0, 0.0)
        wsb = bfx.solve_ir_workspace_size(3, 4, 1, p)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        code = bfx.lib().bfx_solve_ir_async(3, 4, 1, A.data_ptr(), 4, b.data_ptr(), 1,
                                            x.data_ptr(), 1, ctypes.byref(p), res.data_ptr(),
                                            ws.data_ptr(), wsb, None)
        assert code == 1
