"""The workspace-free GEMM entry point, called through the C ABI.

bfx_gemm_bf16xN_noalloc serves callers that cannot allocate device memory
(a host application that owns all device memory and forbids library
allocations, or a loop that cannot afford one): it keeps the bfloat16 pieces
in a fixed array inside the library instead of a caller workspace.  Its
results must match the workspace entry point, bfx_gemm_bf16xN, within the
tolerance the GEMM tests use, on consecutive calls that reuse the shared
array.  This file is collected last so a failure here stops a run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import bfx_inputs as bi
from _tol import tol

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def _noalloc(bfx):
    f = bfx.lib().bfx_gemm_bf16xN_noalloc
    i64, f32, vp = ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp]
    return f


def _call(bfx, mode, A, B, C, alpha=1.0, beta=0.0):
    m, k = A.shape
    n = B.shape[1]
    return _noalloc(bfx)(mode, m, n, k, alpha, A.data_ptr(), A.stride(0), B.data_ptr(),
                         B.stride(0), beta, C.data_ptr(), C.stride(0),
                         torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("mode", [3, 6, 9])
def test_noalloc_matches_workspace_entry_point_twice(bfx, orc, mode):
    # two calls in a row with different shapes and data: the second must not
    # see anything left in the shared array by the first
    cases = [(300, 520, 200, 1), (512, 256, 1000, 2)]
    for m, n, k, seed in cases:
        An = bi.wide_range((m, k), 10 * seed)
        Bn = bi.wide_range((k, n), 10 * seed + 1)
        A, B = torch.from_numpy(An).cuda(), torch.from_numpy(Bn).cuda()
        C0 = torch.from_numpy(bi.uniform_pm1((m, n), 10 * seed + 2)).cuda()
        ref = bfx.gemm_bf16xN(mode, A, B, C0.clone(), alpha=-1.0, beta=1.0)
        C = C0.clone()
        assert _call(bfx, mode, A, B, C, alpha=-1.0, beta=1.0) == 0
        torch.cuda.synchronize()
        _, Cabs = orc.dgemm_rows(An, Bn)
        diff = np.abs(C.cpu().numpy().astype(np.float64) - ref.cpu().numpy())
        assert np.all(diff <= tol(mode, k) * Cabs + 1e-38)


def test_noalloc_rejects_problems_beyond_its_array(bfx):
    """x6 at 2048^3 needs 48 MiB of pieces, more than the 32 MiB array."""
    m = n = k = 2048
    need = 2 * 3 * 2 * m * k
    assert need > SCRATCH_BYTES
    A = torch.zeros((m, k), device="cuda")
    B = torch.zeros((k, n), device="cuda")
    C = torch.zeros((m, n), device="cuda")
    assert _call(bfx, 6, A, B, C) == 2  # BFX_ENOMEM, nothing launched
    # the largest cube that fits still works
    m = n = k = 1536
    A = torch.from_numpy(bi.uniform_pm1((m, k), 3)).cuda()
    B = torch.from_numpy(bi.uniform_pm1((k, n), 4)).cuda()
    C = torch.empty((m, n), device="cuda")
    assert _call(bfx, 6, A, B, C) == 0
    ref = bfx.gemm_bf16xN(6, A, B)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
