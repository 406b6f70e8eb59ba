"""The workspace-free GEMM entry point, called through the C ABI.

bfx_gemm_bf16xN_noalloc serves callers that cannot allocate device memory
(a host application that owns all device memory and forbids library
allocations, or a loop that cannot afford one): it keeps the bfloat16 pieces
in a fixed array inside the library instead of a caller workspace.  It runs
the same split and GEMM kernels as the workspace entry point,
bfx_gemm_bf16xN, on the same pieces, so its results must equal that entry
point's bit for bit, on consecutive calls that reuse the shared array, and
lie within the GEMM error bound of the FP64 product.  This file is collected
last so a failure here stops a run only after every other test has run.
"""
import ctypes

import pytest
import torch

import bfx_inputs as bi
from _tol import check_bound

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
    return _noalloc(bfx)(mode, m, n, k, alpha, A.data_ptr(), max(A.stride(0), 1),
                         B.data_ptr(), max(B.stride(0), 1), beta, C.data_ptr(), C.stride(0),
                         torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("mode", [1, 3, 5, 6, 8, 9])
def test_noalloc_matches_workspace_entry_point_twice(bfx, orc, mode):
    # Calls in a row with different shapes and data: a larger call first,
    # then smaller ones whose k is not a multiple of 8, so piece rows are
    # padded and anything the earlier call left in the shared array (pieces
    # or padding) would show.
    cases = [(512, 256, 1000, 2), (300, 520, 203, 1), (129, 77, 13, 3)]
    for m, n, k, seed in cases:
        An = bi.wide_range((m, k), 10 * seed)
        Bn = bi.wide_range((k, n), 10 * seed + 1)
        A, B = torch.from_numpy(An).cuda(), torch.from_numpy(Bn).cuda()
        C0 = torch.from_numpy(bi.uniform_pm1((m, n), 10 * seed + 2)).cuda()
        ref = bfx.gemm_bf16xN(mode, A, B, C0.clone(), alpha=-1.0, beta=1.0)
        C = C0.clone()
        assert _call(bfx, mode, A, B, C, alpha=-1.0, beta=1.0) == 0
        torch.cuda.synchronize()
        assert torch.equal(C, ref), (mode, m, n, k)
        # and within the mode's error bound of the FP64 product
        C64, Cabs = orc.dgemm_rows(An, Bn)
        check_bound(C.cpu().numpy(), C64, Cabs, mode, k, alpha=-1.0, Cin=C0.cpu().numpy(),
                    beta=1.0)


def test_noalloc_k_zero_scales_c(bfx):
    """k = 0: C = beta C, nothing split."""
    C0 = torch.from_numpy(bi.uniform_pm1((40, 24), 5)).cuda()
    A = torch.zeros((40, 0), device="cuda")
    B = torch.zeros((0, 24), device="cuda")
    C = C0.clone()
    assert _call(bfx, 6, A, B, C, alpha=1.0, beta=0.5) == 0
    torch.cuda.synchronize()
    assert torch.equal(C, C0 * 0.5)


def test_noalloc_rejects_modes_without_pieces(bfx):
    A = torch.zeros((8, 8), device="cuda")
    B = torch.zeros((8, 8), device="cuda")
    C = torch.zeros((8, 8), device="cuda")
    for mode in (0, 2, 4, 7, 10, -1):
        assert _call(bfx, mode, A, B, C) == 1  # BFX_EINVAL
    assert _call(bfx, 5, A, B, C) == 0


def test_noalloc_rejects_problems_beyond_its_array(bfx):
    """x6 at 2048^3 needs 48 MiB of pieces, more than the 32 MiB array; x5
    (two pieces of A, three of B) at 1800 x 1800 x 1600 needs 28.8 MB and fits."""
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
    m, n, k = 1800, 1800, 1600
    assert 2 * (2 * m * k + 3 * n * k) <= SCRATCH_BYTES < 2 * 3 * (m + n) * k
    A = torch.from_numpy(bi.uniform_pm1((m, k), 5)).cuda()
    B = torch.from_numpy(bi.uniform_pm1((k, n), 6)).cuda()
    C = torch.empty((m, n), device="cuda")
    assert _call(bfx, 5, A, B, C) == 0
    ref = bfx.gemm_bf16xN(5, A, B)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
