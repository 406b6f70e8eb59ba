"""ctypes binding of libbfx.so: argument marshalling only.

Tensors are torch CUDA tensors; their data pointers, leading dimensions and
the current torch stream are passed to the C entry points of ``include/bfx.h``.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libbfx.so")

BFX_FP32, BFX_X1, BFX_X3, BFX_X5, BFX_X6, BFX_X8, BFX_X9 = 0, 1, 3, 5, 6, 8, 9
PIECES = {BFX_X1: 1, BFX_X3: 2, BFX_X6: 3, BFX_X8: 3, BFX_X9: 3}
# pieces of (A, B) a GEMM mode reads; X5 is the asymmetric 2 x 3 split
GEMM_PIECES = {BFX_X1: (1, 1), BFX_X3: (2, 2), BFX_X5: (2, 3), BFX_X6: (3, 3), BFX_X8: (3, 3),
               BFX_X9: (3, 3)}

_STATUS = {
    0: "ok", 1: "invalid argument", 2: "workspace too small", 3: "CUDA error",
    4: "unsupported shape, alignment or device", 5: "exactly zero pivot",
    6: "iterative refinement did not converge", 7: "a bounded device-side wait expired",
}


class BfxError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn}: {_STATUS.get(code, 'unknown')} (status {code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _LIBPATH


def lib() -> ctypes.CDLL:
    """Load libbfx.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise ImportError(f"bfx CUDA library not built: {_LIBPATH} missing "
                          "(run python -m paper_1904_06376_b300.build or __graft_entry__.build())")
    L = ctypes.CDLL(_LIBPATH)
    i64, i32, f32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "bfx_version": (i32, []),
        "bfx_status_string": (ctypes.c_char_p, [i32]),
        "bfx_num_sms": (i32, []),
        "bfx_device_error": (i32, [vp, vp]),
        "bfx_split": (i32, [i64, i64, vp, i64, i32, vp, vp, vp, i64, vp]),
        "bfx_split_transpose": (i32, [i64, i64, vp, i64, i32, vp, vp, vp, i64, vp]),
        "bfx_split_pair": (i32, [i64, i64, vp, i64, i32, vp, vp, vp, i64,
                                 i64, i64, vp, i64, i32, vp, vp, vp, i64, vp]),
        "bfx_gemm_workspace_size": (sz, [i32, i64, i64, i64]),
        "bfx_gemm_bf16xN": (i32, [i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp, sz, vp]),
        "bfx_gemm_bf16xN_fused": (i32, [i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp]),
        "bfx_lowp_lu_ir_batched": (i32, [i32, i32, i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "bfx_gemm_bf16xN_f64": (i32, [i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, sz, vp]),
        "bfx_gemm_presplit": (i32, [i32, i64, i64, i64, f32, vp, i64, i64, vp, i64, i64, f32, vp, i64, vp]),
        "bfx_sgemm_simt": (i32, [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp]),
        "bfx_dot_workspace_size": (sz, []),
        "bfx_lu_workspace_size": (sz, [i32, i64, i32]),
        "bfx_lu_bf16xN": (i32, [i32, i64, i32, vp, i64, vp, vp, vp, sz, vp]),
        "bfx_solve_ir_workspace_size": (sz, [i32, i64, i64, vp]),
        "bfx_solve_ir": (i32, [i32, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp, sz, vp]),
        "bfx_solve_ir_async": (i32, [i32, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp, sz, vp]),
        "bfx_measure_fma_peak": (i32, [i32, vp, vp]),
        "bfx_batch_create": (i32, [vp, i32, i32, vp, i32, vp]),
        "bfx_batch_workspace_size": (sz, [vp]),
        "bfx_batch_solve": (i32, [vp, vp, vp, vp, vp, vp, sz, vp]),
        "bfx_batch_destroy": (None, [vp]),
        "bfx_batch_create_config": (i32, [vp, i32, i32, vp, i32, vp, vp]),
        "bfx_batch_get_config": (i32, [vp, vp]),
        "bfx_batch_autotune": (i32, [i32, i32, vp, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]),
        "bfx_batch_tuned_config": (i32, [i32, i32, vp, i32, vp, vp]),
        "bfx_server_create": (i32, [vp, vp]),
        "bfx_server_submit": (i32, [vp, i64, i64, vp, vp, vp, vp]),
        "bfx_server_wait": (i32, [vp, i64, vp, ctypes.c_double]),
        "bfx_server_stats": (i32, [vp, vp]),
        "bfx_server_destroy": (None, [vp]),
        "bfx_dot_bf16xN": (i32, [i32, i64, vp, vp, vp, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(fn: str, code: int) -> None:
    if code != 0:
        raise BfxError(fn, code)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride (row-major)")
    return t.stride(0)


def version() -> int:
    return lib().bfx_version()


def num_sms() -> int:
    return lib().bfx_num_sms()


def device_error(stream=None) -> int:
    """Read and clear the device error word (bounded-wait expiries)."""
    code = ctypes.c_int(0)
    _check("bfx_device_error", lib().bfx_device_error(ctypes.byref(code), _stream(stream)))
    return code.value


def split(x: torch.Tensor, npieces: int = 3, out=None, stream=None):
    """hi, mid, lo bfloat16 pieces (as int16 bit patterns) of FP32 x (Sec. II-A)."""
    assert x.dtype == torch.float32 and x.is_cuda
    rows, cols = x.shape
    if out is None:
        out = [torch.empty((rows, cols), dtype=torch.int16, device=x.device) for _ in range(npieces)]
    ldp = _ld(out[0]) if rows and cols else max(cols, 1)
    ps = list(out) + [None] * (3 - len(out))
    _check("bfx_split", lib().bfx_split(rows, cols, _ptr(x), _ld(x) if rows and cols else max(cols, 1),
                                        npieces, _ptr(ps[0]), _ptr(ps[1]), _ptr(ps[2]), ldp,
                                        _stream(stream)))
    return out


def split_transpose(x: torch.Tensor, npieces: int = 3, out=None, stream=None):
    """Pieces of x written transposed (cols x rows)."""
    assert x.dtype == torch.float32 and x.is_cuda
    rows, cols = x.shape
    if out is None:
        out = [torch.empty((cols, rows), dtype=torch.int16, device=x.device) for _ in range(npieces)]
    ldp = _ld(out[0]) if rows and cols else max(rows, 1)
    ps = list(out) + [None] * (3 - len(out))
    _check("bfx_split_transpose",
           lib().bfx_split_transpose(rows, cols, _ptr(x), _ld(x) if rows and cols else max(cols, 1),
                                     npieces, _ptr(ps[0]), _ptr(ps[1]), _ptr(ps[2]), ldp,
                                     _stream(stream)))
    return out


def split_pair(a: torch.Tensor, b: torch.Tensor, npa: int = 3, npb: int = 3, out_a=None, out_b=None,
               stream=None):
    """split(a) and split_transpose(b) in one launch (the two operands of a
    product); returns (pieces of a, pieces of b^T)."""
    assert a.dtype == torch.float32 and a.is_cuda and b.dtype == torch.float32 and b.is_cuda
    ra, ca = a.shape
    rb, cb = b.shape
    if out_a is None:
        out_a = [torch.empty((ra, ca), dtype=torch.int16, device=a.device) for _ in range(npa)]
    if out_b is None:
        out_b = [torch.empty((cb, rb), dtype=torch.int16, device=b.device) for _ in range(npb)]
    pa = list(out_a) + [None] * (3 - len(out_a))
    pb = list(out_b) + [None] * (3 - len(out_b))
    lda = _ld(a) if ra and ca else max(ca, 1)
    ldb = _ld(b) if rb and cb else max(cb, 1)
    ldpa = _ld(out_a[0]) if ra and ca else max(ca, 1)
    ldpb = _ld(out_b[0]) if rb and cb else max(rb, 1)
    _check("bfx_split_pair",
           lib().bfx_split_pair(ra, ca, _ptr(a), lda, npa, _ptr(pa[0]), _ptr(pa[1]), _ptr(pa[2]), ldpa,
                                rb, cb, _ptr(b), ldb, npb, _ptr(pb[0]), _ptr(pb[1]), _ptr(pb[2]), ldpb,
                                _stream(stream)))
    return out_a, out_b


def gemm_workspace_size(mode: int, m: int, n: int, k: int) -> int:
    return int(lib().bfx_gemm_workspace_size(mode, m, n, k))


def gemm_bf16xN(mode: int, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None,
                alpha: float = 1.0, beta: float = 0.0, workspace: torch.Tensor = None, stream=None):
    """C = alpha * (A B by the mode's bfloat16 products) + beta * C."""
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
        beta = 0.0
    wsb = gemm_workspace_size(mode, m, n, k) if mode != BFX_FP32 else 0
    if wsb and (workspace is None or workspace.numel() * workspace.element_size() < wsb):
        workspace = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    ws_ptr = _ptr(workspace) if wsb else None
    ws_bytes = workspace.numel() * workspace.element_size() if wsb else 0
    lda = A.stride(0) if m and k else max(k, 1)
    ldb = B.stride(0) if k and n else max(n, 1)
    ldc = C.stride(0) if m and n else max(n, 1)
    _check("bfx_gemm_bf16xN", lib().bfx_gemm_bf16xN(mode, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb,
                                                   beta, _ptr(C), ldc, ws_ptr, ws_bytes,
                                                   _stream(stream)))
    return C


def gemm_bf16xN_f64(mode: int, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None,
                    workspace: torch.Tensor = None, stream=None):
    """C = A B with the mode's partial products added in FP64 and kept in FP64
    (the "d" variant of Sec. IV-A).  C: float64 (m, n)."""
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    wsb = gemm_workspace_size(mode, m, n, k)
    if wsb and (workspace is None or workspace.numel() * workspace.element_size() < wsb):
        workspace = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    ws_bytes = workspace.numel() * workspace.element_size() if wsb else 0
    lda = A.stride(0) if m and k else max(k, 1)
    ldb = B.stride(0) if k and n else max(n, 1)
    ldc = C.stride(0) if m and n else max(n, 1)
    _check("bfx_gemm_bf16xN_f64",
           lib().bfx_gemm_bf16xN_f64(mode, m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc,
                                     _ptr(workspace) if wsb else None, ws_bytes, _stream(stream)))
    return C


LOWP_FP32, LOWP_BF16, LOWP_FP16 = 0, 1, 2


def lowp_lu_ir_batched(typ: int, A: torch.Tensor, b: torch.Tensor, tol: torch.Tensor,
                       max_iter: int = 50, factors: bool = False, stream=None):
    """Single-type LU (every operation rounded to FP32, bfloat16 or binary16)
    and FP64 residual-form refinement of ``count`` n x n systems (the plain IR
    table of Sec. IV-B).  A: (count, n, n) float32, b: (count, n) float64,
    tol: (count,) float64.  Returns x, iters, conv, info (and LU, ipiv when
    ``factors``)."""
    count, n, _ = A.shape
    dev = A.device
    x = torch.empty((count, n), dtype=torch.float64, device=dev)
    iters = torch.empty(count, dtype=torch.int32, device=dev)
    conv = torch.empty(count, dtype=torch.int32, device=dev)
    info = torch.empty(count, dtype=torch.int32, device=dev)
    LU = torch.empty((count, n, n), dtype=torch.float32, device=dev) if factors else None
    ipiv = torch.empty((count, n), dtype=torch.int32, device=dev) if factors else None
    _check("bfx_lowp_lu_ir_batched",
           lib().bfx_lowp_lu_ir_batched(typ, count, n, _ptr(A), _ptr(b), _ptr(tol), int(max_iter),
                                        _ptr(x), _ptr(LU), _ptr(ipiv), _ptr(iters), _ptr(conv),
                                        _ptr(info), _stream(stream)))
    if factors:
        return x, iters, conv, info, LU, ipiv
    return x, iters, conv, info


def gemm_bf16xN_fused(mode: int, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None,
                      alpha: float = 1.0, beta: float = 0.0, stream=None):
    """As ``gemm_bf16xN`` with the split fused into the tensor-core kernel (no
    workspace).  Row strides of A and B must be multiples of 4 elements."""
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
        beta = 0.0
    lda = A.stride(0) if m and k else max(k, 1)
    ldb = B.stride(0) if k and n else max(n, 1)
    ldc = C.stride(0) if m and n else max(n, 1)
    _check("bfx_gemm_bf16xN_fused",
           lib().bfx_gemm_bf16xN_fused(mode, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C),
                                       ldc, _stream(stream)))
    return C


def gemm_presplit(mode: int, Ap: torch.Tensor, Btp: torch.Tensor, k: int, C: torch.Tensor,
                  alpha: float = 1.0, beta: float = 0.0, stream=None):
    """GEMM from piece planes: Ap (np, m, lda_p) and Btp (np, n, ldb_p) int16
    bit patterns of bfloat16; the first k entries of each row are used."""
    _, m, _ = Ap.shape
    _, n, _ = Btp.shape
    _check("bfx_gemm_presplit",
           lib().bfx_gemm_presplit(mode, m, n, k, alpha, _ptr(Ap), Ap.stride(1), Ap.stride(0),
                                   _ptr(Btp), Btp.stride(1), Btp.stride(0), beta, _ptr(C),
                                   C.stride(0), _stream(stream)))
    return C


def sgemm_simt(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None, alpha: float = 1.0,
               beta: float = 0.0, stream=None):
    """Plain FP32 SIMT GEMM (Sec. II-C reference computation)."""
    m, k = A.shape
    _, n = B.shape
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
        beta = 0.0
    lda = A.stride(0) if m and k else max(k, 1)
    ldb = B.stride(0) if k and n else max(n, 1)
    ldc = C.stride(0) if m and n else max(n, 1)
    _check("bfx_sgemm_simt", lib().bfx_sgemm_simt(m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                                                 _ptr(C), ldc, _stream(stream)))
    return C


def dot_bf16xN(mode: int, x: torch.Tensor, y: torch.Tensor, out: torch.Tensor = None,
               workspace: torch.Tensor = None, stream=None) -> torch.Tensor:
    """x^T y by the mode's bfloat16 products; returns a 1-element device tensor."""
    assert x.is_contiguous() and y.is_contiguous() and x.numel() == y.numel()
    if out is None:
        out = torch.empty(1, dtype=torch.float32, device=x.device)
    wsb = int(lib().bfx_dot_workspace_size())
    if workspace is None or workspace.numel() * workspace.element_size() < wsb:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=x.device)
    _check("bfx_dot_bf16xN", lib().bfx_dot_bf16xN(mode, x.numel(), _ptr(x), _ptr(y), _ptr(out),
                                                 _ptr(workspace), wsb, _stream(stream)))
    return out


GMRES_MAX_M = 4096


class IrParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("tol_b", ctypes.c_double),
                ("stall", ctypes.c_double), ("escalate", ctypes.c_int), ("nb", ctypes.c_int),
                ("gmres", ctypes.c_int), ("gmres_m", ctypes.c_int), ("gmres_tol", ctypes.c_double),
                ("gmres_inverses", ctypes.c_int)]


class IrResult(ctypes.Structure):
    _fields_ = [("info", ctypes.c_int32), ("mode_used", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("refactorizations", ctypes.c_int32), ("berr", ctypes.c_double),
                ("gmres_steps", ctypes.c_int32), ("arnoldi", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lu_bf16xN(mode: int, A: torch.Tensor, nb: int = 64, ipiv: torch.Tensor = None,
              info: torch.Tensor = None, workspace: torch.Tensor = None, stream=None):
    """In-place LU with partial pivoting (bf16xN trailing update).  Returns (A, ipiv, info)."""
    n = A.shape[0]
    assert A.shape == (n, n) and A.dtype == torch.float32
    if ipiv is None:
        ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    wsb = int(lib().bfx_lu_workspace_size(mode, n, nb))
    if wsb and (workspace is None or workspace.numel() * workspace.element_size() < wsb):
        workspace = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    _check("bfx_lu_bf16xN", lib().bfx_lu_bf16xN(mode, n, nb, _ptr(A), A.stride(0) if n else 1,
                                               _ptr(ipiv), _ptr(info), _ptr(workspace) if wsb else None,
                                               wsb, _stream(stream)))
    return A, ipiv, info


def solve_ir_workspace_size(mode: int, n: int, nrhs: int, params: "IrParams" = None) -> int:
    return int(lib().bfx_solve_ir_workspace_size(mode, n, nrhs,
                                                 ctypes.byref(params) if params is not None else None))


def solve_ir(mode: int, A: torch.Tensor, b: torch.Tensor, x: torch.Tensor = None, max_iter: int = 50,
             tol: float = 2.0 ** -53, tol_b: float = -1.0, stall: float = 0.5, escalate: bool = True,
             nb: int = 64, gmres: int = 1, gmres_m: int = 0, gmres_tol: float = 1e-10,
             gmres_inverses: bool = True, workspace: torch.Tensor = None, stream=None,
             raise_on_status: bool = False):
    """Solve A x = b (A FP32 n x n, b FP64 n x nrhs) by residual-form refinement.

    gmres: 0 plain refinement only; 1 GMRES-IR once plain refinement stalls
    (after any escalation); 2 GMRES-IR from the first correction.  gmres_m:
    Arnoldi steps per refinement step (0: min(n, GMRES_MAX_M)).
    gmres_inverses: the GMRES preconditioner through explicit FP64 inverses of
    the factors (True) or by row-sliced block substitution (False).
    Returns (x, result dict, status code).  Synchronous."""
    n = A.shape[0]
    if b.dim() == 1:
        b = b[:, None]
    nrhs = b.shape[1]
    if x is None:
        x = torch.empty((n, nrhs), dtype=torch.float64, device=A.device)
    p = IrParams(max_iter, tol, tol_b, stall, int(bool(escalate)), nb, int(gmres), int(gmres_m),
                 float(gmres_tol), int(bool(gmres_inverses)))
    wsb = solve_ir_workspace_size(mode, n, nrhs, p)
    if wsb and (workspace is None or workspace.numel() * workspace.element_size() < wsb):
        workspace = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    r = IrResult()
    code = lib().bfx_solve_ir(mode, n, nrhs, _ptr(A), A.stride(0) if n else 1, _ptr(b),
                              b.stride(0) if n else 1, _ptr(x), x.stride(0) if n else 1,
                              ctypes.byref(p), ctypes.byref(r), _ptr(workspace) if wsb else None, wsb,
                              _stream(stream))
    if code not in (0, 5, 6) or (raise_on_status and code != 0):
        _check("bfx_solve_ir", code)
    return x, r.as_dict(), code


def measure_fma_peak(fp64: bool = False, stream=None) -> float:
    """Measured FP32 (or FP64) FMA rate of the CUDA cores, TFLOP/s."""
    out = ctypes.c_double()
    _check("bfx_measure_fma_peak", lib().bfx_measure_fma_peak(int(bool(fp64)), ctypes.byref(out),
                                                             _stream(stream)))
    return float(out.value)


IR_RESULT_BYTES = ctypes.sizeof(IrResult)


def solve_ir_async(mode: int, A: torch.Tensor, b: torch.Tensor, x: torch.Tensor = None,
                   max_iter: int = 50, tol: float = 2.0 ** -53, tol_b: float = -1.0,
                   stall: float = 0.5, nb: int = 64, result: torch.Tensor = None,
                   workspace: torch.Tensor = None, stream=None):
    """Enqueue the plain refinement solve (no escalation, no GMRES) on the
    stream; nothing is read back.  Returns (x, result) with ``result`` a
    device uint8 tensor holding the bfx_ir_result (``decode_ir_result``)."""
    n = A.shape[0]
    if b.dim() == 1:
        b = b[:, None]
    nrhs = b.shape[1]
    if x is None:
        x = torch.empty((n, nrhs), dtype=torch.float64, device=A.device)
    if result is None:
        result = torch.zeros(IR_RESULT_BYTES, dtype=torch.uint8, device=A.device)
    p = IrParams(max_iter, tol, tol_b, stall, 0, nb, 0, 0, 0.0)
    wsb = solve_ir_workspace_size(mode, n, nrhs, p)
    if workspace is None or workspace.numel() * workspace.element_size() < wsb:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    _check("bfx_solve_ir_async",
           lib().bfx_solve_ir_async(mode, n, nrhs, _ptr(A), A.stride(0), _ptr(b), b.stride(0),
                                    _ptr(x), x.stride(0), ctypes.byref(p), _ptr(result),
                                    _ptr(workspace), wsb, _stream(stream)))
    return x, result


def decode_ir_result(result: torch.Tensor) -> dict:
    """The bfx_ir_result an asynchronous solve wrote (copies it to the host)."""
    raw = bytes(result.cpu().numpy().tobytes())
    return IrResult.from_buffer_copy(raw[:IR_RESULT_BYTES]).as_dict()


class BatchConfig(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("gemm_bn", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("config", BatchConfig), ("ms", ctypes.c_float), ("status", ctypes.c_int32)]


def _batch_params(max_iter, tol, tol_b, stall, gmres=1):
    return IrParams(max_iter, tol, tol_b, stall, 0, 64, int(gmres), 0, 0.0)


def batch_autotune(mode: int, ns, A, b, nrhs: int = 1, x=None, status=None, reps: int = 3,
                   max_iter: int = 20, tol: float = 2.0 ** -53, tol_b: float = -1.0,
                   stall: float = 0.5, gmres: int = 1, stream=None):
    """Time the batch (packed A, b on the device) under every tile shape and
    return ((nb, gemm_bn) of the fastest, its median ms, [(nb, gemm_bn, ms,
    status), ...])."""
    import numpy as np

    ns = np.asarray(ns, dtype=np.int32)
    if x is None:
        x = torch.empty(int((ns.astype(np.int64) * nrhs).sum()), dtype=torch.float64, device=A.device)
    if status is None:
        status = torch.zeros(3 * int(ns.size), dtype=torch.float64, device=A.device)
    p = _batch_params(max_iter, tol, tol_b, stall, gmres)
    best = BatchConfig()
    best_ms = ctypes.c_float()
    table = (TuneEntry * 9)()
    tlen = ctypes.c_int(9)
    _check("bfx_batch_autotune",
           lib().bfx_batch_autotune(mode, int(ns.size), ns.ctypes.data, nrhs, ctypes.byref(p), _ptr(A),
                                    _ptr(b), _ptr(x), _ptr(status), int(reps), _stream(stream),
                                    ctypes.byref(best), ctypes.byref(best_ms), table, ctypes.byref(tlen)))
    rows = [(e.config.nb, e.config.gemm_bn, float(e.ms), int(e.status)) for e in table[: tlen.value]]
    return (best.nb, best.gemm_bn), float(best_ms.value), rows


class Batch:
    """Batched solves of many uneven-size systems (bfx_batch_* of the C ABI).

    ns: sizes of the systems (1..1024); matrices / right-hand sides are packed
    back to back (see ``pack``).  ``solve`` enqueues one CUDA-graph launch and
    returns the device status tensor (decode with ``decode_status``).
    config: None (default shape), (nb, gemm_bn), or "tuned" (the shape the
    autotuner recorded for batches like this one; default if none)."""

    def __init__(self, mode: int, ns, nrhs: int = 1, max_iter: int = 20, tol: float = 2.0 ** -53,
                 tol_b: float = -1.0, stall: float = 0.5, config=None, gmres: int = 1):
        import numpy as np

        self.ns = np.asarray(ns, dtype=np.int32)
        self.nrhs = nrhs
        self.mode = mode
        h = ctypes.c_void_p()
        p = _batch_params(max_iter, tol, tol_b, stall, gmres)
        cfg = None
        if config == "tuned":
            c = BatchConfig()
            if lib().bfx_batch_tuned_config(mode, int(self.ns.size), self.ns.ctypes.data, nrhs,
                                            ctypes.byref(p), ctypes.byref(c)) == 0:
                cfg = c
        elif config is not None:
            cfg = BatchConfig(int(config[0]), int(config[1]))
        _check("bfx_batch_create_config",
               lib().bfx_batch_create_config(ctypes.byref(h), mode, int(self.ns.size), self.ns.ctypes.data,
                                             nrhs, ctypes.byref(p),
                                             ctypes.byref(cfg) if cfg is not None else None))
        self.handle = h
        got = BatchConfig()
        _check("bfx_batch_get_config", lib().bfx_batch_get_config(h, ctypes.byref(got)))
        self.config = (got.nb, got.gemm_bn)
        self.ws_bytes = int(lib().bfx_batch_workspace_size(h))
        self.offA = np.concatenate([[0], np.cumsum(self.ns.astype(np.int64) ** 2)])
        self.offV = np.concatenate([[0], np.cumsum(self.ns.astype(np.int64) * nrhs)])
        self.workspace = None

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bfx_batch_destroy(self.handle)
            self.handle = None

    def pack(self, mats, rhs, device="cuda"):
        """Pack lists of (n,n) FP32 matrices and (n,nrhs) FP64 right-hand sides."""
        import numpy as np

        A = np.concatenate([np.asarray(m, np.float32).ravel() for m in mats])
        b = np.concatenate([np.asarray(v, np.float64).reshape(-1) for v in rhs])
        return torch.from_numpy(A).to(device), torch.from_numpy(b).to(device)

    def unpack(self, x):
        import numpy as np

        xa = x.cpu().numpy()
        return [xa[self.offV[i]:self.offV[i + 1]].reshape(int(n), self.nrhs) for i, n in enumerate(self.ns)]

    def solve(self, A, b, x=None, status=None, stream=None):
        if x is None:
            x = torch.empty(int(self.offV[-1]), dtype=torch.float64, device=A.device)
        if status is None:
            status = torch.zeros(3 * int(self.ns.size), dtype=torch.float64, device=A.device)
        if self.workspace is None:
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=A.device)
        _check("bfx_batch_solve", lib().bfx_batch_solve(self.handle, _ptr(A), _ptr(b), _ptr(x),
                                                       _ptr(status), _ptr(self.workspace), self.ws_bytes,
                                                       _stream(stream)))
        return x, status

    @staticmethod
    def decode_status(status):
        """converged, iters, info (int arrays) and berr (float array) per system."""
        import numpy as np

        raw = status.cpu().numpy().view(np.uint8).reshape(-1, 24)
        ints = raw[:, :16].copy().view(np.int32).reshape(-1, 4)
        berr = raw[:, 16:].copy().view(np.float64).ravel()
        return ints[:, 0], ints[:, 1], ints[:, 2], berr

    @staticmethod
    def gmres_steps(status):
        """GMRES-IR refinement steps per system (0 if plain refinement converged)."""
        import numpy as np

        raw = status.cpu().numpy().view(np.uint8).reshape(-1, 24)
        return raw[:, :16].copy().view(np.int32).reshape(-1, 4)[:, 3]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int), ("mode", ctypes.c_int),
                ("nb", ctypes.c_int), ("escalate", ctypes.c_int), ("gmres", ctypes.c_int),
                ("batch_max_n", ctypes.c_int), ("batch_max", ctypes.c_int)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("converged", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("info", ctypes.c_int32), ("mode_used", ctypes.c_int32),
                ("refactorizations", ctypes.c_int32), ("berr", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("gmres_steps", ctypes.c_int32), ("arnoldi", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("peak_running", ctypes.c_int32),
                ("batches", ctypes.c_int32), ("pool_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_used_bytes", ctypes.c_size_t)]


class Server:
    """Continuous-admission solve server (bfx_server_* of the C ABI).

    submit() takes host numpy arrays (kept alive here until the request
    completes) and returns a ticket; wait() returns (x, result dict)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 16, mode: int = BFX_X3, nb: int = 64,
                 escalate: bool = True, gmres: int = 1, batch_max_n: int = 0, batch_max: int = 0):
        cfg = ServerConfig(int(budget_bytes), int(max_inflight), int(mode), int(nb), int(bool(escalate)),
                           int(gmres), int(batch_max_n), int(batch_max))
        h = ctypes.c_void_p()
        _check("bfx_server_create", lib().bfx_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self.handle = h
        self._live = {}

    def submit(self, A, b):
        import numpy as np

        A = np.ascontiguousarray(A, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float64)
        if b.ndim == 1:
            b = b[:, None]
        n, nrhs = b.shape
        x = np.empty((n, nrhs), dtype=np.float64)
        t = ctypes.c_int64()
        _check("bfx_server_submit", lib().bfx_server_submit(self.handle, n, nrhs, A.ctypes.data, b.ctypes.data,
                                                           x.ctypes.data, ctypes.byref(t)))
        self._live[t.value] = (A, b, x)
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        r = RequestResult()
        code = lib().bfx_server_wait(self.handle, ticket, ctypes.byref(r), float(timeout_s))
        if code == 7:
            return None
        _check("bfx_server_wait", code)
        _, _, x = self._live.pop(ticket)
        return x, r.as_dict()

    def stats(self):
        st = ServerStats()
        _check("bfx_server_stats", lib().bfx_server_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_ if f != "pad"}

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bfx_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
