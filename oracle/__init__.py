"""CPU oracle for the BF16-split method (Henry, Tang & Heinecke, ARITH 2019).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import it; the library under test never does.
It shares no code with the CUDA path.  The arithmetic lives in ``oracle.c``
(plain C, compiled with ``oracle/build.py``); this module marshals numpy arrays.

Functions and the passages they follow:

* ``bf16_rne``       -- the conversion (B16) of Sec. II-A, round to nearest even.
* ``split``          -- the decomposition b0, b1, b2 of Sec. II-A.
* ``gemm`` / ``dot`` -- the partial products Z^(i,j) with FP32 FMA accumulation,
  level sums and smallest-first combinations of Sec. II-D / II-G
  (mode 0 = the plain FP32 FMA reference of Sec. II-C).
* ``dot_partials``   -- the nine Z^(i,j) of Sec. II-D for one vector pair.
* ``dgemm_rows``     -- FP64 product and |A||B| (the DGEMM baseline of Sec. IV-A).
* ``dgetrf`` / ``dgetrs`` -- FP64 LU with partial pivoting and solve.
* ``lu``             -- the LU of record: unblocked, partial pivoting, division
  by the pivot, each trailing-update product the mode's product (Sec. IV-A).
* ``lu_mirror``      -- regression mirror of the device's blocked LU schedule.
* ``solve_ir``       -- residual-form iterative refinement (Sec. III).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

MODES = (0, 1, 3, 5, 6, 8, 9)  # 0 = plain FP32 FMA; else the number of bf16 products
PIECES = {1: 1, 3: 2, 6: 3, 9: 3}


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        vp = ctypes.c_void_p
        L.orc_bf16_rne.restype = ctypes.c_uint16
        L.orc_bf16_rne.argtypes = [f32]
        L.orc_f16_rne_array.restype = None
        L.orc_f16_rne_array.argtypes = [i64, vp, vp]
        L.orc_lu_lowp.restype = i32
        L.orc_lu_lowp.argtypes = [i32, i64, vp, i64, vp]
        L.orc_bf16_rne_array.argtypes = [i64, vp, vp]
        L.orc_split.argtypes = [i64, vp, i32, vp, vp, vp]
        L.orc_split_bits_range.argtypes = [ctypes.c_uint64, i64, i32, vp, vp, vp]
        L.orc_gemm.restype = i32
        L.orc_gemm.argtypes = [i32, i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64]
        L.orc_gemm_f64out.restype = i32
        L.orc_gemm_f64out.argtypes = [i32, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64]
        L.orc_dot_partials.argtypes = [i64, vp, vp, vp]
        L.orc_dot.restype = f32
        L.orc_dot.argtypes = [i32, i32, i64, vp, vp]
        L.orc_dgemm_rows.argtypes = [i64, vp, i64, i64, vp, i64, vp, i64, vp, vp]
        L.orc_dgetrf.restype = i32
        L.orc_dgetrf.argtypes = [i64, vp, i64, vp]
        L.orc_dgetrs.argtypes = [i64, i64, vp, i64, vp, vp, i64]
        L.orc_lu.restype = i32
        L.orc_lu.argtypes = [i32, i64, i64, vp, i64, vp]
        L.orc_lu_plain.restype = i32
        L.orc_lu_plain.argtypes = [i32, i64, vp, i64, vp]
        L.orc_solve_ir.argtypes = [i64, i64, vp, i64, vp, i64, vp, vp, i64, vp, i64, i32, f64,
                                   f64, f64, vp, vp, vp]
        L.orc_num_threads.restype = i32
        L.orc_gmres.argtypes = [i64, vp, i64, vp, i64, vp, vp, vp, vp, i32, f64, vp, vp]
        L.orc_gmres.restype = i32
        L.orc_solve_gmres_ir.argtypes = [i64, i64, vp, i64, vp, i64, vp, vp, i64, vp, i64, i32,
                                         f64, f64, f64, i32, f64, i32, vp, vp, vp, vp]
        L.orc_tri_inverse.argtypes = [i64, vp, i64, i32, vp]
        L.orc_set_num_threads.argtypes = [i32]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- (B16), split
def bf16_rne(x) -> np.ndarray:
    """(B16) of Sec. II-A: FP32 -> bfloat16 bit patterns, round to nearest even."""
    x = _f32(x)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_bf16_rne_array(x.size, _p(x), _p(out))
    return out


def f16_rne(x) -> np.ndarray:
    """IEEE binary16 bit patterns of FP32 values, round to nearest even."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_f16_rne_array(x.size, _p(x), _p(out))
    return out


LOWP_FP32, LOWP_BF16, LOWP_FP16 = 0, 1, 2


def lu_lowp(typ: int, A):
    """Single-type LU (Sec. IV-B plain IR table, reading R26): every operation
    rounded to the type (0 FP32, 1 bfloat16, 2 binary16).  Returns the
    factors (FP32 array of type values), ipiv (0-based) and info."""
    LU = np.array(A, dtype=np.float32, order="C", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().orc_lu_lowp(int(typ), n, _p(LU), n, _p(ipiv))
    return LU, ipiv, int(info)


def lowp_lu_solve_ir(typ: int, A32, b, tol: float, max_iter: int = 50):
    """The single-type LU, then the refinement of Sec. III with those factors
    and no stall rule: converged when a correction is <= tol |x|_inf within
    max_iter corrections (reading R26)."""
    LU, ipiv, info = lu_lowp(typ, A32)
    x, iters, conv, berr = solve_ir(A32, LU, ipiv, b, max_iter=max_iter, tol=tol,
                                    tol_b=0.0, stall=float("inf"))
    return x, int(iters[0]), int(conv[0]), info, LU, ipiv


def bf16_to_f32(bits) -> np.ndarray:
    """(F32) of a bfloat16 bit pattern: exact widening (the top half of an FP32 word)."""
    bits = np.asarray(bits, dtype=np.uint16)
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)


def split(x, npieces: int = 3):
    """b0, b1, b2 of Sec. II-A (bfloat16 bit patterns, same shape as x)."""
    if npieces not in (1, 2, 3):
        raise ValueError("npieces must be 1, 2 or 3")
    x = _f32(x)
    outs = [np.zeros(x.shape, dtype=np.uint16) for _ in range(3)]
    lib().orc_split(x.size, _p(x), npieces, _p(outs[0]), _p(outs[1]), _p(outs[2]))
    return outs[:npieces]


def split_bits_range(start: int, count: int, npieces: int = 3):
    """Split of every FP32 bit pattern start .. start+count-1."""
    outs = [np.zeros(count, dtype=np.uint16) for _ in range(3)]
    lib().orc_split_bits_range(start, count, npieces, _p(outs[0]), _p(outs[1]), _p(outs[2]))
    return outs[:npieces]


# ---------------------------------------------------------------- products
def gemm(mode: int, A, B, alpha: float = 1.0, beta: float = 0.0, C=None, sum64: bool = False):
    """C = alpha * (A B by the mode's products) + beta * C, FP32 in / out.

    mode 0: plain FP32 FMA accumulation (Sec. II-C); 1/3/6/8/9: bf16x1 .. x9
    (Sec. II-D, II-G); 5: A in two pieces, B in three (Sec. II-G's asymmetric
    case); ``sum64`` is the FP64 final collection ("d" variant).
    """
    A = _f32(A)
    B = _f32(B)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = np.zeros((m, n), dtype=np.float32)
        beta = 0.0
    else:
        C = _f32(C).copy()
    rc = lib().orc_gemm(int(mode), int(bool(sum64)), m, n, k, float(alpha), _p(A), k, _p(B), n,
                        float(beta), _p(C), n)
    if rc:
        raise ValueError(f"orc_gemm failed ({rc})")
    return C


def gemm_f64out(mode: int, A, B, sum64: bool = True) -> np.ndarray:
    """A B by the mode's products with the final collection kept in FP64.

    With ``sum64`` this is the "d" variant of Sec. IV-A (bx3_6d): the FP32
    partial products are collected in FP64 and not rounded back to FP32.
    """
    A = _f32(A)
    B = _f32(B)
    m, k = A.shape
    n = B.shape[1]
    Cd = np.zeros((m, n))
    rc = lib().orc_gemm_f64out(int(mode), int(bool(sum64)), m, n, k, _p(A), k, _p(B), n, _p(Cd), n)
    if rc:
        raise ValueError(f"orc_gemm_f64out failed ({rc})")
    return Cd


def dot(mode: int, x, y, sum64: bool = False) -> np.float32:
    x = _f32(x).ravel()
    y = _f32(y).ravel()
    return np.float32(lib().orc_dot(int(mode), int(bool(sum64)), x.size, _p(x), _p(y)))


def dot_partials(x, y) -> np.ndarray:
    """The nine FP32 partial inner products Z^(i,j) of Sec. II-D as a 3x3 array."""
    x = _f32(x).ravel()
    y = _f32(y).ravel()
    Z = np.zeros(9, dtype=np.float32)
    lib().orc_dot_partials(x.size, _p(x), _p(y), _p(Z))
    return Z.reshape(3, 3)


def dgemm_rows(A, B, rows=None):
    """FP64 A[rows] @ B and |A[rows]| @ |B| (the DGEMM reference of Sec. IV-A)."""
    A = _f32(A)
    B = _f32(B)
    m, k = A.shape
    n = B.shape[1]
    rows = np.arange(m, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    C64 = np.empty((rows.size, n))
    Cabs = np.empty((rows.size, n))
    lib().orc_dgemm_rows(rows.size, _p(rows), n, k, _p(A), k, _p(B), n, _p(C64), _p(Cabs))
    return C64, Cabs


# ---------------------------------------------------------------- LU / solve
def dgetrf(A):
    """FP64 LU with partial pivoting.  Returns (LU, ipiv (0-based), info)."""
    LU = np.array(A, dtype=np.float64, order="C", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().orc_dgetrf(n, _p(LU), n, _p(ipiv))
    return LU, ipiv, int(info)


def dgetrs(LU, ipiv, b):
    LU = np.ascontiguousarray(LU, dtype=np.float64)
    x = np.array(b, dtype=np.float64, order="C", copy=True)
    if x.ndim == 1:
        x = x[:, None]
    n, nrhs = x.shape
    lib().orc_dgetrs(n, nrhs, _p(LU), n, _p(np.ascontiguousarray(ipiv, np.int32)), _p(x), nrhs)
    return x


def dgesv(A, b):
    LU, ipiv, info = dgetrf(A)
    return dgetrs(LU, ipiv, b), info


def lu(mode: int, A):
    """The LU of record (Sec. IV-A "SGETRF based on triplets", reading R12):
    unblocked right-looking LU with partial pivoting of an FP32 matrix,
    multipliers by IEEE division, every trailing-update product the mode's
    product (mode 0: the FP32 FMA).  Returns (LU, ipiv (0-based), info)."""
    LU = np.array(A, dtype=np.float32, order="C", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().orc_lu_plain(int(mode), n, _p(LU), n, _p(ipiv))
    if info < 0:
        raise RuntimeError("orc_lu_plain failed")
    return LU, ipiv, int(info)


def lu_mirror(mode: int, A, nb: int = 64):
    """Regression mirror, not the oracle of record: the blocked schedule of
    the device LU (8-column panel tiles, division by the pivot, rank-nb trailing
    updates by the mode's product), so a change of the device's FP32
    arithmetic shows bit for bit."""
    LU = np.array(A, dtype=np.float32, order="C", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().orc_lu(int(mode), n, int(nb), _p(LU), n, _p(ipiv))
    if info < 0:
        raise RuntimeError("orc_lu failed")
    return LU, ipiv, int(info)


def solve_ir(A32, LU, ipiv, b, max_iter: int = 50, tol: float = 2.0**-53, tol_b=None,
             stall: float = 0.5):
    """Residual-form iterative refinement of Sec. III with given FP32 factors.

    Stops converged when a correction is below ``tol`` relative to x, or when
    the corrections stop shrinking (ratio >= ``stall``) with the normwise
    backward error <= ``tol_b`` (default sqrt(n) 2^-53).
    """
    A32 = _f32(A32)
    LU = _f32(LU)
    n = A32.shape[0]
    b = np.array(b, dtype=np.float64, order="C", copy=True)
    if b.ndim == 1:
        b = b[:, None]
    nrhs = b.shape[1]
    if tol_b is None:
        tol_b = 2.0 ** -53 * np.sqrt(n)
    x = np.zeros((n, nrhs))
    iters = np.zeros(nrhs, dtype=np.int32)
    conv = np.zeros(nrhs, dtype=np.int32)
    berr = np.zeros(nrhs)
    lib().orc_solve_ir(n, nrhs, _p(A32), n, _p(LU), n, _p(np.ascontiguousarray(ipiv, np.int32)),
                       _p(b), nrhs, _p(x), nrhs, int(max_iter), float(tol), float(tol_b), float(stall),
                       _p(iters), _p(conv), _p(berr))
    return x, iters, conv, berr


def lu_solve_ir(mode: int, A32, b, **kw):
    """The LU of record, then the refinement of Sec. III with its factors."""
    LU, ipiv, info = lu(mode, A32)
    x, iters, conv, berr = solve_ir(A32, LU, ipiv, b, **kw)
    return x, iters, conv, berr, info


def tri_inverse(LU, lower: bool) -> np.ndarray:
    """Reading R27: L^-1 (lower, unit diagonal) or U^-1 of the packed FP32
    factors, in FP64, column c by substitution on e_c."""
    LU = _f32(LU)
    n = LU.shape[0]
    X = np.zeros((n, n))
    lib().orc_tri_inverse(n, _p(LU), n, int(bool(lower)), _p(X))
    return X


def gmres(A32, LU, ipiv, rhs, m: int = 50, tau: float = 1e-10, inverses: bool = False):
    """Left-preconditioned GMRES on M^-1 A d = M^-1 rhs (M from the FP32
    factors, FP64 arithmetic), zero first guess; M^-1 by substitution, or
    through the explicit inverses when ``inverses`` (R27).  Returns d, the
    number of Arnoldi steps k and the residual estimates |g_1| .. |g_k|."""
    A32 = _f32(A32)
    LU = _f32(LU)
    n = A32.shape[0]
    rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(n)
    d = np.zeros(n)
    hist = np.zeros(max(m, 1))
    XL = tri_inverse(LU, True) if inverses else None
    XU = tri_inverse(LU, False) if inverses else None
    k = lib().orc_gmres(n, _p(A32), n, _p(LU), n, _p(np.ascontiguousarray(ipiv, np.int32)),
                        _p(XL) if inverses else None, _p(XU) if inverses else None,
                        _p(rhs), int(m), float(tau), _p(d), _p(hist))
    return d, int(k), hist[:k].copy()


def solve_gmres_ir(A32, LU, ipiv, b, max_iter: int = 50, tol: float = 2.0**-53, tol_b=None,
                   stall: float = 0.5, m: int = 50, tau: float = 1e-10, inverses: bool = False):
    """Refinement whose corrections come from GMRES(m) preconditioned by the
    FP32 factors (reading R18; through their explicit FP64 inverses inside
    GMRES when ``inverses``, reading R27); stop rules as ``solve_ir``.
    Returns x, refinement steps, Arnoldi steps, converged flags and backward
    errors."""
    A32 = _f32(A32)
    LU = _f32(LU)
    n = A32.shape[0]
    b = np.array(b, dtype=np.float64, order="C", copy=True)
    if b.ndim == 1:
        b = b[:, None]
    nrhs = b.shape[1]
    if tol_b is None:
        tol_b = 2.0 ** -53 * np.sqrt(n)
    x = np.zeros((n, nrhs))
    iters = np.zeros(nrhs, dtype=np.int32)
    inner = np.zeros(nrhs, dtype=np.int32)
    conv = np.zeros(nrhs, dtype=np.int32)
    berr = np.zeros(nrhs)
    lib().orc_solve_gmres_ir(n, nrhs, _p(A32), n, _p(LU), n,
                             _p(np.ascontiguousarray(ipiv, np.int32)), _p(b), nrhs, _p(x), nrhs,
                             int(max_iter), float(tol), float(tol_b), float(stall), int(m),
                             float(tau), int(bool(inverses)), _p(iters), _p(inner), _p(conv),
                             _p(berr))
    return x, iters, inner, conv, berr
