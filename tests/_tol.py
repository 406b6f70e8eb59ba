"""Elementwise error bounds used by the GPU parity tests.

|C - C64|_ij <= tol(mode, k) * (|A||B|)_ij + ulp-level slack, where C64 is the
FP64 product of the FP32 inputs (the oracle's plain definition).

* x6 / x9: 2 max(k, 2) 2^-24 (the stated tolerance 2 k 2^-24, with k >= 2 so
  that k = 1 still covers the final FP32 rounding plus the dropped 2^-24 bin,
  whose size Sec. II-G bounds by (513/512) 2^-23 |a0 b0|).
* x3: the pair split drops the 2^-16 bin and below: 3 products each at most
  2^-16 |a0||b0| <= 2^-16 (1 + 2^-8)^2 |a||b|, so 3.03 2^-16, plus the
  accumulation term of x6.
* x5 (A in two pieces, B in three, Sec. II-G): A's dropped third piece,
  |a2| <= 2^-16 |a|, plus a1 b2 (<= 1.01 2^-24): 1.01 2^-16 plus the
  accumulation term.
* x1: one piece each, |ab - a0 b0| <= (2 + 2^-8) 2^-8 |a||b|: 2.01 2^-8 plus the
  accumulation term.
* FP32 SIMT: gamma_k = k 2^-24 / (1 - k 2^-24) (Sec. II-C).
"""
import numpy as np

EPS = 2.0 ** -24


def acc_term(k):
    return 2 * max(k, 2) * EPS


def tol(mode, k):
    if mode == 0:
        return k * EPS / (1 - k * EPS)
    if mode in (6, 8, 9):
        return acc_term(k)
    if mode == 3:
        return 3.03 * 2.0 ** -16 + acc_term(k)
    if mode == 5:
        return 1.01 * 2.0 ** -16 + acc_term(k)
    if mode == 1:
        return 2.01 * 2.0 ** -8 + acc_term(k)
    raise ValueError(mode)


def check_bound(C, C64, Cabs, mode, k, alpha=1.0, Cin=None, beta=0.0):
    """Assert the elementwise bound; returns the max ratio error / bound."""
    C = np.asarray(C, np.float64)
    ref = alpha * C64
    bnd = tol(mode, k) * abs(alpha) * Cabs
    if Cin is not None and beta != 0.0:
        ref = ref + beta * np.asarray(Cin, np.float64)
        bnd = bnd + EPS * np.abs(ref) + EPS * abs(beta) * np.abs(Cin)  # rounding of the update
    bnd = bnd + np.finfo(np.float32).tiny
    err = np.abs(C - ref)
    r = err / bnd
    worst = float(np.max(r)) if r.size else 0.0
    assert worst <= 1.0, (mode, k, worst, np.unravel_index(np.argmax(r), r.shape))
    return worst
