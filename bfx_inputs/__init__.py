"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and builds test problems; it holds none
of the split/product/LU/refinement arithmetic of the method, so that the CUDA
library and the CPU oracle can both be fed the same inputs without sharing any
of the code under test.

Workloads (all numpy ``default_rng(seed)``):

* ``uniform_pm1``: FP32 entries uniform in [-1, 1], the narrow-range GEMM
  case of Sec. IV-A (the paper draws with drand48 in [-1, 1]).
* ``wide_range``: FP32 entries u * 2**e, u uniform in [-1, 1], e an integer
  uniform in [emin, emax]; a controlled stand-in for the paper's wide
  exponent-range GEMM case of Sec. IV-A.
* ``svd_system``: A = U diag(sigma) V^T with U, V the Q factors of Householder
  QR of Gaussian matrices and sigma geometric from 1 down to 1/kappa, rounded
  to FP32 (the FP32 matrix *is* the problem), x_true Gaussian and
  b = A32 x_true evaluated in FP64.  Used for the solves of Sec. III/IV-B at
  prescribed condition numbers.
* ``batched_systems`` / ``serving_stream``: many independent systems of that
  kind with sizes, right-hand-side counts, conditioning and (for the stream)
  Poisson arrival times drawn from stated distributions.
* ``fast_system``: the same kind of system built in O(n^2): A = H1 H2 P1
  diag(sigma) P2^T H4 H3 with Householder reflectors H = I - 2 v v^T / v^T v
  of Gaussian v and random permutations P, so kappa(A) is exactly
  sigma_max / sigma_min; used for the serving stream, whose thousands of
  requests up to n = 4096 cannot each afford two QR factorisations.
* ``random_exponent`` / ``gaussian_exponent``: the wide and medium exponent
  ranges of Sec. IV-A's GEMM study: random sign and 23 mantissa bits with the
  exponent uniform over a range symmetric about 0 (the paper's "randomly chosen
  exponent bits", bounded so that products and their sums stay finite) or
  rounded from a Gaussian (its "medium range").
* ``diag_dominant_system``: row and column diagonally dominant unsymmetric
  matrices (off-diagonal U[-1,1], each diagonal entry of random sign and
  magnitude above both its row and its column sum of the other entries), the
  GMRES case of Sec. IV-B.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "uniform_pm1",
    "wide_range",
    "svd_system",
    "SolveProblem",
    "batched_systems",
    "serving_stream",
    "Request",
    "special_values_f32",
    "fast_system",
    "diag_dominant_system",
    "random_exponent",
    "gaussian_exponent",
]


def uniform_pm1(shape, seed: int) -> np.ndarray:
    """FP32 array, entries uniform in [-1, 1] (seeded)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)


def wide_range(shape, seed: int, emin: int = -8, emax: int = 8) -> np.ndarray:
    """FP32 array, entries u * 2**e with u ~ U[-1,1] (FP32) and e ~ U{emin..emax}.

    The scaling by a power of two is exact, so every entry is exactly the
    product of its two drawn factors.
    """
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)
    e = rng.integers(emin, emax + 1, size=shape)
    return np.ldexp(u, e).astype(np.float32)


def special_values_f32() -> np.ndarray:
    """A fixed set of FP32 edge cases (zeros, subnormals, extremes, Inf, NaN, ties)."""
    bits = [
        0x00000000, 0x80000000,  # +-0
        0x00000001, 0x80000001,  # smallest subnormals
        0x007FFFFF, 0x00400000, 0x00008000, 0x00018000,  # subnormals incl. ties
        0x00800000, 0x00800001, 0x00808000, 0x00818000,  # smallest normals, ties
        0x0C800000, 0x0C8FFFFF, 0x0CFFFFFF,  # around 2^-102 .. 2^-101
        0x08800000, 0x088FFFFF,  # around 2^-110
        0x3F800000, 0x3F808000, 0x3F818000, 0x3F80FFFF, 0x3F7FFFFF,  # around 1
        0xBF808000, 0xBF818000, 0xBF7FFFFF,
        0x7F7F0000, 0x7F7F7FFF, 0x7F7F8000, 0x7F7FFFFF,  # top of the range
        0xFF7F8000, 0xFF7FFFFF,
        0x7F800000, 0xFF800000,  # +-Inf
        0x7FC00000, 0xFFC00001, 0x7F800001, 0x7FBFFFFF,  # NaNs (quiet, signalling)
        0x00C0FFFF,  # the "bad number" shape of Sec. II-F (small exponent, low bits set)
    ]
    return np.array(bits, dtype=np.uint32).view(np.float32)


def _haar_like_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Q factor (FP64) of a Householder QR of an n x n standard Gaussian matrix."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    # fix the sign convention so Q does not depend on LAPACK's choice of signs
    q *= np.sign(np.diag(r))[None, :]
    return q


@dataclass
class SolveProblem:
    """One dense system A32 x = b.  A32 is FP32 (the problem matrix itself)."""

    A32: np.ndarray  # (n, n) float32, row-major
    b: np.ndarray  # (n, nrhs) float64
    x_true: np.ndarray  # (n, nrhs) float64
    kappa_nominal: float
    seed: int

    @property
    def n(self) -> int:
        return self.A32.shape[0]

    @property
    def nrhs(self) -> int:
        return self.b.shape[1]


_UV_CACHE = {}


def _orthogonal_pair(n: int, seed: int):
    """U, V of svd_system (two QRs of Gaussians from the seed) and the
    generator's state after them; large pairs are kept for reuse, so the
    four condition numbers of one size and seed cost two QRs, not eight."""
    key = (n, seed)
    if key in _UV_CACHE:
        U, V, state = _UV_CACHE[key]
        rng = np.random.default_rng()
        rng.bit_generator.state = state
        return U, V, rng
    rng = np.random.default_rng(seed)
    U = _haar_like_orthogonal(n, rng)
    V = _haar_like_orthogonal(n, rng)
    if n >= 1024:
        _UV_CACHE.clear()  # at most one large pair at a time
        _UV_CACHE[key] = (U, V, rng.bit_generator.state)
    return U, V, rng


def svd_system(n: int, kappa: float, seed: int, nrhs: int = 1) -> SolveProblem:
    """A = U diag(sigma) V^T, sigma_i = kappa**(-i/(n-1)), rounded to FP32.

    b = A32 @ x_true is evaluated in FP64 from the FP32 matrix, so x_true is the
    exact solution of the FP32 problem up to the FP64 rounding of b.
    """
    U, V, rng = _orthogonal_pair(n, seed)
    if n > 1:
        sigma = kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))
    else:
        sigma = np.ones(1)
    A64 = (U * sigma[None, :]) @ V.T
    A32 = np.ascontiguousarray(A64.astype(np.float32))
    x_true = rng.standard_normal((n, nrhs))
    b = A32.astype(np.float64) @ x_true
    return SolveProblem(A32=A32, b=b, x_true=x_true, kappa_nominal=float(kappa), seed=seed)


def batched_systems(count: int, seed: int, n_lo: int = 32, n_hi: int = 512,
                    log10k_lo: float = 2.0, log10k_hi: float = 8.0):
    """Many independent systems: n ~ U{n_lo..n_hi}, log10(kappa) ~ U[lo, hi], nrhs = 1."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    lk = rng.uniform(log10k_lo, log10k_hi, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [svd_system(int(n), float(10.0 ** k), int(s)) for n, k, s in zip(ns, lk, seeds)]


def batched_sizes(count: int, seed: int, n_lo: int = 32, n_hi: int = 512):
    """Only the size list of ``batched_systems`` (same draws), for cost estimates."""
    rng = np.random.default_rng(seed)
    return rng.integers(n_lo, n_hi + 1, size=count)


@dataclass
class Request:
    """One solve request of the serving stream."""

    t_arrival: float  # seconds from stream start
    n: int
    nrhs: int
    log10_kappa: float
    seed: int


def serving_stream(count: int, seed: int, rate: float = 5000.0, n_lo: int = 64,
                   n_hi: int = 4096, nrhs_hi: int = 16, log10k_lo: float = 1.0,
                   log10k_hi: float = 10.0):
    """Poisson arrivals (exponential gaps of mean 1/rate) with mixed sizes.

    n is log-uniform in [n_lo, n_hi] (rounded down to an integer), nrhs is
    uniform in {1..nrhs_hi}, log10(kappa) is uniform in [lo, hi].
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi + 1), size=count))).astype(int)
    ns = np.clip(ns, n_lo, n_hi)
    nr = rng.integers(1, nrhs_hi + 1, size=count)
    lk = rng.uniform(log10k_lo, log10k_hi, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [Request(float(a), int(b), int(c), float(d), int(e))
            for a, b, c, d, e in zip(t, ns, nr, lk, seeds)]


def _apply_reflector_left(X: np.ndarray, v: np.ndarray) -> None:
    X -= np.outer(v, (2.0 / (v @ v)) * (v @ X))


def _apply_reflector_right(X: np.ndarray, v: np.ndarray) -> None:
    X -= np.outer((2.0 / (v @ v)) * (X @ v), v)


def fast_system(n: int, kappa: float, seed: int, nrhs: int = 1) -> SolveProblem:
    """A = H1 H2 P1 diag(sigma) P2^T H4 H3 (see the module docstring), FP32."""
    rng = np.random.default_rng(seed)
    sigma = kappa ** (-np.arange(n, dtype=np.float64) / (n - 1)) if n > 1 else np.ones(1)
    p1, p2 = rng.permutation(n), rng.permutation(n)
    X = np.zeros((n, n))
    X[p1, p2] = sigma
    for _ in range(2):
        _apply_reflector_left(X, rng.standard_normal(n))
    for _ in range(2):
        _apply_reflector_right(X, rng.standard_normal(n))
    A32 = np.ascontiguousarray(X.astype(np.float32))
    x_true = rng.standard_normal((n, nrhs))
    b = A32.astype(np.float64) @ x_true
    return SolveProblem(A32=A32, b=b, x_true=x_true, kappa_nominal=float(kappa), seed=seed)


def diag_dominant_system(n: int, seed: int, nrhs: int = 1, margin: float = 1.0) -> SolveProblem:
    """Row and column diagonally dominant A (FP32), x_true Gaussian, b = A32 x_true (FP64).

    Off-diagonal entries U[-1, 1]; |a_ii| = max(row sum, column sum of the
    other |a_ij|) + margin * U[0, 1], with a random sign.
    """
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(n, n))
    np.fill_diagonal(A, 0.0)
    dom = np.maximum(np.abs(A).sum(axis=1), np.abs(A).sum(axis=0))
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    np.fill_diagonal(A, sign * (dom + margin * rng.random(n)))
    A32 = np.ascontiguousarray(A.astype(np.float32))
    x_true = rng.standard_normal((n, nrhs))
    b = A32.astype(np.float64) @ x_true
    return SolveProblem(A32=A32, b=b, x_true=x_true, kappa_nominal=float("nan"), seed=seed)


def _compose_f32(rng, shape, e):
    """FP32 values with random sign, random 23-bit mantissa and exponent e (int array)."""
    sign = rng.integers(0, 2, size=shape).astype(np.uint32) << 31
    mant = rng.integers(0, 1 << 23, size=shape).astype(np.uint32)
    bits = sign | ((e.astype(np.int64) + 127).astype(np.uint32) << 23) | mant
    return bits.view(np.float32)


def random_exponent(shape, seed: int, emin: int = -60, emax: int = 60) -> np.ndarray:
    """FP32 normal numbers whose exponent is uniform in [emin, emax]."""
    rng = np.random.default_rng(seed)
    e = rng.integers(emin, emax + 1, size=shape)
    return _compose_f32(rng, shape, e)


def gaussian_exponent(shape, seed: int, sigma: float = 10.0, emax: int = 60) -> np.ndarray:
    """FP32 normal numbers whose exponent is a rounded N(0, sigma^2), clipped to +-emax."""
    rng = np.random.default_rng(seed)
    e = np.clip(np.rint(rng.normal(0.0, sigma, size=shape)), -emax, emax).astype(np.int64)
    return _compose_f32(rng, shape, e)
