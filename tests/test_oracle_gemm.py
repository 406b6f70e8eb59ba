"""Pins of the oracle's partial products, level sums and combinations
(Sec. II-B .. II-G) and of its FP64 reference product.

Expected values come from exact rational arithmetic (Python fractions), from
permutation special cases whose result is known exactly, from the paper's
error bounds and stated accuracy orderings, never from the oracle itself.
"""
import os
from fractions import Fraction as F

import numpy as np
import pytest

import bfx_inputs as bi

EPS_F = 2.0**-24  # unit roundoff of FP32 (Sec. II-B)
EPS_B = 2.0**-8  # of bfloat16


def gam(k):
    return k * EPS_F / (1 - k * EPS_F)


def _pieces(orc, x, npieces=3):
    return [orc.bf16_to_f32(p) for p in orc.split(np.asarray(x, np.float32), npieces)]


def _perm_matrix(perm):
    n = len(perm)
    P = np.zeros((n, n), np.float32)
    P[np.arange(n), perm] = 1.0
    return P


# ----------------------------------------------------------------- exact cases
@pytest.mark.parametrize("mode", [1, 3, 5, 6, 8, 9])
def test_left_permutation_exact(orc, mode):
    """C = P B with P a permutation: every row of C is exactly the sum of the
    pieces of a row of B that the mode keeps (products (0,j))."""
    rng = np.random.default_rng(1)
    n = 24
    perm = rng.permutation(n)
    B = bi.wide_range((n, 17), 2, -20, 20)
    C = orc.gemm(mode, _perm_matrix(perm), B)
    b0, b1, b2 = _pieces(orc, B)
    expect = {1: b0, 3: b0 + b1, 5: B, 6: B, 8: B, 9: B}[mode][perm]
    assert np.array_equal(C, expect)


@pytest.mark.parametrize("mode", [1, 3, 5, 6, 8, 9])
def test_right_permutation_exact(orc, mode):
    """C = A Q: every column of C is exactly the kept pieces of a column of A
    (products (i,0)); catches a transposed operand or a dropped (i,0) term."""
    rng = np.random.default_rng(3)
    n = 20
    perm = rng.permutation(n)
    Q = _perm_matrix(perm).T  # Q[perm[j], j] = 1
    A = bi.wide_range((13, n), 4, -20, 20)
    C = orc.gemm(mode, A, Q)
    a0, a1, a2 = _pieces(orc, A)
    # x5 splits A in two pieces only (Sec. II-G's asymmetric case)
    expect = {1: a0, 3: a0 + a1, 5: a0 + a1, 6: A, 8: A, 9: A}[mode][:, perm]
    assert np.array_equal(C, expect)


def test_single_products_exact_in_fp32(orc):
    """Sec. I: a bfloat16 x bfloat16 product is exact in FP32, so with one term
    each partial product Z^(i,j) equals the exact product of pieces i and j."""
    rng = np.random.default_rng(5)
    for t in range(300):
        x = bi.wide_range(1, 100 + t, -40, 40)
        y = bi.wide_range(1, 1000 + t, -40, 40)
        Z = orc.dot_partials(x, y)
        xp = [F(float(v[0])) for v in _pieces(orc, x)]
        yp = [F(float(v[0])) for v in _pieces(orc, y)]
        for i in range(3):
            for j in range(3):
                assert F(float(Z[i, j])) == xp[i] * yp[j], (t, i, j)


def test_already_bfloat16_inputs_all_modes_equal(orc):
    """Inputs that are bfloat16 values have zero mid/lo pieces: x3/x6/x8/x9 == x1."""
    A = orc.bf16_to_f32(orc.bf16_rne(bi.uniform_pm1((32, 40), 6)))
    B = orc.bf16_to_f32(orc.bf16_rne(bi.uniform_pm1((40, 24), 7)))
    C1 = orc.gemm(1, A, B)
    for mode in (3, 6, 8, 9):
        assert np.array_equal(orc.gemm(mode, A, B), C1)


# ----------------------------------------------------------------- bounds vs exact
def _exact_dot(x, y):
    z = sum(F(float(a)) * F(float(b)) for a, b in zip(x, y))
    zh = sum(abs(F(float(a)) * F(float(b))) for a, b in zip(x, y))
    return z, zh


@pytest.mark.parametrize("gen", ["uniform", "wide", "cancel"])
def test_bounds_against_exact_sums(orc, gen):
    """Sec. II-C: |Z - z| <= gamma_n zhat for FP32.  Sec. II-E: |Z_2 - z| <=
    1.01 (gamma_{n+2} + eps_b^3) zhat for x6 (eps_b^3 = 2^-24).  x9 keeps every
    term: 1.01 gamma_{n+4} zhat.  x3 drops the 2^-16 bin and below:
    3.03 * 2^-16 zhat + 1.01 gamma_{n+1} zhat."""
    rng = np.random.default_rng({"uniform": 8, "wide": 9, "cancel": 10}[gen])
    worst = {m: 0.0 for m in (0, 3, 6, 9)}
    for t in range(60):
        k = int(rng.integers(1, 48))
        if gen == "uniform":
            x, y = bi.uniform_pm1(k, 2 * t), bi.uniform_pm1(k, 2 * t + 1)
        elif gen == "wide":
            x, y = bi.wide_range(k, 2 * t, -30, 30), bi.wide_range(k, 2 * t + 1, -30, 30)
        else:  # heavy cancellation: x, -x pairs
            h = bi.uniform_pm1((k + 1) // 2, 3 * t)
            x = np.concatenate([h, h])[:k].astype(np.float32)
            y = np.concatenate([bi.uniform_pm1((k + 1) // 2, 3 * t + 1)] * 2)[:k]
            y[(k + 1) // 2:] *= -1
        z, zh = _exact_dot(x, y)
        bound = {0: gam(k), 6: 1.01 * (gam(k + 2) + EPS_F), 9: 1.01 * gam(k + 4),
                 3: 3.03 * 2.0**-16 + 1.01 * gam(k + 1)}
        for m in (0, 3, 6, 9):
            Z = orc.dot(m, x, y)
            err = abs(F(float(Z)) - z)
            if zh == 0:
                assert err == 0
                continue
            r = float(err / zh) / bound[m]
            worst[m] = max(worst[m], r)
    for m, r in worst.items():
        assert r <= 1.0, (m, r)


def test_z0_exactness_condition(orc):
    """Sec. II-E: when the hi*hi products fit one FP32 accumulator, Z^(0) = z^(0)
    and |Z_2 - z| <= 1.01 (gamma_2 + eps_b^3) zhat <= 1.01 gamma_3 zhat.

    The printed condition compares max|x y| with min|x y|; the text bounds the
    sum by n max|x y|, and the condition is applied here with that factor n
    (without it the condition is not sufficient: it admits counterexamples)."""
    rng = np.random.default_rng(11)
    used = 0
    for t in range(800):
        k = int(rng.integers(2, 64))
        e = int(rng.integers(0, 4))
        x = (rng.uniform(1, 2, k) * 2.0 ** rng.integers(-e, e + 1, k) * rng.choice([-1, 1], k)).astype(np.float32)
        y = (rng.uniform(1, 2, k) * 2.0 ** rng.integers(-e, e + 1, k) * rng.choice([-1, 1], k)).astype(np.float32)
        p = np.abs(x.astype(np.float64) * y)
        if np.ceil(np.log2(1.01 * k * p.max())) - 23 > np.ceil(np.log2(0.99 * p.min())) - 15:
            continue
        used += 1
        Z = orc.dot_partials(x, y)
        x0, y0 = _pieces(orc, x)[0], _pieces(orc, y)[0]
        z0, _ = _exact_dot(x0, y0)
        assert F(float(Z[0, 0])) == z0
        z, zh = _exact_dot(x, y)
        Z2 = orc.dot(6, x, y)
        assert float(abs(F(float(Z2)) - z) / zh) <= 1.01 * gam(3)
    assert used > 200


# ----------------------------------------------------------------- matrices
@pytest.fixture(scope="module")
def c1_case(orc):
    A = bi.uniform_pm1((256, 256), 0)
    B = bi.uniform_pm1((256, 256), 1)
    C64, Cabs = orc.dgemm_rows(A, B)
    return A, B, C64, Cabs


def test_dgemm_rows_reference(orc, c1_case):
    """The FP64 product against exact rationals on sampled entries."""
    A, B, C64, Cabs = c1_case
    for i, j in [(0, 0), (3, 200), (255, 17), (128, 255)]:
        z, zh = _exact_dot(A[i], B[:, j])
        assert abs(F(C64[i, j]) - z) <= 256 * 2.0**-53 * zh
        assert abs(F(Cabs[i, j]) - zh) <= 256 * 2.0**-53 * zh


def test_c1_bounds(orc, c1_case):
    """Config 256^3 uniform[-1,1]: elementwise bounds of Sec. II-C/II-E and the
    stated GPU tolerance 2 k 2^-24 |A||B| for x6/x9 hold for the FMA model."""
    A, B, C64, Cabs = c1_case
    k = A.shape[1]
    ratios = {}
    for m, bnd in [(0, gam(k)), (6, 1.01 * (gam(k + 2) + EPS_F)), (9, 1.01 * gam(k + 4)),
                   (8, 1.01 * (gam(k + 3) + 2.0**-32)),  # drops only the lo*lo bin, <= 2^-32 zhat
                   (3, 3.03 * 2.0**-16 + 1.01 * gam(k + 1))]:
        C = orc.gemm(m, A, B)
        r = np.max(np.abs(C - C64) / (bnd * Cabs))
        ratios[m] = r
        assert r <= 1.0, (m, r)
    for m in (6, 8, 9):
        C = orc.gemm(m, A, B)
        assert np.all(np.abs(C - C64) <= 2 * k * EPS_F * Cabs)


def test_e1_accuracy_order(orc):
    """Sec. IV-A, narrow range [-1,1]: the order of accuracy is bx2_3 (x3),
    SGEMM, bx3_6 (x6), bx3_6d (x6 collected in FP64), least to most accurate,
    in average relative Frobenius error against the FP64 product."""
    errs = {"x3": [], "sgemm": [], "x6": [], "x6d": []}
    for s in range(6):
        A = bi.uniform_pm1((192, 192), 100 + 2 * s)
        B = bi.uniform_pm1((192, 192), 101 + 2 * s)
        C64, _ = orc.dgemm_rows(A, B)
        nrm = np.linalg.norm(C64)
        errs["x3"].append(np.linalg.norm(orc.gemm(3, A, B) - C64) / nrm)
        errs["sgemm"].append(np.linalg.norm(orc.gemm(0, A, B) - C64) / nrm)
        errs["x6"].append(np.linalg.norm(orc.gemm(6, A, B) - C64) / nrm)
        errs["x6d"].append(np.linalg.norm(orc.gemm_f64out(6, A, B) - C64) / nrm)
    e = {k: np.mean(v) for k, v in errs.items()}
    assert e["x3"] > e["sgemm"] > e["x6"] > e["x6d"], e


def test_e2_wide_range_comparable(orc):
    """Sec. IV-A: with a wide exponent range x6 and SGEMM errors are "very
    comparable" (within a factor 2 here, for e in [-8, 8])."""
    A = bi.wide_range((192, 192), 40)
    B = bi.wide_range((192, 192), 41)
    C64, _ = orc.dgemm_rows(A, B)
    nrm = np.linalg.norm(C64)
    es = np.linalg.norm(orc.gemm(0, A, B) - C64) / nrm
    e6 = np.linalg.norm(orc.gemm(6, A, B) - C64) / nrm
    assert 0.5 < e6 / es < 2.0, (e6, es)


def test_alpha_beta_form(orc):
    """C = alpha Z + beta C (reading R13): alpha = -1, beta = 1 gives the
    correctly rounded difference C - Z (the LU trailing update)."""
    A = bi.uniform_pm1((40, 33), 50)
    B = bi.uniform_pm1((33, 29), 51)
    C0 = bi.uniform_pm1((40, 29), 52)
    for m in (0, 3, 6):
        Z = orc.gemm(m, A, B)
        D = orc.gemm(m, A, B, alpha=-1.0, beta=1.0, C=C0)
        assert np.array_equal(D, (C0.astype(np.float64) - Z).astype(np.float32))
        D2 = orc.gemm(m, A, B, alpha=2.0, beta=0.0, C=np.full_like(C0, np.nan))
        assert np.array_equal(D2, 2 * Z)  # beta = 0 does not read C


def test_worked_example_a1b2(orc):
    """Sec. II-G example x = 0.578921..., y = -7447.659...: because |y| >> |x|,
    the 2^-24-bin term a1*b2 is the significant one of its bin, and adding it
    to the six products brings the (exact-sum) error down.  Partially pinned:
    the paper's surrounding sentence is garbled (see the design notes)."""
    x = np.float32(0.57892173110418099213)
    y = np.float32(-7447.6596637651937272)
    assert int(np.array(x).view(np.uint32)) == 0x3F143437
    assert int(np.array(y).view(np.uint32)) == 0xC5E8BD47
    a = [F(float(v[0])) for v in _pieces(orc, [x])]
    b = [F(float(v[0])) for v in _pieces(orc, [y])]
    assert sum(a) == F(float(x)) and sum(b) == F(float(y))
    ex = F(float(x)) * F(float(y))
    six = sum(a[i] * b[j] for i in range(3) for j in range(3) if i + j <= 2)
    assert abs(a[1] * b[2]) > 4 * abs(a[2] * b[1])
    assert abs(six + a[1] * b[2] - ex) < abs(six - ex) / 3


def test_x8_keeps_exactly_the_z3_bin(orc):
    """Sec. II-D's Z3 sum (x8) adds the 2^-24 bin {12, 21} to x6.  With
    x = [a, -a] and y = [b, b0 + b1] every piece product cancels except those
    with b's lo piece: Z^(i,2) = a_i b2, so x6 = a0 b2 (exact), x8 =
    fl32(a0 b2 + a1 b2) and x9 additionally adds a2 b2."""
    rng = np.random.default_rng(17)
    checked = 0
    for t in range(400):
        a = np.float32(rng.uniform(-1, 1))
        b = np.float32(rng.uniform(-1, 1) * 2.0 ** rng.integers(-5, 6))
        a0, a1, a2 = (float(v[0]) for v in _pieces(orc, np.array([a])))
        b0, b1, b2 = (float(v[0]) for v in _pieces(orc, np.array([b])))
        c = np.float32(b0 + b1)
        p = [float(v[0]) for v in _pieces(orc, np.array([c]))]
        if p != [b0, b1, 0.0] or b2 == 0.0 or a1 == 0.0:
            continue  # only inputs whose truncated value splits as (b0, b1, 0)
        checked += 1
        x = np.array([[a, -a]], dtype=np.float32)
        y = np.array([[b], [c]], dtype=np.float32)
        x6 = float(orc.gemm(6, x, y)[0, 0])
        x8 = float(orc.gemm(8, x, y)[0, 0])
        assert F(x6) == F(a0) * F(b2), t
        assert x8 == float(np.float32(a0 * b2) + np.float32(a1 * b2)), t
    assert checked > 100


# ----------------------------------------------------------------- asymmetric split
def _sixteen_bit(shape, seed):
    """FP32 values with at most 16 significant bits: their third piece is 0."""
    x = bi.uniform_pm1(shape, seed)
    return (x.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)


def test_x5_equals_x6_when_a_has_sixteen_bits(orc):
    """Sec. II-G's 2 x 3 split keeps {00,01,10,02,11}; x6 adds a2 b0.  When A
    has at most 16 significant bits a2 = 0, so the two modes must agree
    exactly: a dropped or misplaced 02 / 11 term breaks the equality."""
    A = _sixteen_bit((40, 56), 70)
    assert not np.any(_pieces(orc, A)[2])
    B = bi.wide_range((56, 33), 71, -12, 12)
    C5 = orc.gemm(5, A, B)
    assert np.array_equal(C5, orc.gemm(6, A, B))
    assert not np.array_equal(C5, orc.gemm(3, A, B))
    assert np.array_equal(orc.gemm_f64out(5, A, B), orc.gemm_f64out(6, A, B))


def test_x5_accuracy_bounded_by_the_missing_third_piece(orc):
    """Sec. II-G: with A in two pieces, the 2^-16 bin's two products cannot
    bring the result to FP32 accuracy: A's dropped remainder a2 (|a2| <=
    2^-16 |a|) bounds the error, |C - C64| <= (1.01 2^-16 + 2 k 2^-24)
    (|A||B|), and the relative error stays far above x6's (>= 10x), while the
    extra products make it smaller than x3's."""
    k = 96
    A = bi.uniform_pm1((64, k), 72)
    B = bi.uniform_pm1((k, 48), 73)
    C64 = A.astype(np.float64) @ B.astype(np.float64)
    Cabs = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    e = {}
    for mode in (3, 5, 6):
        C = orc.gemm(mode, A, B).astype(np.float64)
        e[mode] = np.linalg.norm(C - C64) / np.linalg.norm(C64)
        if mode == 5:
            bound = (1.01 * 2.0**-16 + 2 * k * EPS_F) * Cabs
            assert np.all(np.abs(C - C64) <= bound)
    assert e[5] >= 10 * e[6], e
    assert e[5] < e[3], e


ORDER_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "combine_order.txt")


def _bits_f32(words):
    return np.array([int(w, 16) for w in words], dtype=np.uint32).view(np.float32)


def _order_golden():
    rows = []
    for line in open(ORDER_GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, a, b, exp, wrong = (f.strip() for f in line.split("|"))
        expected = {int(m): int(v, 16) for m, v in (t.split(":") for t in exp.split())}
        w6, w9 = (int(v, 16) for v in wrong.split())
        rows.append((name, _bits_f32(a.split()), _bits_f32(b.split()), expected, w6, w9))
    return rows


@pytest.mark.parametrize("row", _order_golden(), ids=lambda r: r[0])
def test_combination_order_golden(orc, row):
    """Sec. II-D's smallest-first combination, pinned by hand-worked cases
    (tests/golden/combine_order.txt) in which another order gives another
    FP32 result: G1 separates Z0 + (Z1 + Z2) from (Z0 + Z1) + Z2; G2 is the
    x9 chain, where Z4 tips a double tie that x8, x6 and a left-to-right x9
    round the other way."""
    name, a, b, expected, wrong6, wrong9 = row
    for mode, want in expected.items():
        C = orc.gemm(mode, a[None, :], b[:, None])
        assert int(C.view(np.uint32)[0, 0]) == want, (name, mode, hex(int(C.view(np.uint32)[0, 0])))
        assert int(np.float32(orc.dot(mode, a, b)).view(np.uint32)) == want
    # the other orders, evaluated in FP32 from the oracle's own partial
    # products, give the golden's "wrong order" values, which differ
    Z = orc.dot_partials(a, b).astype(np.float32)
    f = np.float32
    Z0, Z1 = Z[0, 0], f(Z[0, 1] + Z[1, 0])
    Z2 = f(Z[0, 2] + f(Z[1, 1] + Z[2, 0]))
    Z3, Z4 = f(Z[1, 2] + Z[2, 1]), Z[2, 2]
    ltr6 = f(f(Z0 + Z1) + Z2)
    ltr9 = f(f(f(f(Z0 + Z1) + Z2) + Z3) + Z4)
    assert int(ltr6.view(np.uint32)) == wrong6 and int(ltr9.view(np.uint32)) == wrong9
    assert expected[9] != wrong9
    if name == "G1":
        assert expected[6] != wrong6
    if name == "G2":
        assert expected[9] != expected[8]  # the lo*lo bin decides


def test_combination_order_golden_partials_g2(orc):
    """G2 has k = 1, so each partial product is an exact product of pieces;
    the values worked out by hand in the golden file."""
    row = [r for r in _order_golden() if r[0] == "G2"][0]
    Z = orc.dot_partials(row[1], row[2]).astype(np.float64)
    want = [[F(19781, 2**14), F(-15589, 2**22), F(-3537, 2**29)],
            [F(-453, 2**20), F(357, 2**28), F(81, 2**35)],
            [F(-151, 2**27), F(119, 2**35), F(27, 2**42)]]
    for i in range(3):
        for j in range(3):
            assert F(float(Z[i, j])) == want[i][j], (i, j)
