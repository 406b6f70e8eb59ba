"""Device dot_bf16xN against the oracle: exact-rational bound checks and the
FP64 product (Sec. II-B..II-G); FP32 mode against Sec. II-C's bound."""
from fractions import Fraction as F

import numpy as np
import pytest
import torch

import bfx_inputs as bi
from _tol import tol

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1, 3, 6, 8, 9])
@pytest.mark.parametrize("n", [1, 7, 1000, 4099, 1 << 20])
def test_dot_bound_vs_fp64(bfx, orc, mode, n):
    x = bi.wide_range(n, 3 * n + mode, -12, 12)
    y = bi.wide_range(n, 3 * n + mode + 1, -12, 12)
    got = float(bfx.dot_bf16xN(mode, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).item())
    z64, zabs = orc.dgemm_rows(x[None, :], y[:, None])
    z64, zabs = float(z64[0, 0]), float(zabs[0, 0])
    assert abs(got - z64) <= tol(mode, n) * zabs + 1e-38
    # element by element against the oracle's sequential model of the same mode
    assert abs(got - float(orc.dot(mode, x, y))) <= 2 * tol(mode, n) * zabs + 1e-38


def test_dot_exact_cases(bfx, orc):
    """Exactly representable sums: x = pieces-friendly integers, result exact."""
    n = 3000
    rng = np.random.default_rng(1)
    x = rng.integers(-64, 65, n).astype(np.float32)
    y = rng.integers(-64, 65, n).astype(np.float32)
    exact = float(sum(F(int(a)) * F(int(b)) for a, b in zip(x, y)))
    for mode in (0, 1, 3, 6, 8, 9):
        got = float(bfx.dot_bf16xN(mode, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).item())
        assert got == exact


def test_dot_x6_more_accurate_than_x3(bfx, orc):
    n = 1 << 16
    x, y = bi.uniform_pm1(n, 5), bi.uniform_pm1(n, 6)
    z64, _ = orc.dgemm_rows(x[None, :], y[:, None])
    e = {}
    for mode in (3, 6):
        got = float(bfx.dot_bf16xN(mode, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).item())
        e[mode] = abs(got - z64[0, 0])
    assert e[6] < e[3]


def test_dot_empty(bfx):
    x = torch.empty(0, device="cuda")
    assert float(bfx.dot_bf16xN(6, x, x).item()) == 0.0
