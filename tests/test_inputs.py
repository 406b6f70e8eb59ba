"""The synthetic generators produce what they promise (shapes, conditioning)."""
import numpy as np
import pytest

import bfx_inputs as bi


@pytest.mark.parametrize("gen", [bi.svd_system, bi.fast_system])
@pytest.mark.parametrize("kappa", [1e1, 1e4, 1e8])
def test_condition_number(gen, kappa):
    P = gen(120, kappa, 3, nrhs=2)
    s = np.linalg.svd(P.A32.astype(np.float64), compute_uv=False)
    assert abs(np.log10(s[0] / s[-1]) - np.log10(kappa)) < 0.05
    assert P.b.shape == (120, 2)
    assert np.allclose(P.A32.astype(np.float64) @ P.x_true, P.b)


def test_wide_range_exponents():
    x = bi.wide_range(100000, 1)
    e = np.frexp(x)[1]
    assert e.min() >= -30 and e.max() <= 9
    assert np.all(np.abs(x) <= 2.0 ** 8)


def test_serving_stream_distributions():
    reqs = bi.serving_stream(20000, 0)
    t = np.array([r.t_arrival for r in reqs])
    assert abs(np.mean(np.diff(t)) - 1 / 5000) < 2e-5
    n = np.array([r.n for r in reqs])
    assert n.min() >= 64 and n.max() <= 4096
    assert abs(np.mean(np.log(n)) - (np.log(64) + np.log(4097)) / 2) < 0.05
    nr = np.array([r.nrhs for r in reqs])
    assert nr.min() == 1 and nr.max() == 16


def test_exponent_generators():
    import bfx_inputs as bi

    x = bi.random_exponent((400, 400), 1)
    e = ((x.view(np.uint32) >> 23) & 0xFF).astype(np.int64)
    assert x.dtype == np.float32 and np.all(np.isfinite(x))
    assert e.min() - 127 == -60 and e.max() - 127 == 60  # the full range is drawn
    assert abs(np.mean(x < 0) - 0.5) < 0.01
    g = bi.gaussian_exponent((400, 400), 2)
    eg = ((g.view(np.uint32) >> 23) & 0xFF).astype(np.int64) - 127
    assert abs(np.std(eg) - 10.0) < 0.2 and abs(np.mean(eg)) < 0.2
    assert np.array_equal(x, bi.random_exponent((400, 400), 1))
