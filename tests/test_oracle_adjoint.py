"""Pins of the oracle's differentiable form: the forward with unit weights
and integer data equals the integer dedispersion; <A x, g> = <x, A^T g> to
FP64 rounding; the gradients of the MSE loss equal central finite
differences of the oracle's own FP64 loss."""
import numpy as np
import pytest


def _plan(oracle, C=24, T=600, D=7):
    pl = oracle.plan(C, 1400.0, -6.0, 64e-6, [(0.0, 20.0, D, 1)], T)[0]
    return pl


def test_unit_weights_equal_integer_dedispersion(oracle):
    rng = np.random.default_rng(21)
    pl = _plan(oracle)
    x = rng.integers(0, 256, (24, 600), dtype=np.uint8)
    y = oracle.forward_f64(x.astype(np.float64), np.ones(24), pl.shifts, pl.length)
    for d in range(pl.ndm):
        assert np.array_equal(y[d], oracle.dedisperse_row(x, pl.shifts[d], 0, pl.length))


def test_weights_scale_channels(oracle):
    """Weight c multiplies exactly channel c's contribution."""
    rng = np.random.default_rng(22)
    pl = _plan(oracle)
    x = rng.standard_normal((24, 600))
    w = np.zeros(24)
    w[5] = 2.5
    y = oracle.forward_f64(x, w, pl.shifts, pl.length)
    for d in range(pl.ndm):
        s = pl.shifts[d][5]
        assert np.allclose(y[d], 2.5 * x[5, s:s + pl.length], rtol=0, atol=1e-14)


def test_dot_product_identity(oracle):
    rng = np.random.default_rng(23)
    pl = _plan(oracle)
    x = rng.standard_normal((24, 600))
    w = rng.uniform(0.5, 1.5, 24)
    g = rng.standard_normal((pl.ndm, pl.length))
    lhs = float(np.sum(oracle.forward_f64(x, w, pl.shifts, pl.length) * g))
    gx, gw = oracle.adjoint_f64(x, w, pl.shifts, g)
    assert lhs == pytest.approx(float(np.sum(x * gx)), rel=1e-12)
    # <A_w x, g> is linear in w too: d/dw_c = gw[c]
    assert lhs == pytest.approx(float(np.dot(w, gw)), rel=1e-12)


def test_mse_gradient_finite_differences(oracle):
    rng = np.random.default_rng(24)
    pl = _plan(oracle, C=12, T=300, D=5)
    x = rng.standard_normal((12, 300))
    w = rng.uniform(0.5, 1.5, 12)
    T = rng.standard_normal((pl.ndm, pl.length))
    n = pl.ndm * pl.length
    y = oracle.forward_f64(x, w, pl.shifts, pl.length)
    gx, gw = oracle.adjoint_f64(x, w, pl.shifts, 2.0 * (y - T) / n)
    h = 1e-6
    for c in (0, 7, 11):
        wp, wm = w.copy(), w.copy()
        wp[c] += h
        wm[c] -= h
        fd = (oracle.mse_f64(x, wp, pl.shifts, pl.length, T)
              - oracle.mse_f64(x, wm, pl.shifts, pl.length, T)) / (2 * h)
        assert fd == pytest.approx(gw[c], rel=1e-6, abs=1e-9)
    for (c, t) in ((3, 10), (9, 250), (0, 299)):
        xp, xm = x.copy(), x.copy()
        xp[c, t] += h
        xm[c, t] -= h
        fd = (oracle.mse_f64(xp, w, pl.shifts, pl.length, T)
              - oracle.mse_f64(xm, w, pl.shifts, pl.length, T)) / (2 * h)
        assert fd == pytest.approx(gx[c, t], rel=1e-6, abs=1e-9)
