"""Pins for the oracle's k-sigma clipped statistics (robust mean and standard
deviation for the single-pulse search's SNR): scipy's iterative sigma clip,
hand cases at the inclusive bound, the plain moments when nothing is clipped,
and invariance under shifting and scaling the data."""
import numpy as np
import pytest

from paper_1912_07704_gb300 import abi
from paper_1912_07704_gb300.api import Plan


@pytest.mark.parametrize("seed,c16", [(1, 40), (2, 48), (3, 32), (4, 56)])
def test_matches_scipy_sigmaclip(oracle, seed, c16):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(seed)
    y = rng.normal(3000, 25, 40000).round().astype(np.int64)
    y[rng.integers(0, y.size, 400)] += rng.integers(100, 2000, 400)  # bright outliers
    y[rng.integers(0, y.size, 50)] -= 500
    mu, sg, kept = oracle.moments_clipped(y, c16, 1000)
    c, _, _ = stats.sigmaclip(y.astype(np.float64), c16 / 16, c16 / 16)
    assert kept == c.size
    assert mu == pytest.approx(c.mean(), rel=1e-13)
    assert sg == pytest.approx(c.std(), rel=1e-10)


def test_no_passes_is_plain(oracle):
    y = np.random.default_rng(5).integers(0, 5000, 3001)
    assert oracle.moments_clipped(y, 48, 0)[:2] == oracle.moments(y)
    # and a bound no sample reaches clips nothing
    g = np.random.default_rng(6).normal(0, 10, 5000).round().astype(np.int64)
    mu, sg, kept = oracle.moments_clipped(g, 255, 10)
    assert kept == g.size and (mu, sg) == pytest.approx(oracle.moments(g), rel=1e-15)


def test_inclusive_bound_hand(oracle):
    # mean 0, sigma 1: the two +-2 samples sit exactly at 2 sigma
    y = np.array([-2, 2, 0, 0, 0, 0, 0, 0])
    assert oracle.moments_clipped(y, 32, 5) == (0.0, 1.0, 8)
    # just inside k = 31/16: they go; the six zeros have sigma 0
    assert oracle.moments_clipped(y, 31, 5) == (0.0, 0.0, 6)
    # one outlier: mean 20, sigma 40; k = 1.5 drops 100 (80 > 60), keeps the zeros
    assert oracle.moments_clipped(np.array([0, 0, 0, 0, 100]), 24, 5) == (0.0, 0.0, 4)
    # a pass that would keep nothing is dropped: sigma 1, k = 15/16 < |y - mu| = 1
    assert oracle.moments_clipped(np.array([-1, 1, -1, 1]), 15, 5) == (0.0, 1.0, 4)


def test_one_pass_versus_many(oracle):
    """A single pass removes only what the full-sample bound excludes."""
    y = np.concatenate([np.zeros(1000, np.int64), [30, 35, 400]])
    full_mu, full_sg = oracle.moments(y)
    one = oracle.moments_clipped(y, 48, 1)
    assert one[2] == int(np.sum(np.abs(y - full_mu) <= 3 * full_sg))
    assert one[2] == 1002  # 400 goes; 30 and 35 lie within 3 sigma of the full sample
    many = oracle.moments_clipped(y, 48, 50)
    assert many[:3] == (0.0, 0.0, 1000)  # the second pass removes them


def test_shift_and_scale_invariance(oracle):
    y = np.random.default_rng(8).normal(100, 7, 8000).round().astype(np.int64)
    y[::97] += 90
    mu, sg, kept = oracle.moments_clipped(y, 40, 20)
    mu2, sg2, kept2 = oracle.moments_clipped(3 * y + 12345, 40, 20)
    assert kept2 == kept
    assert mu2 == pytest.approx(3 * mu + 12345, rel=1e-14)
    assert sg2 == pytest.approx(3 * sg, rel=1e-12)


def test_plan_setting_arguments():
    p = Plan(100, 1400.0, -2.0, 64e-6, [(0.0, 3.0, 37, 1)])
    p.set_sps_clip(48, 5)
    p.set_sps_clip(0, 0)  # back to plain statistics; c16 ignored
    for c16, it in [(0, 3), (256, 3), (48, -1), (48, 65)]:
        with pytest.raises(abi.AAError):
            p.set_sps_clip(c16, it)


def test_gaussian_fixed_point(oracle):
    """Iterated k-sigma clipping of Gaussian data converges to the truncation
    point c with c = k*s(c), s(c) the standard deviation of N(0,1) truncated to
    [-c, c] (closed form); below k ~ 1.73 no such point exists and the kept
    set collapses."""
    stats = pytest.importorskip("scipy.stats")
    optimize = pytest.importorskip("scipy.optimize")
    s = lambda c: np.sqrt(1 - 2 * c * stats.norm.pdf(c) / (2 * stats.norm.cdf(c) - 1))
    y = np.random.default_rng(9).normal(0, 1000, 400000).round().astype(np.int64)
    for c16 in (32, 40, 48):
        k = c16 / 16
        c = optimize.brentq(lambda c: c - k * s(c), 0.5, 10)
        mu, sg, kept = oracle.moments_clipped(y, c16, 200)
        assert sg / 1000 == pytest.approx(s(c), rel=0.01)
        assert kept / y.size == pytest.approx(2 * stats.norm.cdf(c) - 1, rel=0.01)
    _, sg, _ = oracle.moments_clipped(y, 24, 200)  # k = 1.5
    assert sg < 100
