"""Pins of the oracle's decimated width ladder (oracle_boxcar_dec), the
approximate single-pulse search for wide boxcars: level 0 takes every width
1..W0 at full time resolution; level k takes the widths m * 2^k,
W0/2 < m <= W0, of the windows that start at the level-k grid point at or
before t, i.e. m samples of the series decimated k times by pairs (the cited
search method of Sec. 1 evaluates wide boxcars on decimated series).

Independent checks:
* the hand-derived worked example (hand_cases.json "dec_ladder");
* brute force in pure Python that decimates the series explicitly by pairs
  (the oracle's decimate) and slides windows over each decimated series;
* W0 >= W is the exhaustive search (oracle_boxcar);
* closed form: an aligned box pulse on a zero background has B = A sqrt(w)
  over its first grid cell, at its own width;
* invariants: B never exceeds the exhaustive B at t or at a grid point
  before it, and never falls below the exhaustive search restricted to
  widths <= W0.
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


@pytest.mark.parametrize("case", GOLD["dec_ladder"])
def test_hand_case(oracle, case):
    y = np.array(case["y"], dtype=np.int64)
    B, wb, _ = oracle.boxcar(y, case["mu"], case["sigma"], case["W"], dec_w0=case["W0"])
    assert np.allclose(B, case["B"], rtol=0, atol=1e-12)
    assert wb.tolist() == case["wbest"]
    assert oracle.peaks_thr(B, case["thr"]).tolist() == case["peaks"]


def _brute(y, mu, sigma, W, W0):
    """Every window of the ladder from explicitly decimated series."""
    n = len(y)
    B, wb = [], []
    levels = [np.asarray(y, dtype=np.int64)]
    k = 1
    while (W0 << (k - 1)) < W:
        levels.append(np.asarray(levels[-1][: (len(levels[-1]) // 2) * 2].reshape(-1, 2).sum(axis=1)))
        k += 1
    for t in range(n):
        best, bw = -math.inf, 0
        for w in range(1, min(W0, W, n - t) + 1):
            snr = (int(levels[0][t:t + w].sum()) - w * mu) / (sigma * math.sqrt(w))
            if snr > best:
                best, bw = snr, w
        for k in range(1, len(levels)):
            yk = levels[k]
            j = t >> k
            for m in range(W0 // 2 + 1, W0 + 1):
                w = m << k
                if w > W or j + m > len(yk):
                    break
                snr = (int(yk[j:j + m].sum()) - w * mu) / (sigma * math.sqrt(w))
                if snr > best:
                    best, bw = snr, w
        B.append(best)
        wb.append(bw)
    return np.array(B), np.array(wb)


@pytest.mark.parametrize("seed,n,W,W0", [(1, 200, 64, 4), (2, 301, 100, 8), (3, 257, 256, 16),
                                         (4, 150, 33, 32), (5, 64, 64, 2)])
def test_brute_force_decimated_series(oracle, seed, n, W, W0):
    rng = np.random.default_rng(seed)
    y = rng.integers(-50, 60, size=n)
    y[n // 3:n // 3 + 23] += 40  # a wide box
    mu, sigma = float(y.mean()), float(y.std())
    B, wb, _ = oracle.boxcar(y, mu, sigma, W, dec_w0=W0)
    Bb, wbb = _brute(y, mu, sigma, W, W0)
    assert np.allclose(B, Bb, rtol=1e-12, atol=1e-12)
    assert np.array_equal(wb, wbb)
    # the pair sums taken k times are the dedispersion's decimation by 2^k
    x = rng.integers(0, 256, size=(1, n)).astype(np.uint8)
    d = x[0].astype(np.int64)
    for _ in range(2):
        d = d[: (len(d) // 2) * 2].reshape(-1, 2).sum(axis=1)
    assert np.array_equal(oracle.decimate(x, 4)[0], d)


@pytest.mark.parametrize("W0", [16, 32, 64])
def test_w0_at_least_w_is_the_exhaustive_search(oracle, W0):
    rng = np.random.default_rng(W0)
    y = rng.integers(0, 255, size=500)
    mu, sigma = float(y.mean()), float(y.std())
    B, wb, mg = oracle.boxcar(y, mu, sigma, W0, dec_w0=W0)
    Be, wbe, mge = oracle.boxcar(y, mu, sigma, W0)
    assert np.array_equal(B, Be) and np.array_equal(wb, wbe) and np.array_equal(mg, mge)


@pytest.mark.parametrize("k,m,j", [(1, 9, 5), (3, 12, 7), (4, 16, 2), (2, 11, 20)])
def test_aligned_box_closed_form(oracle, k, m, j):
    W0, A = 16, 3.0
    w, s = m << k, j << k
    n = s + w + 300
    W = W0 << 5
    y = np.zeros(n, dtype=np.int64)
    y[s:s + w] = int(A)
    B, wb, _ = oracle.boxcar(y, 0.0, 1.0, W, dec_w0=W0)
    for t in range(s, s + (1 << k)):
        assert abs(B[t] - A * math.sqrt(w)) < 1e-9 and wb[t] == w, t
    assert B[s - 1] < A * math.sqrt(w)
    assert s in oracle.peaks_thr(B, 1.0).tolist()


@pytest.mark.parametrize("seed", [7, 8])
def test_bounded_by_exhaustive_search(oracle, seed):
    rng = np.random.default_rng(seed)
    n, W, W0 = 700, 256, 16
    y = rng.integers(0, 255, size=n)
    y[300:380] += 30
    mu, sigma = float(y.mean()), float(y.std())
    B, wb, _ = oracle.boxcar(y, mu, sigma, W, dec_w0=W0)
    Be, _, _ = oracle.boxcar(y, mu, sigma, W)
    B0, _, _ = oracle.boxcar(y, mu, sigma, W0)
    for t in range(n):
        starts = {t} | {(t >> k) << k for k in range(1, 5)}
        assert B[t] <= max(Be[s] for s in starts) + 1e-12
        assert B[t] >= B0[t] - 1e-12
    # level-k widths are multiples of 2^k above W0 * 2^(k-1)
    for w in set(wb.tolist()):
        if w > W0:
            k = max(1, math.ceil(math.log2(w / W0)))
            assert w % (1 << k) == 0 and W0 << (k - 1) < w <= W0 << k


def test_search_row_uses_the_ladder(oracle):
    rng = np.random.default_rng(11)
    n, W, W0 = 3000, 512, 16
    y = rng.normal(1000, 30, size=n).round().astype(np.int64)
    y[1024:1024 + 256] += 25  # wide, aligned to 256
    cands, B, wb, mu, sigma = oracle.search_row(y, W, 6.0, 3, 0, dec_w0=W0)
    Bd, wbd, _ = oracle.boxcar(y, mu, sigma, W, dec_w0=W0)
    assert np.array_equal(B, Bd) and np.array_equal(wb, wbd)
    solid = [c for c in cands if not c.fragile]
    assert any(abs(c.t - 1024) <= 16 and c.width >= 128 for c in solid)


def test_set_sps_decimated_arguments():
    from paper_1912_07704_gb300 import abi
    from paper_1912_07704_gb300.api import Plan
    p = Plan(64, 1400.0, -4.0, 64e-6, [(0.0, 4.0, 20, 1)])
    for w0 in (0, 16, 32, 64, 128, 256):
        p.set_sps_decimated(w0)
    for w0 in (-16, 8, 24, 48, 512):
        with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
            p.set_sps_decimated(w0)
    # the two width ladders exclude each other
    p.set_sps_decimated(32)
    with pytest.raises(abi.AAError, match="AA_ERR_CONFIG"):
        p.set_sps_ladder(24)
    p.set_sps_decimated(0)
    p.set_sps_ladder(24)
    with pytest.raises(abi.AAError, match="AA_ERR_CONFIG"):
        p.set_sps_decimated(32)
    p.set_sps_ladder(0)
    p.set_sps_decimated(32)
