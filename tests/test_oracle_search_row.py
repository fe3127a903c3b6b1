"""Pins for ``oracle.search_row``, the function every single-pulse parity test
compares the GPU with.

Its candidate decision must be exactly the thresholded local-maximum rule
(Sec. 1, peak finding; B(t) >= thr, B(t) > B(t-1), B(t) >= B(t+1), missing
neighbours -inf) that ``peaks_thr`` implements and ``test_peaks_hand`` pins by
hand, evaluated on the full series: a window [t_lo, t_hi) must not turn an
interior sample into an edge.  Its fragility flag must mark every decision
whose margin is below the FP32/FP64 disagreement allowed to the GPU.

The hand cases of ``hand_cases.json`` ("peaks") are run as real series: with
a single width (W = 1) B is the z-score (y - mu)/sigma, an increasing affine
map of y, so y = 100*B keeps every order and tie of the hand array, and the
hand threshold maps to (100*thr - mu)/sigma, evaluated in the same IEEE double
operations as the oracle's SNR (so threshold equality survives the map).
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


def _full_peaks(oracle, y, W, thr):
    mu, sg = oracle.moments(y)
    B, wb, mg = oracle.boxcar(y, mu, sg, W)
    return set(oracle.peaks_thr(B, thr).tolist()), B, wb, mg


def _split(cands):
    solid = {c.t: c for c in cands if not c.fragile}
    frag = {c.t: c for c in cands if c.fragile}
    return solid, frag


@pytest.mark.parametrize("case", GOLD["peaks"], ids=lambda c: c["derivation"][:30])
def test_hand_cases_as_series(oracle, case):
    y = np.rint(100.0 * np.array(case["B"])).astype(np.int64)
    mu, sg = oracle.moments(y)
    thr_z = (100.0 * case["thr"] - 1.0 * mu) / (sg * math.sqrt(1.0))
    cands, B, wb, _, _ = oracle.search_row(y, 1, thr_z, 7, 0)
    got = sorted(c.t for c in cands)
    expected = case["expected"]
    # every hand peak is reported (solid or fragile); nothing else is solid
    assert set(expected) <= set(got)
    solid, frag = _split(cands)
    assert set(solid) <= set(expected)
    for c in cands:
        assert c.dm_index == 7 and c.range == 0 and c.width == 1
        assert c.snr == B[c.t]


def test_hand_threshold_equality_is_inclusive_and_fragile(oracle):
    """[7, 1, 6, 6] at thr 6: t = 2 sits exactly on the threshold (a peak,
    inclusive) and ties with its right neighbour: reported, flagged."""
    case = next(c for c in GOLD["peaks"] if c["B"] == [7.0, 1.0, 6.0, 6.0])
    y = np.rint(100.0 * np.array(case["B"])).astype(np.int64)
    mu, sg = oracle.moments(y)
    thr_z = (100.0 * case["thr"] - 1.0 * mu) / (sg * math.sqrt(1.0))
    cands, B, *_ = oracle.search_row(y, 1, thr_z, 0, 0)
    by_t = {c.t: c for c in cands}
    assert B[2] == thr_z  # the map kept the equality
    assert 2 in by_t and by_t[2].fragile
    assert 0 in by_t and not by_t[0].fragile  # the left edge: a clear peak
    assert 3 not in by_t or by_t[3].fragile


def test_plateau_leftmost_only(oracle):
    """A wide plateau well above the threshold: its leftmost sample is the
    only peak (fragile: it ties its right neighbour), the rest are not."""
    y = np.array([0, 0, 50, 50, 50, 50, 0, 0, 0, 0], np.int64)
    cands, B, *_ = oracle.search_row(y, 1, 0.5, 0, 0)
    ts = {c.t: c for c in cands}
    assert 2 in ts and ts[2].fragile
    assert not any(t in ts and not ts[t].fragile for t in (3, 4, 5))


def test_edges_compare_with_minus_infinity(oracle):
    """Peaks at both ends of the series (no neighbour outside): found even
    when the search window starts or ends there."""
    y = np.array([90, 10, 20, 10, 15, 10, 80], np.int64)
    for lo, hi in [(0, 7), (0, 3), (4, 7), (0, 1), (6, 7)]:
        cands, *_ = oracle.search_row(y, 1, 1.0, 0, 0, lo, hi)
        solid, frag = _split(cands)
        want = {t for t in (0, 6) if lo <= t < hi}
        assert set(solid) == want, (lo, hi, sorted(solid))


def test_window_keeps_true_neighbours(oracle):
    """An interior window boundary is not an edge: a sample whose left
    neighbour (outside the window) is larger is no peak, and one whose right
    neighbour (outside) is larger is no peak either."""
    y = np.array([10, 95, 90, 10, 10, 70, 75, 10], np.int64)
    full, B, *_ = _full_peaks(oracle, y, 1, 0.5)
    assert full == {1, 6}
    for lo, hi in [(2, 6), (2, 3), (5, 6), (2, 8), (0, 2)]:
        cands, *_ = oracle.search_row(y, 1, 0.5, 0, 0, lo, hi)
        solid, frag = _split(cands)
        assert set(solid) == {t for t in full if lo <= t < hi}, (lo, hi)
        assert not frag


@pytest.mark.parametrize("seed", range(6))
def test_random_rows_equal_peaks_thr(oracle, seed):
    """Seeded rows with many ties (small value ranges), several widths and
    thresholds and random windows: the solid candidates are peaks_thr of
    the full B, every peak in the window is reported, and each record's
    SNR and width are the full search's B and smallest maximising width."""
    rng = np.random.default_rng(100 + seed)
    checked = 0
    for _ in range(25):
        n = int(rng.integers(2, 400))
        vmax = int(rng.choice([3, 6, 40, 5000]))
        y = rng.integers(0, vmax, n).astype(np.int64)
        if rng.random() < 0.3:  # a plateau run
            a = int(rng.integers(0, n))
            y[a:a + int(rng.integers(2, 9))] = vmax
        W = int(rng.choice([1, 2, 3, 8, 33]))
        mu, sg = oracle.moments(y)
        if sg == 0.0:
            continue
        _, Bfull, wbf, _ = _full_peaks(oracle, y, W, 0.0)
        thr = float(np.quantile(Bfull, rng.uniform(0.5, 0.99)))
        peaks, B, wb, mg = _full_peaks(oracle, y, W, thr)
        lo = int(rng.integers(0, n))
        hi = int(rng.integers(lo, n + 1))
        if rng.random() < 0.3:
            lo, hi = 0, n
        cands, Bw, wbw, mu2, sg2 = oracle.search_row(y, W, thr, 3, 1, lo, hi)
        assert (mu2, sg2) == (mu, sg)
        assert np.array_equal(Bw, B[lo:hi]) and np.array_equal(wbw, wb[lo:hi])
        solid, frag = _split(cands)
        inwin = {t for t in peaks if lo <= t < hi}
        assert set(solid) <= inwin
        assert inwin <= set(solid) | set(frag)
        for c in cands:
            assert lo <= c.t < hi
            assert c.snr == B[c.t] and c.width == wb[c.t]
        checked += len(solid)
    assert checked > 0


def test_fragile_flags(oracle):
    """Hand-built near-decision cases.  Values spread over 0..10^6 give
    sigma ~ 3e5, so one count is ~3e-6 in SNR units: far below the 2e-4
    comparison margin.  W = 1, so B(t) = (y(t) - mu)/sigma."""
    rng = np.random.default_rng(21)
    n = 2000
    y = rng.integers(0, 1_000_000, n).astype(np.int64)
    for a in (90, 290, 495, 695):  # quiet surroundings of each case
        y[a:a + 20] = 10
    y[100:105] = [10, 900_000, 900_001, 100, 10]      # neighbours 1 count apart
    y[300:303] = [10, 990_000, 10]                     # a clear isolated peak
    y[500:504] = [10, 980_000, 980_000, 10]            # an exact tie (plateau)
    y[700:703] = [10, 970_000, 10]                     # threshold just above it below
    mu, sg = oracle.moments(y)
    z = lambda v: (float(v) - 1.0 * mu) / (sg * math.sqrt(1.0))
    peaks, B, wb, mg = _full_peaks(oracle, y, 1, 0.0)
    # (a) peak whose left neighbour is within 2e-4: reported, fragile
    thr = z(800_000)
    cands, *_ = oracle.search_row(y, 1, thr, 0, 0, 90, 110)
    by_t = {c.t: c for c in cands}
    assert 102 in by_t and by_t[102].fragile
    assert 101 in by_t and by_t[101].fragile  # not a peak, but within the margin
    # (b) isolated peak far from the threshold: reported, solid
    cands, *_ = oracle.search_row(y, 1, thr, 0, 0, 290, 310)
    assert [(c.t, c.fragile) for c in cands] == [(301, False)]
    # (c) plateau of equal values: leftmost reported, flagged
    cands, *_ = oracle.search_row(y, 1, thr, 0, 0, 495, 510)
    by_t = {c.t: c for c in cands}
    assert 501 in by_t and by_t[501].fragile
    # (d) |B - thr| < 1e-3 with B below thr: not a peak by the rule, but
    #     reported as fragile (it could flip into an FP32 list)
    v = B[701]
    cands, *_ = oracle.search_row(y, 1, v + 5e-4, 0, 0, 695, 710)
    assert [(c.t, c.fragile) for c in cands] == [(701, True)]
    assert 701 not in set(oracle.peaks_thr(B, v + 5e-4).tolist())
    # ... and just above it: a peak, fragile
    cands, *_ = oracle.search_row(y, 1, v - 5e-4, 0, 0, 695, 710)
    assert [(c.t, c.fragile) for c in cands] == [(701, True)]
    # ... and 2e-3 below: solid
    cands, *_ = oracle.search_row(y, 1, v - 2e-3, 0, 0, 695, 710)
    assert [(c.t, c.fragile) for c in cands] == [(701, False)]


def test_fragile_width_margin(oracle):
    """Two widths whose SNRs differ by less than 2e-4 at a clear peak: the
    width decision is fragile, so the candidate is flagged."""
    rng = np.random.default_rng(5)
    n = 3000
    y = rng.integers(0, 1_000_000, n).astype(np.int64)
    # SNR_1 = (a - mu)/sg, SNR_2 = (a + b - 2 mu)/(sg sqrt 2): equal for
    # b - mu = (sqrt 2 - 1)(a - mu); b moves mu by b/n, so iterate to the
    # fixed point
    a = 3_000_000
    y[990:1010] = 0
    y[1001] = a
    for _ in range(6):
        mu, sg = oracle.moments(y)
        y[1002] = int(round(mu + (math.sqrt(2.0) - 1.0) * (a - mu)))
    mu, sg = oracle.moments(y)
    B, wb, mg = oracle.boxcar(y, mu, sg, 2)
    assert mg[1001] < 2e-4
    cands, *_ = oracle.search_row(y, 2, 1.0, 0, 0, 995, 1010)
    by_t = {c.t: c for c in cands}
    assert 1001 in by_t and by_t[1001].fragile
