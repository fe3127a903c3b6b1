"""Pins for the oracle's 2-D DM-time peak filter (candidate post-processing of
the single-pulse search, Sec. 1), none of which re-uses its formula: hand
cases, a textbook routine (scipy's maximum filter on a dense DM-time grid, for
lists without equal SNRs), closed forms for the zero and unbounded windows,
and the oracle's own unsorted path against its sorted path."""
import json
import os

import numpy as np
import pytest

from paper_1912_07704_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


def _records(rows):
    out = np.zeros(len(rows), dtype=synth.CANDIDATE_RECORD)
    for i, (d, t, r, s) in enumerate(rows):
        out[i] = (d, t, 1, r, 0, s)
    return out


@pytest.mark.parametrize("case", GOLD["peaks2d"], ids=lambda c: c["derivation"][:30])
def test_peaks2d_hand(oracle, case):
    keep = oracle.peaks2d(_records(case["records"]), case["dm_radius"], case["t_radius"])
    assert keep.tolist() == case["expected"]


def test_zero_window_keeps_everything(oracle):
    f = synth.candidate_field([120, 80], [3000, 1500], 10, 500, seed=3, snr_quantum=0.5)
    assert oracle.peaks2d(f, 0, 0).all()


def test_unbounded_window_keeps_one_per_range(oracle):
    f = synth.candidate_field([120, 80, 40], [3000, 1500, 700], 12, 600, seed=4, snr_quantum=0.5)
    keep = oracle.peaks2d(f, 10 ** 6, 10 ** 9)
    kept = f[keep]
    assert sorted(kept["range"].tolist()) == sorted(set(f["range"].tolist()))
    for r in set(f["range"].tolist()):
        g = f[f["range"] == r]
        # the largest SNR, the smallest (dm_index, t) among equals
        best = g[np.lexsort((g["t"], g["dm_index"], -g["snr"].astype(np.float64)))[0]]
        got = kept[kept["range"] == r][0]
        assert (got["dm_index"], got["t"]) == (best["dm_index"], best["t"])


@pytest.mark.parametrize("radii", [(1, 1), (3, 8), (10, 40), (0, 25), (25, 0)])
def test_matches_maximum_filter_without_ties(oracle, radii):
    ndimage = pytest.importorskip("scipy.ndimage")
    ndm, L = [90, 60], [2000, 1000]
    f = synth.candidate_field(ndm, L, 15, 800, seed=5)
    # continuous SNRs: make them distinct
    f["snr"] = f["snr"] + np.float32(1e-4) * np.arange(f.size, dtype=np.float32) / f.size
    assert np.unique(f["snr"]).size == f.size
    R, Tr = radii
    keep = oracle.peaks2d(f, R, Tr)
    offs = np.concatenate([[0], np.cumsum(ndm)])
    expect = np.zeros(f.size, bool)
    for r in range(len(ndm)):
        grid = np.full((ndm[r], L[r]), -np.inf)
        sel = np.nonzero(f["range"] == r)[0]
        d = f["dm_index"][sel].astype(np.int64) - offs[r]
        grid[d, f["t"][sel]] = f["snr"][sel]
        mx = ndimage.maximum_filter(grid, size=(2 * R + 1, 2 * Tr + 1), mode="constant",
                                    cval=-np.inf)
        expect[sel] = grid[d, f["t"][sel]] == mx[d, f["t"][sel]]
    assert np.array_equal(keep, expect)


def test_order_independent(oracle):
    f = synth.candidate_field([150, 50], [4000, 900], 20, 700, seed=6, snr_quantum=0.25)
    keep = oracle.peaks2d(f, 4, 16)
    perm = np.random.Generator(np.random.PCG64(9)).permutation(f.size)
    keep_p = oracle.peaks2d(f[perm], 4, 16)  # unsorted: every record examined
    assert np.array_equal(keep[perm], keep_p)


def test_pulse_apex_survives(oracle):
    f = synth.candidate_field([200], [5000], 1, 0, seed=11)
    keep = oracle.peaks2d(f, 50, 200)
    top = np.argmax(f["snr"])
    assert keep[top] and keep.sum() >= 1
