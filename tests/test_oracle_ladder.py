"""Pins for the oracle's sparse width ladder (the boxcar search over a subset
of widths for large W): hand-derived chunk lists, the ladder that keeps every
chunk equals the exhaustive search, the ladder's B(t) equals a brute-force
maximum over its widths (numpy convolutions) and never exceeds the
exhaustive B(t)."""
import numpy as np
import pytest


def _chunks(mask):
    return sorted(set((np.nonzero(mask)[0] // 16).tolist()))


def test_ladder_chunk_lists_hand(oracle):
    # growth 1.5: 4 -> max(5, ceil(6)) = 6 -> ceil(9) = 9 -> ceil(13.5) = 14 -> 21 -> 32 -> 48
    assert _chunks(oracle.ladder_widths(1024, 24)) == [0, 1, 2, 3, 4, 6, 9, 14, 21, 32, 48]
    # growth 2: chunks 0-3, then 4, 8, 16, 32, ...
    assert _chunks(oracle.ladder_widths(8192, 32)) == [0, 1, 2, 3, 4, 8, 16, 32, 64, 128, 256]
    # the last chunk may be partial: widths past W are not part of it
    m = oracle.ladder_widths(100, 24)
    assert m.size == 100 and _chunks(m) == [0, 1, 2, 3, 4, 6]


def test_every_chunk_equals_exhaustive(oracle):
    # growth 17/16 keeps chunks 0..17 (widths 1..288)
    rng = np.random.default_rng(2)
    y = rng.integers(0, 200, 3000).astype(np.int64)
    y[1000:1080] += 60
    mu, sg = oracle.moments(y)
    wset = oracle.ladder_widths(272, 17)
    assert wset.all()
    B0, w0, _ = oracle.boxcar(y, mu, sg, 272)
    B1, w1, _ = oracle.boxcar(y, mu, sg, 272, wset=wset)
    assert np.array_equal(B0, B1) and np.array_equal(w0, w1)


def test_ladder_is_max_over_its_widths(oracle):
    rng = np.random.default_rng(3)
    n, W = 1500, 400
    y = rng.integers(0, 100, n).astype(np.int64)
    y[600:700] += 25
    mu, sg = oracle.moments(y)
    wset = oracle.ladder_widths(W, 24)
    B, wb, _ = oracle.boxcar(y, mu, sg, W, wset=wset)
    Be, _, _ = oracle.boxcar(y, mu, sg, W)
    best = np.full(n, -np.inf)
    bw = np.zeros(n, np.int64)
    for w in np.nonzero(wset)[0] + 1:
        S = np.convolve(y.astype(np.float64), np.ones(w), mode="valid")  # S[t] = sum y[t..t+w-1]
        snr = (S - w * mu) / (sg * np.sqrt(w))
        t = np.arange(S.size)
        better = snr > best[t] + 1e-12
        best[t] = np.where(better, snr, best[t])
        bw[t] = np.where(better, w, bw[t])
    assert np.allclose(B, best, rtol=0, atol=1e-9)
    assert np.array_equal(wb, bw)
    assert (B <= Be + 1e-12).all()
    on = wset[np.asarray(oracle.boxcar(y, mu, sg, W)[1]) - 1]  # exhaustive best width in the ladder
    assert np.allclose(B[on], Be[on], atol=1e-12)


def test_set_sps_ladder_arguments():
    from paper_1912_07704_gb300 import abi
    from paper_1912_07704_gb300.api import Plan
    p = Plan(64, 1400.0, -4.0, 64e-6, [(0.0, 4.0, 20, 1)])
    for g in (0, 17, 24, 64):
        p.set_sps_ladder(g)
    for g in (-1, 1, 16, 65):
        with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
            p.set_sps_ladder(g)
