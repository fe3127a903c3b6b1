"""Pins for the CPU oracle, none of which re-uses the oracle's own formula.

Each check is either a hand-derived value (tests/golden/hand_cases.json), a
library routine (numpy sum/mean/std/convolve/add.at), a closed form, an
invariant of the method, or a structurally different brute force.  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


# ---------------------------------------------------------------- delays ----

@pytest.mark.parametrize("case", GOLD["shifts"], ids=lambda c: c["name"])
def test_shift_hand_values(oracle, case):
    s = oracle.shifts(case["nchans"], case["fch1"], case["foff"], case["tsamp"], case["dm"],
                      case["dec"])
    assert s.tolist() == case["expected"]


def _exact_shift(nchans, fch1, foff, tsamp, dm, dec, c):
    """Exact rational value of the delay for the given double inputs."""
    F = Fraction
    f = [F(fch1) + i * F(foff) for i in (0, nchans - 1)]
    ft = max(f)
    fc = F(fch1) + c * F(foff)
    v = F(4148808, 1000) * F(dm) * (1 / (fc * fc) - 1 / (ft * ft)) / (F(tsamp) * dec)
    return v


def test_shift_against_exact_rationals(oracle):
    """Double-precision delays round like the exact rational value, except
    within 1e-9 of a half-integer (where neither side is meaningful)."""
    rng = np.random.default_rng(5)
    for (C, fch1, foff, tsamp, dec) in [(256, 1500.0, -1.171875, 64e-6, 1),
                                        (4096, 1508.0, -0.0732421875, 64e-6, 8),
                                        (1024, 1208.0, 0.29296875, 64e-6, 2)]:
        for dm in rng.uniform(0, 3000, 6):
            s = oracle.shifts(C, fch1, foff, tsamp, float(dm), dec)
            for c in rng.integers(0, C, 12):
                v = _exact_shift(C, fch1, foff, tsamp, float(dm), dec, int(c))
                fl = math.floor(v)
                frac = v - fl
                if abs(frac - Fraction(1, 2)) < Fraction(1, 10**9):
                    continue
                want = fl + (1 if frac > Fraction(1, 2) else 0)
                assert s[c] == want, (C, dm, c, float(v))


def test_shift_invariants(oracle):
    C, fch1, foff, ts = 512, 1400.0, -0.5859375, 64e-6
    z = oracle.shifts(C, fch1, foff, ts, 0.0)
    assert (z == 0).all()
    prev = None
    for dm in np.linspace(0, 2000, 41):
        s = oracle.shifts(C, fch1, foff, ts, float(dm))
        assert s[0] == 0                       # top of the band never moves
        assert (np.diff(s) >= 0).all()         # lower frequency -> later arrival
        if prev is not None:
            assert (s >= prev).all()           # monotone in DM
        prev = s
    # mirrored band: ascending channel order gives the reversed delays
    up = oracle.shifts(C, fch1 + (C - 1) * foff, -foff, ts, 700.0)
    down = oracle.shifts(C, fch1, foff, ts, 700.0)
    assert (up[::-1] == down).all()


def test_plan_regression_constants(oracle):
    """Max delays of the two measured workloads (derived independently when
    the workloads were specified): 4110 for 256 ch / DM 0..255, and
    2385/2385/2385/3976 for the 4096-ch four-range plan."""
    pl = oracle.plan(256, 1500.0, -1.171875, 64e-6, [(0.0, 1.0, 256, 1)], 32768)
    assert [r.maxshift for r in pl] == [4110]
    assert [r.length for r in pl] == [32768 - 4110]
    pl = oracle.plan(4096, 1508.0, -0.0732421875, 64e-6,
                     [(0.0, 0.1, 1500, 1), (150.0, 0.2, 750, 2), (300.0, 0.5, 600, 4),
                      (600.0, 1.0, 1400, 8)], 1 << 20)
    assert [r.maxshift for r in pl] == [2385, 2385, 2385, 3976]
    assert sum(r.ndm * r.length for r in pl) == 2294503550


# ---------------------------------------------------------- decimation ----

def test_decimate_hand(oracle):
    g = GOLD["decimate"]
    out = oracle.decimate(np.array(g["x"], np.uint8), g["dec"])
    assert out.tolist() == g["expected"]


def test_decimate_identity_and_total(oracle):
    rng = np.random.default_rng(1)
    x = rng.integers(0, 256, (7, 103), dtype=np.uint8)
    assert (oracle.decimate(x, 1) == x).all()
    for dec in (2, 3, 4, 8, 16):
        d = oracle.decimate(x, dec)
        nd = 103 // dec
        assert d.shape == (7, nd)
        assert (d.astype(np.int64).sum(1) == x[:, :nd * dec].astype(np.int64).sum(1)).all()


# -------------------------------------------------------- dedispersion ----

def test_dedisperse_two_channel_hand(oracle):
    g = GOLD["dedisperse_two_channel"]
    x = np.array(g["x"], np.uint8)
    y = oracle.dedisperse_row(x, np.array(g["shifts"], np.int32), 0, len(g["expected"]))
    assert y.tolist() == g["expected"]


def test_dm_zero_is_channel_sum(oracle):
    rng = np.random.default_rng(2)
    x = rng.integers(0, 256, (64, 3000), dtype=np.uint8)
    pl, ys = oracle.dedisperse(x, 64, 1400.0, -1.0, 64e-6, [(0.0, 5.0, 4, 1)])
    assert (ys[0][0] == x[:, :pl[0].length].astype(np.int64).sum(0)).all()


def test_impulse_response(oracle):
    C, T = 32, 1500
    fch1, foff, ts = 1400.0, -4.0, 64e-6
    rng = [(0.0, 10.0, 12, 1)]
    pl = oracle.plan(C, fch1, foff, ts, rng, T)[0]
    for (c, tau) in [(0, 700), (31, 1400), (17, 900), (5, pl.maxshift)]:
        x = np.zeros((C, T), np.uint8)
        x[c, tau] = 1
        _, ys = oracle.dedisperse(x, C, fch1, foff, ts, rng)
        for i in range(pl.ndm):
            t = tau - pl.shifts[i][c]
            row = ys[0][i]
            if 0 <= t < pl.length:
                assert row[t] == 1 and row.sum() == 1
            else:
                assert row.sum() == 0


def test_linearity(oracle):
    rng = np.random.default_rng(3)
    a = rng.integers(0, 128, (48, 2500), dtype=np.uint8)
    b = rng.integers(0, 128, (48, 2500), dtype=np.uint8)
    r = [(0.0, 25.0, 9, 1)]
    _, ya = oracle.dedisperse(a, 48, 1300.0, -2.0, 64e-6, r)
    _, yb = oracle.dedisperse(b, 48, 1300.0, -2.0, 64e-6, r)
    _, yab = oracle.dedisperse(a + b, 48, 1300.0, -2.0, 64e-6, r)
    assert (ya[0] + yb[0] == yab[0]).all()


def test_scatter_brute_force(oracle):
    """Transpose formulation: every input sample is pushed to the outputs it
    reaches (np.add.at), instead of every output pulling its inputs."""
    rng = np.random.default_rng(4)
    C, T = 16, 256
    x = rng.integers(0, 256, (C, T), dtype=np.uint8)
    r = [(0.0, 40.0, 8, 1)]
    pl, ys = oracle.dedisperse(x, C, 1400.0, -8.0, 64e-6, r)
    L = pl[0].length
    for i in range(8):
        y = np.zeros(L, np.int64)
        cc, tt = np.meshgrid(np.arange(C), np.arange(T), indexing="ij")
        t_out = tt - pl[0].shifts[i][cc]
        ok = (t_out >= 0) & (t_out < L)
        np.add.at(y, t_out[ok], x[cc[ok], tt[ok]].astype(np.int64))
        assert (y == ys[0][i]).all()


def test_decimated_range_equals_prebinned_input(oracle):
    """Range with decimation d == dec-1 search of explicitly pre-binned data
    sampled at tsamp*d."""
    rng = np.random.default_rng(6)
    C, T = 24, 4000
    x = rng.integers(0, 256, (C, T), dtype=np.uint8)
    for d in (2, 4, 8):
        pl, ys = oracle.dedisperse(x, C, 1400.0, -6.0, 64e-6, [(100.0, 30.0, 5, d)])
        nd = T // d
        binned = x[:, :nd * d].astype(np.uint16).reshape(C, nd, d).sum(2).astype(np.uint16)
        ts_d = 64e-6 * d
        for i in range(5):
            sh = oracle.shifts(C, 1400.0, -6.0, ts_d, 100.0 + i * 30.0, 1)
            y = oracle.dedisperse_row(binned, sh, 0, nd - int(pl[0].shifts.max()))
            assert (y == ys[0][i]).all()


# ----------------------------------------------------------- statistics ----

def test_moments_against_numpy(oracle):
    rng = np.random.default_rng(7)
    y = rng.integers(-10**6, 10**7, 10007).astype(np.int64)
    mu, sg = oracle.moments(y)
    assert mu == pytest.approx(np.mean(y.astype(np.float64)), rel=1e-15)
    assert sg == pytest.approx(np.std(y.astype(np.float64)), rel=1e-12)
    mu, sg = oracle.moments(np.full(50, 123, np.int64))
    assert mu == 123.0 and sg == 0.0


# --------------------------------------------------------------- boxcar ----

def test_width_one_is_zscore(oracle):
    rng = np.random.default_rng(8)
    y = rng.integers(0, 5000, 777).astype(np.int64)
    mu, sg = oracle.moments(y)
    B, wb, _ = oracle.boxcar(y, mu, sg, 1)
    z = (y - y.mean()) / y.std()
    assert np.allclose(B, z, rtol=0, atol=1e-12)
    assert (wb == 1).all()


def test_boxcar_brute_force_convolve(oracle):
    """All windows via np.convolve (a library routine), first argmax."""
    rng = np.random.default_rng(9)
    for n, W in [(200, 17), (64, 64), (50, 80)]:
        y = rng.integers(0, 1000, n).astype(np.int64)
        mu, sg = y.mean(), y.std()
        B, wb, _ = oracle.boxcar(y, mu, sg, W)
        table = np.full((W, n), -np.inf)
        for w in range(1, min(W, n) + 1):
            s = np.convolve(y.astype(np.float64), np.ones(w), mode="valid")  # t = 0..n-w
            table[w - 1, :n - w + 1] = (s - w * mu) / (sg * np.sqrt(w))
        assert np.allclose(B, table.max(0), rtol=0, atol=1e-9)
        assert (wb == table.argmax(0) + 1).all()


def test_box_pulse_closed_form(oracle):
    g = GOLD["box_pulse"]
    y = np.zeros(g["L"], np.int64)
    y[g["start"]:g["start"] + g["n"]] = g["amplitude"]
    mu, sg = oracle.moments(y)
    B, wb, _ = oracle.boxcar(y, mu, sg, g["W"], g["start"], g["start"] + 1)
    assert B[0] == pytest.approx(g["expected_snr"], abs=1e-9)
    assert wb[0] == g["expected_width"]


def test_window_clipped_at_series_end(oracle):
    y = np.array([5, 1, 9, 2, 8], np.int64)
    mu, sg = oracle.moments(y)
    B, wb, _ = oracle.boxcar(y, mu, sg, 100, 4, 5)
    assert wb[0] == 1
    assert B[0] == pytest.approx((8 - y.mean()) / y.std(), abs=1e-12)


def test_sigma_zero_guard(oracle):
    y = np.full(100, 7, np.int64)
    c, B, wb, mu, sg = oracle.search_row(y, 16, -1.0, 0, 0)
    assert sg == 0.0 and (B == 0).all() and c == []


# ---------------------------------------------------------------- peaks ----

@pytest.mark.parametrize("case", GOLD["peaks"], ids=lambda c: c["derivation"][:30])
def test_peaks_hand(oracle, case):
    assert oracle.peaks_thr(np.array(case["B"]), case["thr"]).tolist() == case["expected"]
