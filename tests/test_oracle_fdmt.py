"""Pins for the oracle's FDMT-style tree dedispersion (the tree / FDMT form
of the dedispersion module's cited work, Sec. 1; an approximation whose
per-channel delays come from splitting a subband's delay between its halves).

Independent checks: hand-derived delays (hand_cases.json "fdmt"); the
invariants of the split rule (top channel 0, bottom channel D, monotone, two
channels exact); a closed-form bound on the distance to the ideal delay
D * delta_c / delta_bottom, propagated level by level from the 1/2-sample
rounding of each split; and a literal evaluation of the tree -- subband sums
built from their halves' sums, level by level, in numpy -- equal to the
oracle's brute-force sum at its effective delays."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


def _round_half_away(v: float) -> int:
    f = math.floor(v)
    return int(f + (1 if v - f >= 0.5 else 0))  # v >= 0 here


def _dk(nchans, fch1, foff):
    """delta of the channels in falling-frequency order, and that order."""
    fs = [fch1 + c * foff for c in range(nchans)]
    ft = max(fs[0], fs[-1])
    order = list(range(nchans)) if foff < 0 else list(range(nchans - 1, -1, -1))
    return [1.0 / (fs[c] * fs[c]) - 1.0 / (ft * ft) for c in order], order


def _literal(x, nchans, fch1, foff, D):
    """The tree as sums of sums: A(a, b, delta)[t] for t < T - delta."""
    dk, order = _dk(nchans, fch1, foff)
    rows = x[order].astype(np.int64)  # falling-frequency order
    T = x.shape[1]

    def node(a, b, delta):
        if a == b:
            assert delta == 0
            return rows[a]
        m = a + (b - a + 2) // 2
        span = dk[b] - dk[a]
        gap = _round_half_away((delta * (dk[m] - dk[a])) / span) if span > 0 else 0
        du = _round_half_away((delta * (dk[m - 1] - dk[a])) / span) if span > 0 else 0
        up, lo = node(a, m - 1, du), node(m, b, delta - gap)
        n = T - delta
        return up[:n] + lo[gap:gap + n]

    return node(0, nchans - 1, D)


@pytest.mark.parametrize("case", GOLD["fdmt"], ids=lambda c: f"{c['nchans']}ch-D{c['D']}-foff{c['foff']}")
def test_fdmt_hand_cases(oracle, case):
    e = oracle.fdmt_delays(case["nchans"], case["fch1"], case["foff"], case["D"])
    assert e.tolist() == case["expected"]


@pytest.mark.parametrize("nchans,fch1,foff", [(1, 1400.0, -1.0), (2, 1400.0, -10.0), (7, 1400.0, -3.0),
                                               (64, 1500.0, -2.0), (203, 1400.0, -1.5),
                                               (256, 1200.0, 1.171875), (4096, 1508.0, -0.0732421875)])
def test_fdmt_invariants_and_bound(oracle, nchans, fch1, foff):
    dk, order = _dk(nchans, fch1, foff)
    levels = math.ceil(math.log2(nchans)) if nchans > 1 else 0
    # each split rounds once (|err| <= 1/2); the error of a subband's delay
    # after d levels is <= d/2 and its base's is <= d/2 + d(d-1)/4
    bound = 0.5 * levels + 0.25 * levels * max(levels - 1, 0) + 1e-9
    rng = np.random.default_rng(nchans)
    for D in ([0] if nchans == 1 else [0, 1, 2, 17, 255, 2385, int(rng.integers(0, 5000))]):
        e = oracle.fdmt_delays(nchans, fch1, foff, D)
        ek = e[order]  # falling-frequency order
        assert ek[0] == 0 and ek[-1] == D
        assert np.all(np.diff(ek) >= 0) and np.all((ek >= 0) & (ek <= D))
        if nchans == 2:
            assert ek.tolist() == [0, D]
        if nchans > 1 and dk[-1] > 0:
            ideal = np.array([D * v / dk[-1] for v in dk])
            assert np.abs(ek - ideal).max() <= bound, (D, np.abs(ek - ideal).max(), bound)


@pytest.mark.parametrize("nchans,fch1,foff", [(1, 1400.0, -1.0), (2, 1400.0, -10.0), (3, 1400.0, -7.0),
                                               (5, 1300.0, -11.0), (8, 1500.0, -20.0), (13, 1000.0, 9.0),
                                               (16, 1400.0, -15.0)])
def test_fdmt_literal_tree_equals_effective_delay_sum(oracle, nchans, fch1, foff):
    rng = np.random.default_rng(7 + nchans)
    T = 400
    x = rng.integers(0, 256, size=(nchans, T), dtype=np.uint8)
    for D in ([0] if nchans == 1 else [0, 1, 3, 19, 60]):
        e = oracle.fdmt_delays(nchans, fch1, foff, D)
        y = oracle.dedisperse_row(x, e, 0, T - D)
        assert np.array_equal(y, _literal(x, nchans, fch1, foff, D)), D


def test_fdmt_recovers_a_pulse_at_its_delays(oracle):
    """A box pulse laid along the tree's own delays for D sums fully into
    the root row D at its start time, and only there in that row."""
    C, fch1, foff, T, D, t0, A = 37, 1450.0, -4.0, 3000, 211, 900, 5
    e = oracle.fdmt_delays(C, fch1, foff, D)
    x = np.zeros((C, T), np.uint8)
    for c in range(C):
        x[c, t0 + e[c]] = A
    y = oracle.dedisperse_row(x, e, 0, T - D)
    assert y[t0] == A * C and np.count_nonzero(y) == 1


def test_fdmt_against_brute_force_delays(oracle):
    """For a range of the 4096-channel plan, the tree's delays stay within
    the closed-form bound of the brute-force delays s(c, i) (the bottom
    channel's being equal by construction)."""
    C, fch1, foff, ts = 4096, 1508.0, -0.0732421875, 64e-6
    pl = oracle.plan(C, fch1, foff, ts, [(0.0, 0.1, 60, 1), (600.0, 1.0, 20, 8)], 1 << 16)
    levels = 12
    bound = 0.5 * levels + 0.25 * levels * (levels - 1) + 0.5 + 0.5 + 1e-9
    for g in pl:
        tab = oracle.fdmt_table(C, fch1, foff, g)
        b = oracle.fdmt_bottom(C, foff)
        assert np.array_equal(tab[:, b], g.shifts[:, b])
        assert np.abs(tab.astype(np.int64) - g.shifts).max() <= bound


@pytest.mark.parametrize("nchans,fch1,foff,ranges", [
    (100, 1450.0, -3.0, [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (187.0, 8.0, 19, 8)]),
    (37, 1200.0, 2.5, [(0.0, 5.0, 20, 1)]),
    (4096, 1508.0, -0.0732421875, [(600.0, 1.0, 200, 8)]),
])
def test_library_tree_equals_oracle(oracle, nchans, fch1, foff, ranges):
    """The library's host-built tree (aa_plan_set_fdmt) gives the oracle's
    effective delays for every channel and trial (two implementations of the
    split rule, compared through aa_plan_effective_shifts)."""
    from paper_1912_07704_gb300 import abi
    from paper_1912_07704_gb300.api import Plan
    T = 1 << 17
    p = Plan(nchans, fch1, foff, 64e-6, ranges)
    pl = oracle.plan(nchans, fch1, foff, 64e-6, ranges, T)
    for r, g in enumerate(pl):
        p.set_fdmt(r)
        info = abi.aa_plan_range(p.handle, T, r)
        assert info.strategy == abi.AA_DEDISP_FDMT and info.length == g.length
        eff = abi.aa_plan_effective_shifts(p.handle, r, g.ndm, nchans)
        assert np.array_equal(eff, oracle.fdmt_table(nchans, fch1, foff, g))
        p.set_strategy(r, abi.AA_DEDISP_DIRECT)  # back to the exact sum
        assert np.array_equal(abi.aa_plan_effective_shifts(p.handle, r, g.ndm, nchans), g.shifts)
    p.close()
