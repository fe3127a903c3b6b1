"""Pins for the oracle's sub-band dedispersion (an approximation of the
brute-force sum): one-channel bands reduce to brute force, a literal two-stage
evaluation (band sums at the coarse trial, then band sums at the fine trial)
equals the oracle's effective-delay sum, the effective delays stay within the
closed-form smearing bound, a hand-derived relative delay, and the host plan
(library) agrees with the oracle on the effective maximum delay."""
import numpy as np
import pytest

from paper_1912_07704_gb300 import abi
from paper_1912_07704_gb300.api import Plan

K_DM = 4.148808e3


def _range(oracle, C, fch1, foff, ts, rg, T):
    return oracle.plan(C, fch1, foff, ts, [rg], T)[0]


def test_relative_delay_hand(oracle):
    # channel 0 at 1000 MHz (the band's reference), channel 1 at 500 MHz:
    # 4148.808 * 10 * (1/500^2 - 1/1000^2) / 1e-3 = 124.46 -> 124
    assert oracle.subband_rel(2, 1000.0, -500.0, 1e-3, 10.0, 1, 2).tolist() == [0, 124]
    # decimated by 4: 31.12 -> 31; bands of one channel: all zero
    assert oracle.subband_rel(2, 1000.0, -500.0, 1e-3, 10.0, 4, 2).tolist() == [0, 31]
    assert oracle.subband_rel(2, 1000.0, -500.0, 1e-3, 10.0, 1, 1).tolist() == [0, 0]
    # rising band: the reference is the band's last (highest) channel
    assert oracle.subband_rel(2, 500.0, 500.0, 1e-3, 10.0, 1, 2).tolist() == [124, 0]


def test_relative_delay_monotone_nonnegative(oracle):
    prev = np.zeros(300, np.int64)
    for dm in np.linspace(0, 800, 57):
        r = oracle.subband_rel(300, 1500.0, -1.0, 64e-6, dm, 2, 37).astype(np.int64)
        assert (r >= 0).all() and (r >= prev).all()
        prev = r


def test_one_channel_bands_are_brute_force(oracle):
    C, fch1, foff, ts, T = 64, 1400.0, -4.0, 64e-6, 5000
    rng = _range(oracle, C, fch1, foff, ts, (0.0, 3.0, 37, 2), T)
    eff, rmax, s2max = oracle.subband_delays(C, fch1, foff, ts, rng, 1, 16)
    assert rmax == 0 and s2max == rng.maxshift
    assert np.array_equal(eff, rng.shifts.astype(np.int64))


@pytest.mark.parametrize("band,coarse,foff", [(16, 8, -2.0), (7, 16, -2.0), (10, 5, 2.0)])
def test_two_stage_evaluation(oracle, band, coarse, foff):
    C, fch1, ts, T = 45, 1400.0 if foff < 0 else 1310.0, 64e-6, 3000
    rg = (5.0, 2.5, 27, 2)
    rng = _range(oracle, C, fch1, foff, ts, rg, T)
    x = np.random.default_rng(3).integers(0, 256, size=(C, T), dtype=np.uint8)
    y, eff, rmax, s2max = oracle.dedisperse_subband(x, C, fch1, foff, ts, rng, band, coarse)
    xr = oracle.range_input(x, rg[3]).astype(np.int64)
    L = rng.nsamp_dec - (rmax + s2max)
    assert y.shape == (rg[2], L) and L > 0
    nsub = -(-C // band)
    ncoarse = -(-rg[2] // coarse)
    L1 = rng.nsamp_dec - rmax
    bands = [list(range(b * band, min(C, (b + 1) * band))) for b in range(nsub)]
    ref = [bb[-1] if foff > 0 else bb[0] for bb in bands]
    # stage 1 at every coarse trial's middle DM, stage 2 at every fine DM
    z = np.zeros((nsub, ncoarse, L1), np.int64)
    for j in range(ncoarse):
        nj = min(coarse, rg[2] - j * coarse)
        dm_c = rng.dms[j * coarse + (nj - 1) // 2]
        rel = oracle.subband_rel(C, fch1, foff, ts, dm_c, rg[3], band)
        for b, bb in enumerate(bands):
            for c in bb:
                z[b, j] += xr[c, rel[c]:rel[c] + L1]
    for i in range(rg[2]):
        j = i // coarse
        want = np.zeros(L, np.int64)
        for b in range(nsub):
            s = int(rng.shifts[i][ref[b]])
            want += z[b, j, s:s + L]
        assert np.array_equal(y[i], want), i


def test_smearing_bound(oracle):
    """|eff(i,c) - s(c,i)| <= k_DM |DM_i - D_j| (delta_c - delta_ref)/(tsamp dec) + 1.5
    (three roundings of half a sample each)."""
    C, fch1, foff, ts, T = 256, 1500.0, -1.171875, 64e-6, 1 << 14
    for rg, band, coarse in [((0.0, 1.0, 100, 1), 32, 16), ((100.0, 2.0, 50, 4), 8, 4)]:
        rng = _range(oracle, C, fch1, foff, ts, rg, T)
        eff, _, _ = oracle.subband_delays(C, fch1, foff, ts, rng, band, coarse)
        f = fch1 + np.arange(C) * foff
        ft = f.max()
        delta = 1 / f ** 2 - 1 / ft ** 2
        ref = (np.arange(C) // band) * band
        for i in range(rg[2]):
            j = i // coarse
            nj = min(coarse, rg[2] - j * coarse)
            dmj = rng.dms[j * coarse + (nj - 1) // 2]
            bound = K_DM * abs(rng.dms[i] - dmj) * (delta - delta[ref]) / (ts * rg[3]) + 1.5
            err = np.abs(eff[i] - rng.shifts[i].astype(np.int64))
            assert (err <= bound + 1e-9).all(), i
        # coarse trials of one fine trial: rounding only
        eff1, _, _ = oracle.subband_delays(C, fch1, foff, ts, rng, band, 1)
        assert np.abs(eff1 - rng.shifts.astype(np.int64)).max() <= 1


def test_library_plan_agrees_on_effective_maxshift(oracle):
    C, fch1, foff, ts, T = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    p = Plan(C, fch1, foff, ts, ranges)
    opl = oracle.plan(C, fch1, foff, ts, ranges, T)
    for r, (rg, band, coarse) in enumerate(zip(ranges, [64, 32, 16, 8], [16, 5, 16, 2])):
        p.set_subband(r, band, coarse)
        info = abi.aa_plan_range(p.handle, T, r)
        _, rmax, s2max = oracle.subband_delays(C, fch1, foff, ts, opl[r], band, coarse)
        assert info.strategy == abi.AA_DEDISP_SUBBAND
        assert info.maxshift == rmax + s2max
        assert info.length == max(0, T // rg[3] - rmax - s2max)
        assert (info.subband_channels, info.subband_coarse_trials) == (band, coarse)
        nsub, ncoarse = -(-C // band), -(-rg[2] // coarse)
        assert info.subband_work == pytest.approx((ncoarse * C + rg[2] * nsub) / (rg[2] * C))
    p.set_strategy(0, abi.AA_DEDISP_DIRECT)  # back to the exact sum and its length
    assert abi.aa_plan_range(p.handle, T, 0).length == opl[0].length


def test_set_subband_argument_checks():
    p = Plan(100, 1400.0, -2.0, 64e-6, [(0.0, 3.0, 37, 1), (100.0, 5.0, 9, 8)])
    for args, code in [((2, 16, 8), "AA_ERR_ARG"), ((0, 0, 8), "AA_ERR_ARG"),
                       ((0, 101, 8), "AA_ERR_ARG"), ((0, 16, 0), "AA_ERR_ARG"),
                       ((0, 16, 17), "AA_ERR_ARG"), ((0, 129, 8), "AA_ERR_ARG"),
                       ((1, 33, 8), "AA_ERR_CONFIG")]:
        with pytest.raises(abi.AAError, match=code):
            p.set_subband(*args)
    p.set_subband(1, 32, 8)  # 32 * 255 * 8 = 65280 fits 16 bits
