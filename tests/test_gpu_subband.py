"""Sub-band dedispersion (AA_DEDISP_SUBBAND) through the C ABI: bit-exact
against the oracle's effective-delay sum on ragged multi-range plans (partial
last band and coarse trial, decimations 2 / 3 / 4), a rising band, one-channel
bands (the brute-force result), the host path, and the single-pulse search on
sub-band output against the oracle's search of the oracle's rows."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, oracle_candidates, run_gpu
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan

pytestmark = pytest.mark.gpu


def _device(plan, x):
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    return out, nsamp


def _check(oracle, C, fch1, foff, ts, ranges, x, cfg):
    plan = Plan(C, fch1, foff, ts, ranges)
    for r, (band, coarse) in enumerate(cfg):
        if band:
            plan.set_subband(r, band, coarse)
    out, nsamp = _device(plan, x)
    opl = oracle.plan(C, fch1, foff, ts, ranges, nsamp)
    for r, (v, (band, coarse)) in enumerate(zip(plan.range_views(out, nsamp), cfg)):
        if band:
            want, *_ = oracle.dedisperse_subband(x, C, fch1, foff, ts, opl[r], band, coarse)
        else:
            want = np.stack([oracle.dedisperse_row(oracle.range_input(x, opl[r].dec), opl[r].shifts[i],
                                                   0, opl[r].length) for i in range(opl[r].ndm)])
        assert v.shape == want.shape, (r, tuple(v.shape), want.shape)
        assert np.array_equal(v.double().cpu().numpy(), want.astype(np.float64)), f"range {r}"
    return plan, out, nsamp


def test_ragged_multirange(oracle):
    C, fch1, foff, ts, T = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    x = np.random.default_rng(41).integers(0, 256, size=(C, T), dtype=np.uint8)
    _check(oracle, C, fch1, foff, ts, ranges, x, [(64, 16), (48, 5), (24, 16), (40, 2)])
    # mixed: sub-band and exact ranges in one plan
    _check(oracle, C, fch1, foff, ts, ranges, x, [(0, 0), (16, 16), (0, 0), (8, 1)])


def test_rising_band_and_saturation(oracle):
    C, fch1, foff, ts, T = 96, 1300.0, 2.0, 64e-6, 12000
    ranges = [(0.0, 2.0, 40, 1), (80.0, 4.0, 16, 2)]
    x = np.random.default_rng(42).integers(0, 256, size=(C, T), dtype=np.uint8)
    x[:, 5000:5100] = 255  # saturated block: largest partial sums
    _check(oracle, C, fch1, foff, ts, ranges, x, [(96, 16), (64, 8)])


def test_one_channel_bands_equal_brute_force(oracle):
    C, fch1, foff, ts, T = 64, 1400.0, -4.0, 64e-6, 8000
    ranges = [(0.0, 4.0, 33, 1), (132.0, 6.0, 17, 2)]
    x = np.random.default_rng(43).integers(0, 256, size=(C, T), dtype=np.uint8)
    sub, out_s, nsamp = _check(oracle, C, fch1, foff, ts, ranges, x, [(1, 16), (1, 4)])
    exact = Plan(C, fch1, foff, ts, ranges)
    out_e, _ = _device(exact, x)
    for a, b in zip(sub.range_views(out_s, nsamp), exact.range_views(out_e, nsamp)):
        assert torch.equal(a, b)


def test_host_path_and_search(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(w, synth.pulses_single(),
                              lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    plan = Plan(w.nchans, w.fch1, w.foff, w.tsamp, list(w.ranges))
    plan.set_subband(0, 32, 16)
    out, snr, gpu_c, total, nsamp = run_gpu(plan, x, w.max_width, w.threshold)
    opl = oracle.plan(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, nsamp)
    y, *_ = oracle.dedisperse_subband(x, w.nchans, w.fch1, w.foff, w.tsamp, opl[0], 32, 16)
    assert np.array_equal(plan.range_views(out, nsamp)[0].double().cpu().numpy(), y.astype(np.float64))
    rows = {i: y[i] for i in range(y.shape[0])}
    solid, fragile, B = oracle_candidates(oracle, rows, w.max_width, w.threshold, 0, 0)
    check_snr_rows(plan.range_views(snr, nsamp)[0], rows, B)
    assert compare_candidate_lists(gpu_c, solid, fragile) > 0  # the pulse is still found
    dd = plan.dedisperse(x)
    host_c, host_total = plan.sps_search(dd, w.max_width, w.threshold, capacity=1 << 16)
    assert host_total == total and np.array_equal(host_c, gpu_c)


def test_batch_refuses_subband():
    p = Plan(64, 1400.0, -4.0, 64e-6, [(0.0, 4.0, 20, 1)])
    p.set_subband(0, 16, 4)
    from paper_1912_07704_gb300.api import Batch
    with pytest.raises(abi.AAError, match="AA_ERR_CONFIG"):
        Batch([p], [8000], 16, 6.0, capacity=1024)


def test_many_bands_staged_in_chunks(oracle):
    """512 bands: stage 2 stages its band windows in several chunks."""
    C, fch1, foff, ts, T = 1024, 1500.0, -0.29296875, 64e-6, 6000
    ranges = [(0.0, 0.5, 40, 1), (20.0, 1.0, 9, 2)]
    x = np.random.default_rng(44).integers(0, 256, size=(C, T), dtype=np.uint8)
    _check(oracle, C, fch1, foff, ts, ranges, x, [(2, 16), (3, 7)])
