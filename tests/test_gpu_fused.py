"""Fused dedispersion -> single-pulse search (stripes of trials, statistics
summed by the dedispersion kernels): bit for bit the unfused path's
candidates and B(t), for both dedispersion strategies, ragged and decimated
plans, stripe sizes from one DM block to more than a range, clipped
statistics and the width ladder; the device ordering works on its search
workspace; and one plan against the oracle."""
import numpy as np
import pytest
import torch

from gpu_common import SNR_TOL, check_snr_rows, compare_candidate_lists, oracle_candidates
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu

RAGGED = (100, 1450.0, -3.0, 64e-6, 20011,
          [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (137.0, 5.0, 10, 3), (187.0, 8.0, 19, 8)])


def _data(oracle, C, fch1, foff, ts, T, ranges, seed):
    w = synth.Workload("fused", C, fch1, foff, ts, T, tuple(ranges), 50, 6.0, seed)
    pulses = [synth.Pulse(ranges[0][0] + 3 * ranges[0][1], T // 4, 8, 30.0),
              synth.Pulse(ranges[-1][0] + 2 * ranges[-1][1], T // 2, 24, 12.0)]
    return synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()


def _unfused(plan, d, nsamp, W, thr, cap, snr=True):
    out = plan.dedisperse_device(d, nsamp)
    s = torch.full_like(out, float("nan")) if snr else None
    info = plan.query(nsamp, W)
    ws = plan.alloc_workspace(info.sps_ws_bytes)
    cands, count, _ = plan.sps_search_device(out, nsamp, W, thr, cap, snr_out=s, ws=ws)
    torch.cuda.synchronize()
    return candidates_from_device(cands, count, cap), int(count.item()), s, ws, cands, count


def _fused(plan, d, nsamp, W, thr, cap, stripe, snr=True):
    s = torch.full((plan.query(nsamp).dd_elems,), float("nan"), device="cuda") if snr else None
    cands, count, ws = plan.search_fused_device(d, nsamp, W, thr, cap, stripe, snr_out=s)
    torch.cuda.synchronize()
    assert abi.aa_workspace_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream) == abi.AA_OK
    return candidates_from_device(cands, count, cap), int(count.item()), s, ws, cands, count


def _equal_snr(plan, nsamp, a, b):
    for va, vb in zip(plan.range_views(a, nsamp), plan.range_views(b, nsamp)):
        assert torch.equal(va, vb)


@pytest.mark.parametrize("strategy", [abi.AA_DEDISP_GROUPED, abi.AA_DEDISP_DIRECT])
@pytest.mark.parametrize("stripe", [16, 48, 0, 4096])
def test_fused_equals_unfused(oracle, strategy, stripe):
    C, fch1, foff, ts, T, ranges = RAGGED
    x = _data(oracle, C, fch1, foff, ts, T, ranges, 81)
    plan = Plan(C, fch1, foff, ts, ranges)
    for r in range(len(ranges)):
        if strategy != abi.AA_DEDISP_GROUPED or abi.aa_plan_range(plan.handle, T, r).grouped_available:
            plan.set_strategy(r, strategy)
    d, nsamp = plan.device_input(x)
    W, thr, cap = 50, 6.0, 1 << 16
    ref, nref, sref, *_ = _unfused(plan, d, nsamp, W, thr, cap)
    got, ngot, sgot, *_ = _fused(plan, d, nsamp, W, thr, cap, stripe)
    assert nref > 0 and ngot == nref and np.array_equal(got, ref)
    _equal_snr(plan, nsamp, sref, sgot)
    # the pruned form (no B output), as the benchmark runs it
    got2, n2, *_ = _fused(plan, d, nsamp, W, thr, cap, stripe, snr=False)
    assert n2 == nref and np.array_equal(got2, ref)
    plan.close()


def test_fused_4096_channels_grouped_chunks(oracle):
    """Wide channel chunks of the grouped strategy (4096 channels, fine DM
    steps) and decimations 1/2/8, stripes of 32 trials."""
    C, fch1, foff, ts, T = 4096, 1508.0, -0.0732421875, 64e-6, 6000
    ranges = [(0.0, 0.1, 40, 1), (150.0, 0.2, 19, 2), (600.0, 1.0, 17, 8)]
    rng = np.random.default_rng(11)
    x = rng.integers(0, 256, size=(C, T), dtype=np.uint8)
    plan = Plan(C, fch1, foff, ts, ranges)
    d, nsamp = plan.device_input(x)
    W, thr, cap = 64, 3.5, 1 << 18
    ref, nref, sref, *_ = _unfused(plan, d, nsamp, W, thr, cap)
    got, ngot, sgot, *_ = _fused(plan, d, nsamp, W, thr, cap, 32)
    assert nref > 0 and ngot == nref and np.array_equal(got, ref)
    _equal_snr(plan, nsamp, sref, sgot)
    plan.close()


def test_fused_clipped_statistics_and_ladder(oracle):
    C, fch1, foff, ts, T, ranges = RAGGED
    x = _data(oracle, C, fch1, foff, ts, T, ranges, 82)
    x[:, 5000:5003] = 255  # broadband spike: the clipping has something to do
    plan = Plan(C, fch1, foff, ts, ranges)
    plan.set_sps_clip(40, 3)
    d, nsamp = plan.device_input(x)
    W, thr, cap = 50, 6.0, 1 << 16
    ref, nref, sref, *_ = _unfused(plan, d, nsamp, W, thr, cap)
    got, ngot, sgot, *_ = _fused(plan, d, nsamp, W, thr, cap, 16)
    assert nref > 0 and ngot == nref and np.array_equal(got, ref)
    _equal_snr(plan, nsamp, sref, sgot)
    plan.close()
    plan = Plan(C, fch1, foff, ts, ranges)
    plan.set_sps_ladder(24)
    ref, nref, *_ = _unfused(plan, d, nsamp, 400, thr, cap, snr=False)
    got, ngot, *_ = _fused(plan, d, nsamp, 400, thr, cap, 32, snr=False)
    assert nref > 0 and ngot == nref and np.array_equal(got, ref)
    plan.close()


def test_fused_device_order_and_overflow(oracle):
    C, fch1, foff, ts, T, ranges = RAGGED
    x = _data(oracle, C, fch1, foff, ts, T, ranges, 83)
    plan = Plan(C, fch1, foff, ts, ranges)
    d, nsamp = plan.device_input(x)
    W, thr, cap = 50, 6.0, 1 << 16
    ref, nref, *_ = _unfused(plan, d, nsamp, W, thr, cap, snr=False)
    got, ngot, s, ws, cands, count = _fused(plan, d, nsamp, W, thr, cap, 16, snr=False)
    off = plan.fused_ws_bytes(nsamp, W, 16)[1]
    srt = plan.sps_order_device(nsamp, W, ws[off:], cands, count, cap)
    torch.cuda.synchronize()
    dev = srt[: ngot * 16].cpu().numpy().view(synth.CANDIDATE_RECORD)
    assert np.array_equal(dev, ref)
    # overflow: the count keeps the true total
    small, nsmall, *_ = _fused(plan, d, nsamp, W, thr, 5, 16, snr=False)
    assert nsmall == nref and len(small) == 5
    plan.close()


def test_fused_against_oracle(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(
        w, synth.pulses_single(),
        lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    plan = Plan.from_workload(w)
    d, nsamp = plan.device_input(x)
    got, n, snr, *_ = _fused(plan, d, nsamp, w.max_width, w.threshold, 1 << 16, 32)
    pl, ys = oracle.dedisperse(x, w.nchans, w.fch1, w.foff, w.tsamp, w.ranges)
    y = ys[0]
    rows = {i: y[i] for i in range(y.shape[0])}
    solid, fragile, B = oracle_candidates(oracle, rows, w.max_width, w.threshold, 0, 0)
    assert compare_candidate_lists(got, solid, fragile) > 0
    check_snr_rows(plan.range_views(snr, nsamp)[0], rows, B)
    plan.close()
