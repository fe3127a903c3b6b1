"""The boxcar kernel's tile segments: a CTA searches several consecutive
tiles of a series, sliding the staged prefix sums by one tile and staging
only the new samples.  Candidates and B(t) must not depend on how many tiles
a CTA takes (forced through the test hook), including tiles on the exact
int64 path and series whose prefix sums leave the sliding range (the tile is
then staged afresh); and they match the oracle."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, oracle_candidates
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _search(plan, x, W, thr, seg, cap=1 << 18):
    abi.aa_debug_inject(3, seg)
    try:
        d, nsamp = plan.device_input(x)
        out = plan.dedisperse_device(d, nsamp)
        snr = torch.full_like(out, float("nan"))
        c1, n1, _ = plan.sps_search_device(out, nsamp, W, thr, cap, snr_out=snr)
        c2, n2, _ = plan.sps_search_device(out, nsamp, W, thr, cap)  # pruned
        torch.cuda.synchronize()
        a1 = candidates_from_device(c1, n1, cap)
        a2 = candidates_from_device(c2, n2, cap)
        assert np.array_equal(a1, a2)
        return a1, snr.cpu(), out, nsamp
    finally:
        abi.aa_debug_inject(0, 0)


def _same_for_all_segments(plan, x, W, thr, segs=(1, 2, 3, 7)):
    ref = None
    for seg in segs:
        got = _search(plan, x, W, thr, seg)
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]), f"candidates differ with {seg} tiles per CTA"
            views_a = plan.range_views(got[1], got[3])
            views_b = plan.range_views(ref[1], ref[3])
            assert all(torch.equal(u, v) for u, v in zip(views_a, views_b)), f"B(t) differs ({seg})"
    return ref


def test_segments_multirange_match_oracle(oracle):
    C, fch1, foff, ts, T = 100, 1400.0, -2.0, 64e-6, 30011
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (187.0, 8.0, 19, 8)]
    w = synth.Workload("seg", C, fch1, foff, ts, T, tuple(ranges), 1024, 5.0, 9)
    pulses = [synth.Pulse(30.0, 4090, 300, 6.0), synth.Pulse(160.0, 8188, 40, 12.0),
              synth.Pulse(10.0, 12285, 3, 40.0), synth.Pulse(60.0, 20470, 900, 3.0)]
    x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
    plan = Plan(C, fch1, foff, ts, ranges)
    cands, snr, out, nsamp = _same_for_all_segments(plan, x, 1024, 5.0)
    pl, ys = oracle.dedisperse(x, C, fch1, foff, ts, ranges)
    n = 0
    for r, o in enumerate(ys):
        rows = {i: o[i] for i in range(o.shape[0])}
        solid, fragile, B = oracle_candidates(oracle, rows, 1024, 5.0, pl[r].dm_offset, r)
        check_snr_rows(plan.range_views(snr, nsamp)[r], rows, B)
        n += compare_candidate_lists(cands[cands["range"] == r], solid, fragile)
    assert n > 0


def test_segments_exact_tile_path():
    C, nsamp = 4096, 40000
    x = np.zeros((C, nsamp), np.uint8)
    for b in range(0, nsamp, 128):
        if (b // 128) % 2 == 0:
            x[:, b:b + 64] = 255
    x[:, 25000:25003] = 200
    p = Plan(C, 1508.0, -0.0732421875, 64e-6, [(0.0, 0.0, 3, 1), (0.0, 0.5, 2, 2)])
    cands = _same_for_all_segments(p, x, 300, 1.5)[0]
    assert len(cands) > 0


def test_segments_prefix_leaves_sliding_range(oracle):
    # per-channel level 144 for the first half, 112 for the second: the row
    # sum moves 1024 per sample away from its mean, so the prefix sums pass
    # 2^23 after about two tiles and the sliding tiles are restaged
    C, T = 64, 60000
    rng = np.random.default_rng(3)
    x = np.where(np.arange(T)[None, :] < T // 2, 144, 112).astype(np.int64)
    x = np.clip(x + rng.integers(-3, 4, size=(C, T)), 0, 255).astype(np.uint8)
    x[:, 40000:40020] = 200
    ranges = [(0.0, 5.0, 4, 1)]
    p = Plan(C, 1400.0, -4.0, 64e-6, ranges)
    cands, snr, out, nsamp = _same_for_all_segments(p, x, 512, 4.0, segs=(1, 4, 16))
    pl, ys = oracle.dedisperse(x, C, 1400.0, -4.0, 64e-6, ranges)
    rows = {i: ys[0][i] for i in range(ys[0].shape[0])}
    solid, fragile, B = oracle_candidates(oracle, rows, 512, 4.0, 0, 0)
    check_snr_rows(p.range_views(snr, nsamp)[0], rows, B)
    compare_candidate_lists(cands, solid, fragile)


def test_segment_hook_arguments():
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        abi.aa_debug_inject(3, -1)
    abi.aa_debug_inject(3, 4096)
    abi.aa_debug_inject(0, 0)
