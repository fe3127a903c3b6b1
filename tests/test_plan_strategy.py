"""Host-side strategy selection (no GPU): which ranges get the grouped
dedispersion, the work it saves, and the checks of aa_plan_set_strategy."""
import numpy as np
import pytest

from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan


def test_ska_plan_selects_grouped():
    w = synth.SKA_4096
    p = Plan.from_workload(w)
    for r in range(len(w.ranges)):
        info = abi.aa_plan_range(p.handle, w.nsamp, r)
        assert info.grouped_available == 1
        # fine DM steps: a quarter to a half of the direct adds
        assert 0.2 < info.grouped_work < 0.5, (r, info.grouped_work)
        assert info.strategy == abi.AA_DEDISP_GROUPED
        assert info.tile_dms == 16 and info.tile_samples == 512
        assert info.smem_bytes <= 113 * 1024  # two CTAs per SM


def _pattern_work(shifts, ndm, C, cc, B=16, split=16):
    """Adds of the grouped form over those of the direct form, counting the
    distinct delay patterns of every (B-trial block, cc-channel chunk) by brute
    force (a partial block repeats its last trial); a pattern shared by n
    channels makes ceil(n / split) group sums."""
    sh = np.asarray(shifts).reshape(ndm, C)
    direct = grouped = 0
    for d0 in range(0, ndm, B):
        nb = min(B, ndm - d0)
        rows = sh[[d0 + min(d, nb - 1) for d in range(B)]]
        rel = (rows - rows[0]).T
        for c0 in range(0, C, cc):
            nch = min(cc, C - c0)
            pats = {}
            for x in rel[c0:c0 + nch]:
                pats[tuple(x)] = pats.get(tuple(x), 0) + 1
            G = sum(-(-n // split) for n in pats.values())
            direct += nch * nb
            grouped += nch + G * nb
    return grouped / direct


@pytest.mark.parametrize("ranges,C", [(synth.SKA_4096.ranges[:2], 4096),
                                      ([(0.0, 0.25, 45, 1), (11.0, 0.5, 21, 4)], 1024)])
def test_grouped_work_counts_delay_patterns(ranges, C):
    p = Plan(C, 1508.0, -300.0 / C, 64e-6, list(ranges))
    for r, rg in enumerate(ranges):
        p.set_strategy(r, abi.AA_DEDISP_GROUPED)  # stage_channels of the grouped tiles
        info = abi.aa_plan_range(p.handle, 1 << 17, r)
        # a group sum holds at most 16 members (32 for decimated input), fewer
        # when 16-bit lanes need it
        split = min(16 if rg[3] == 1 else 32, 65535 // (255 * rg[3]))
        want = _pattern_work(p.shifts(r), rg[2], C, info.stage_channels, split=split)
        assert info.grouped_work == pytest.approx(want, rel=1e-12)
        # chunks of 1024 channels for 8-bit input, 4096 for decimated 16-bit
        # input (the 16-bit lanes are flushed group by group, not per chunk)
        assert info.stage_channels == (1024 if rg[3] == 1 else 4096)


def test_coarse_plan_keeps_direct():
    w = synth.PLAIN_256  # DM step 1 over 256 channels: patterns almost all distinct
    p = Plan.from_workload(w)
    info = abi.aa_plan_range(p.handle, w.nsamp, 0)
    assert info.grouped_work > 0.9
    assert info.strategy == abi.AA_DEDISP_DIRECT
    p.set_strategy(0, abi.AA_DEDISP_GROUPED)  # available, just not chosen
    assert abi.aa_plan_range(p.handle, w.nsamp, 0).strategy == abi.AA_DEDISP_GROUPED
    p.set_strategy(0, abi.AA_DEDISP_DIRECT)
    assert abi.aa_plan_range(p.handle, w.nsamp, 0).strategy == abi.AA_DEDISP_DIRECT


def test_grouped_wide_spans_then_unavailable():
    """Wider delay spans over 16 trials make each group sum longer (fewer fit
    in shared memory per batch); beyond 4096 samples the grouped tiles are
    refused."""
    p = Plan(203, 1400.0, -1.5, 64e-6, [(0.0, 3.0, 35, 1)])  # span ~940 samples
    p.set_strategy(0, abi.AA_DEDISP_GROUPED)
    info = abi.aa_plan_range(p.handle, 9001, 0)
    assert info.grouped_available == 1 and info.stage_channels == 1024
    assert info.smem_bytes <= 113 * 1024
    p = Plan(203, 1400.0, -1.5, 64e-6, [(0.0, 15.0, 35, 1)])  # span ~4700 samples
    info = abi.aa_plan_range(p.handle, 9001, 0)
    assert info.span_max > 4096
    assert info.grouped_available == 0 and info.strategy == abi.AA_DEDISP_DIRECT
    with pytest.raises(abi.AAError, match="AA_ERR_CONFIG"):
        p.set_strategy(0, abi.AA_DEDISP_GROUPED)


def test_set_strategy_argument_checks():
    p = Plan(64, 1400.0, -1.0, 64e-6, [(0.0, 0.5, 20, 1)])
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        p.set_strategy(1, abi.AA_DEDISP_DIRECT)
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        p.set_strategy(0, 7)
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        abi.aa_plan_set_strategy(None, 0, 0)


def test_fused_workspace_replaces_the_series():
    """The fused search's workspace holds one stripe of series instead of
    the whole plan's, and one decimated input instead of all of them: on the
    4096-channel plan (series 9.18 GB, decimated inputs 7.5 GB) 256-trial
    stripes need 1.07 GB of series and 4.29 GB of decimated input (dec 2);
    stripe sizes are checked."""
    from paper_1912_07704_gb300 import synth
    w = synth.SKA_4096
    p = Plan.from_workload(w)
    info = p.query(w.nsamp, w.max_width)
    unfused = info.dd_elems * 4 + info.dedisp_ws_bytes + info.sps_ws_bytes
    fused, off = abi.aa_search_fused_ws_bytes(p.handle, w.nsamp, w.max_width, 256)
    lay = p.layout(w.nsamp)
    stripe_bytes = 256 * max(g.pitch for g in lay) * 4
    dec2 = w.nchans * 524288 * 2  # the largest decimated input
    expect = dec2 + info.sps_ws_bytes + stripe_bytes
    assert abs(fused - expect) < 1 << 20, (fused, expect)
    assert off >= dec2
    assert fused < 0.35 * unfused
    with pytest.raises(abi.AAError):
        abi.aa_search_fused_ws_bytes(p.handle, w.nsamp, w.max_width, 24)  # not a multiple of 16
    p.close()
