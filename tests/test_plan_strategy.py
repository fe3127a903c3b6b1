"""Host-side strategy selection (no GPU): which ranges get the grouped
dedispersion, the work it saves, and the checks of aa_plan_set_strategy."""
import pytest

from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan


def test_ska_plan_selects_grouped():
    w = synth.SKA_4096
    p = Plan.from_workload(w)
    for r in range(len(w.ranges)):
        info = abi.aa_plan_range(p.handle, w.nsamp, r)
        assert info.grouped_available == 1
        # fine DM steps: about a third to a half of the direct adds
        assert 0.25 < info.grouped_work < 0.5, (r, info.grouped_work)
        assert info.strategy == abi.AA_DEDISP_GROUPED
        assert info.tile_dms == 16 and info.tile_samples == 512
        assert info.smem_bytes <= 113 * 1024  # two CTAs per SM


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
    assert info.grouped_available == 1 and info.stage_channels == 64
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
