"""The allocation-free single-pulse search agrees with the workspace one.

aa_sps_search_device_noalloc serves callers that may not allocate device
memory while they run (a real-time loop with memory fixed at start-up, a
plug-in whose host framework owns all allocations): its scratch is a fixed
array inside the library.  Two calls in a row must each reproduce the
regular entry point's candidates and B(t) exactly (same kernels, same
input).  This file is collected last so
that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest
import torch

from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu



def _compare(a, b):
    """Both entry points run the same kernels on the same input; only where
    their scratch lives differs, so every record is identical."""
    assert len(a) == len(b)
    assert np.array_equal(a, b)


def test_noalloc_search_matches_workspace_search():
    w = synth.PLAIN_256
    plan = Plan.from_workload(w)
    delays = plan.shifts(0)[150]  # DM 150 of the plan's only range (dec 1)
    x = synth.make_filterbank(w, synth.pulses_single(), lambda dm: delays, device="cuda",
                              pitch=plan.query(w.nsamp).in_pitch_min)
    out = plan.dedisperse_device(x, w.nsamp)
    cap = 1 << 16
    snr_ref = torch.full_like(out, float("nan"))
    cands, count, _ = plan.sps_search_device(out, w.nsamp, w.max_width, w.threshold, cap,
                                             snr_out=snr_ref)
    torch.cuda.synchronize()
    ref = candidates_from_device(cands, count, cap)
    assert len(ref) > 0
    assert plan.query(w.nsamp, w.max_width).sps_ws_bytes <= (16 << 20)
    stream = torch.cuda.current_stream().cuda_stream
    views_ref = plan.range_views(snr_ref, w.nsamp)
    for _ in range(2):
        c2 = torch.zeros(cap * 16, dtype=torch.uint8, device="cuda")
        n2 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        snr2 = torch.full_like(out, float("nan"))
        st = abi.aa_sps_search_device_noalloc(plan.handle, w.nsamp, out.data_ptr(), w.max_width,
                                              w.threshold, c2.data_ptr(), cap, n2.data_ptr(),
                                              snr2.data_ptr(), stream)
        assert st == abi.AA_OK, abi.aa_last_error()
        torch.cuda.synchronize()
        assert int(n2.item()) == int(count.item())
        _compare(candidates_from_device(c2, n2, cap), ref)
        for a, b in zip(plan.range_views(snr2, w.nsamp), views_ref):
            assert torch.isfinite(a).all()
            assert torch.equal(a, b)
    plan.close()


def test_noalloc_rejects_searches_larger_than_its_scratch():
    big = Plan.from_workload(synth.SKA_4096)
    big_n = synth.SKA_4096.nsamp
    assert big.query(big_n, 8192).sps_ws_bytes > (16 << 20)
    st = abi.aa_sps_search_device_noalloc(big.handle, big_n, None, 8192, 6.0, None, 0, None,
                                          None, None)
    assert st == abi.AA_ERR_ARG
    assert "scratch" in abi.aa_last_error()
    big.close()
