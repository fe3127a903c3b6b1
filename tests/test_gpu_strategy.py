"""The two dedispersion strategies (direct shift-and-sum; delay-pattern
groups summed once per block of 16 trials) through the C ABI: bit-identical
to each other and to the oracle, on plans chosen so the grouped strategy has
large groups (fine DM steps), singleton groups (coarse steps), ragged chunks
and blocks, decimated inputs, and in the persistent batched kernel."""
import numpy as np
import pytest
import torch

from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan

pytestmark = pytest.mark.gpu


def _dedisperse_with(plan, x, strategy):
    for r in range(len(plan.ranges)):
        info = abi.aa_plan_range(plan.handle, x.shape[1], r)
        if strategy == abi.AA_DEDISP_GROUPED:
            assert info.grouped_available == 1
        plan.set_strategy(r, strategy)
        assert abi.aa_plan_range(plan.handle, x.shape[1], r).strategy == strategy
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    return out, nsamp


def _check_plan(oracle, C, fch1, foff, ts, ranges, x):
    plan = Plan(C, fch1, foff, ts, ranges)
    direct, nsamp = _dedisperse_with(plan, x, abi.AA_DEDISP_DIRECT)
    grouped, _ = _dedisperse_with(plan, x, abi.AA_DEDISP_GROUPED)
    _, ys = oracle.dedisperse(x, C, fch1, foff, ts, plan.ranges)
    for r, (gv, dv, o) in enumerate(zip(plan.range_views(grouped, nsamp),
                                        plan.range_views(direct, nsamp), ys)):
        g = gv.double().cpu().numpy()
        assert np.array_equal(g, dv.double().cpu().numpy()), f"range {r}: strategies differ"
        assert np.array_equal(g, o.astype(np.float64)), f"range {r}: grouped differs from oracle"
    return plan


def test_fine_steps_large_groups(oracle):
    """Fine DM steps over a wide band: most channels of a chunk share their
    delay pattern (few, large groups); 4096 channels = 64 full chunks."""
    C, fch1, foff, ts, nsamp = 4096, 1508.0, -0.0732421875, 64e-6, 6000
    ranges = [(0.0, 0.1, 40, 1), (150.0, 0.2, 19, 2), (600.0, 1.0, 17, 8)]
    rng = np.random.default_rng(11)
    x = rng.integers(0, 256, size=(C, nsamp), dtype=np.uint8)
    plan = _check_plan(oracle, C, fch1, foff, ts, ranges, x)
    for r in range(3):
        assert abi.aa_plan_range(plan.handle, nsamp, r).grouped_work < 0.6


def test_coarse_steps_singleton_groups(oracle):
    """Coarse DM steps: nearly every channel has its own pattern; ragged
    channel count (not a multiple of the chunk), ragged trial count and
    length, a decimation built from another, saturated samples."""
    C, fch1, foff, ts, nsamp = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    rng = np.random.default_rng(12)
    x = rng.integers(0, 256, size=(C, nsamp), dtype=np.uint8)
    x[:, 4000:4100] = 255
    plan = _check_plan(oracle, C, fch1, foff, ts, ranges, x)
    assert abi.aa_plan_range(plan.handle, nsamp, 0).grouped_work > 0.9  # nearly all singletons


def test_synthetic_workload_with_pulses(oracle):
    """The 256-channel workload (its pulse included) under both strategies."""
    w = synth.PLAIN_256
    x = synth.make_filterbank(
        w, synth.pulses_single(),
        lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    _check_plan(oracle, w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, x)


def test_grouped_has_no_staging_waits():
    """The grouped kernel reads its rows from global memory and has no
    device-side waits: the staging-fault injection (which makes the direct
    kernel time out) leaves it correct."""
    C, nsamp = 256, 4096
    p = Plan(C, 1500.0, -1.171875, 64e-6, [(0.0, 0.05, 16, 1)])
    p.set_strategy(0, abi.AA_DEDISP_GROUPED)
    x = np.full((C, nsamp), 7, np.uint8)
    d, n = p.device_input(x)
    info = p.query(n)
    ws = p.alloc_workspace(info.dedisp_ws_bytes)
    out = p.alloc_output(n)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        abi.aa_debug_inject(2, 20_000_000)  # 20 ms
        abi.aa_debug_inject(1, 1)           # chunk 1 of the direct kernel never staged
        p.dedisperse_device(d, n, out=out, ws=ws)
        assert abi.aa_workspace_status(ws.data_ptr(), stream) == abi.AA_OK
    finally:
        abi.aa_debug_inject(0, 0)
    torch.cuda.synchronize()
    assert torch.all(p.range_views(out, n)[0] == 7 * C)


@pytest.mark.parametrize("branches", [8, 0], ids=["branches", "persistent"])
def test_grouped_in_batch(branches):
    """Grouped and direct ranges side by side in a batch (each beam's kernels
    on graph branches, or the persistent batched kernel); every beam's
    candidates equal those of the beam searched alone."""
    from paper_1912_07704_gb300.api import Batch, candidates_from_device
    C, fch1, foff, ts, W, thr = 1024, 1508.0, -0.29296875, 64e-6, 32, 4.5
    rng = np.random.default_rng(13)
    specs = [([(0.0, 0.1, 33, 1), (100.0, 0.5, 20, 2)], 20000),
             ([(0.0, 2.0, 18, 1)], 16384)]
    plans, xs = [], []
    for i, (ranges, nsamp) in enumerate(specs):
        p = Plan(C, fch1, foff, ts, ranges)
        if i == 0:
            p.set_strategy(0, abi.AA_DEDISP_GROUPED)
            p.set_strategy(1, abi.AA_DEDISP_DIRECT)
        plans.append(p)
        xs.append(rng.integers(0, 256, size=(C, nsamp), dtype=np.uint8))
    alone = []
    for p, x in zip(plans, xs):
        d, n = p.device_input(x)
        out = p.dedisperse_device(d, n)
        cands, count, _ = p.sps_search_device(out, n, W, thr, 1 << 16)
        torch.cuda.synchronize()
        alone.append(candidates_from_device(cands, count, 1 << 16))
    b = Batch(plans, [x.shape[1] for x in xs], W, thr, capacity=1 << 18)
    b.set_branches(branches)
    for i, x in enumerate(xs):
        b.input_view(i)[:, : x.shape[1]].copy_(torch.from_numpy(x))
    b.run()
    arr, total = b.candidates()
    assert total == sum(len(a) for a in alone)
    for i, ref in enumerate(alone):
        got = arr[arr["reserved"] == i].copy()
        got["reserved"] = 0
        assert len(ref) > 0 and np.array_equal(got, ref), f"beam {i}"
    b.close()
