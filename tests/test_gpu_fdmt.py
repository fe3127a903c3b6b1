"""FDMT-style tree dedispersion on the GPU (one launch per depth of the
channel tree) against the oracle's tree form: bit-exact rows for ragged,
decimated, rising-band and 4096-channel plans, the single-pulse search on
tree rows against the oracle's search, and mixed tree / exact ranges."""
import numpy as np
import pytest
import torch

from gpu_common import compare_candidate_lists, oracle_candidates, run_gpu
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan

pytestmark = pytest.mark.gpu


def _check(oracle, C, fch1, foff, ts, ranges, x, fdmt_ranges, W=40, thr=6.0):
    plan = Plan(C, fch1, foff, ts, ranges)
    for r in fdmt_ranges:
        plan.set_fdmt(r)
    out, snr, got, total, nsamp = run_gpu(plan, x, W, thr)
    pl = oracle.plan(C, fch1, foff, ts, ranges, x.shape[1])
    compared = 0
    for r, (g, v) in enumerate(zip(pl, plan.range_views(out, nsamp))):
        if r in fdmt_ranges:
            y, _ = oracle.dedisperse_fdmt(x, C, fch1, foff, ts, g)
        else:
            _, ys = oracle.dedisperse(x, C, fch1, foff, ts, [ranges[r]])
            y = ys[0]
        assert np.array_equal(v.double().cpu().numpy(), y.astype(np.float64)), f"range {r}"
        rows = {i: y[i] for i in range(y.shape[0])}
        solid, fragile, _ = oracle_candidates(oracle, rows, W, thr, g.dm_offset, r)
        compared += compare_candidate_lists(got[got["range"] == r], solid, fragile)
    plan.close()
    return compared


def test_fdmt_ragged_decimated(oracle):
    C, fch1, foff, ts, T = 100, 1450.0, -3.0, 64e-6, 20011
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (137.0, 5.0, 10, 3), (187.0, 8.0, 19, 8)]
    w = synth.Workload("fdmt", C, fch1, foff, ts, T, tuple(ranges), 40, 6.0, 90)
    x = synth.make_filterbank(w, [synth.Pulse(20.0, 3000, 8, 30.0), synth.Pulse(200.0, 9000, 32, 10.0)],
                              lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
    assert _check(oracle, C, fch1, foff, ts, ranges, x, [0, 1, 2, 3]) > 0


def test_fdmt_mixed_with_exact_ranges_rising_band(oracle):
    C, fch1, foff, ts, T = 37, 1200.0, 2.5, 64e-6, 9001
    ranges = [(0.0, 5.0, 20, 1), (100.0, 7.0, 9, 2)]
    rng = np.random.default_rng(91)
    x = rng.integers(0, 256, size=(C, T), dtype=np.uint8)
    x[:, 4000:4003] = 255
    _check(oracle, C, fch1, foff, ts, ranges, x, [1])
    _check(oracle, C, fch1, foff, ts, ranges, x, [0])


def test_fdmt_4096_channels(oracle):
    """The 4096-channel band (12 tree depths), fine and coarse DM steps."""
    C, fch1, foff, ts, T = 4096, 1508.0, -0.0732421875, 64e-6, 12000
    ranges = [(0.0, 0.1, 40, 1), (600.0, 1.0, 17, 8)]
    rng = np.random.default_rng(92)
    x = rng.integers(0, 256, size=(C, T), dtype=np.uint8)
    plan = Plan(C, fch1, foff, ts, ranges)
    plan.set_fdmt(0)
    plan.set_fdmt(1)
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    pl = oracle.plan(C, fch1, foff, ts, ranges, T)
    for r, (g, v) in enumerate(zip(pl, plan.range_views(out, nsamp))):
        y, _ = oracle.dedisperse_fdmt(x, C, fch1, foff, ts, g)
        assert np.array_equal(v.double().cpu().numpy(), y.astype(np.float64)), f"range {r}"
    # the host path runs the same tree
    dd = plan.dedisperse(x)
    host = dd.to_tensor()
    for a, b in zip(plan.range_views(host, nsamp), plan.range_views(out, nsamp)):
        assert torch.equal(a, b)
    dd.close()
    plan.close()


def test_fdmt_refused_where_not_striped(oracle):
    C, T = 64, 4096
    plan = Plan(C, 1400.0, -4.0, 64e-6, [(0.0, 4.0, 16, 1)])
    plan.set_fdmt(0)
    with pytest.raises(abi.AAError):
        plan.fused_ws_bytes(T, 32)
    plan.close()
