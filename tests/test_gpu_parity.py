"""CUDA path (through the C ABI) against the CPU oracle.

Dedispersion must be bit-exact; B(t) within 1e-4 absolute of the FP64
oracle; candidate lists identical away from fragile decisions (oracle
flags); widths equal where the width argmax is not a near-tie.
"""
import hashlib

import numpy as np
import pytest
import torch

from gpu_common import (SNR_TOL, check_snr_rows, compare_candidate_lists, oracle_candidates,
                        run_gpu)
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _full_parity(oracle, plan, x, W, thr, capacity=1 << 16):
    C = x.shape[0]
    out, snr, gpu_c, total, nsamp = run_gpu(plan, x, W, thr, capacity)
    assert total <= capacity
    pl, ys = oracle.dedisperse(x, C, plan.fch1, plan.foff, plan.tsamp, plan.ranges)
    dd_views = plan.range_views(out, nsamp)
    snr_views = plan.range_views(snr, nsamp)
    n_solid = 0
    for r, (g, o) in enumerate(zip(dd_views, ys)):
        assert g.shape == o.shape
        gd = g.double().cpu().numpy()
        assert np.array_equal(gd, o.astype(np.float64)), f"range {r}: dedispersion differs"
        rows = {i: o[i] for i in range(o.shape[0])}
        solid, fragile, B = oracle_candidates(oracle, rows, W, thr, pl[r].dm_offset, r)
        check_snr_rows(snr_views[r], rows, B)
        sel = gpu_c[gpu_c["range"] == r]
        n_solid += compare_candidate_lists(sel, solid, fragile)
    return n_solid


def make_plan(C, fch1, foff, tsamp, ranges):
    return Plan(C, fch1, foff, tsamp, ranges)


def test_plain_256_full(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(
        w, synth.pulses_single(),
        lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    p = make_plan(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges)
    n = _full_parity(oracle, p, x, w.max_width, w.threshold)
    assert n > 0  # the injected pulse produces candidates that were compared


def test_ragged_multirange_full(oracle):
    """Channels not a multiple of the stage, DM counts not a multiple of the
    DM block, ragged length, widths not a multiple of the slot count, and a
    decimation (3) that is not built from another one."""
    C, fch1, foff, ts = 100, 1400.0, -2.0, 64e-6
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (137.0, 5.0, 10, 3), (187.0, 8.0, 19, 8)]
    nsamp = 20011
    w = synth.Workload("ragged", C, fch1, foff, ts, nsamp, tuple(ranges), 50, 5.0, 7)
    pulses = [synth.Pulse(30.0, 3000, 8, 25.0), synth.Pulse(160.0, 9000, 40, 12.0),
              synth.Pulse(250.0, 15000, 3, 30.0)]
    x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
    p = make_plan(C, fch1, foff, ts, ranges)
    n = _full_parity(oracle, p, x, 50, 5.0)
    assert n > 0


def test_exact_fallback_tiles(oracle):
    """Blocks of fully saturated / empty samples push tile partial sums past
    2^24, which forces the int64 boxcar path."""
    C, nsamp = 4096, 9000
    x = np.zeros((C, nsamp), np.uint8)
    for b in range(0, nsamp, 128):
        if (b // 128) % 2 == 0:
            x[:, b:b + 64] = 255
    x[:, 5000:5003] = 200
    p = make_plan(C, 1508.0, -0.0732421875, 64e-6, [(0.0, 0.0, 3, 1), (0.0, 0.5, 2, 2)])
    _full_parity(oracle, p, x, 300, 1.5)


def test_single_channel_and_wide_boxcar(oracle):
    """One channel (no delays at all) and W larger than the series."""
    rng = np.random.default_rng(11)
    x = rng.integers(0, 256, (1, 700), dtype=np.uint8)
    p = make_plan(1, 1400.0, -1.0, 64e-6, [(0.0, 10.0, 5, 1), (0.0, 1.0, 3, 4)])
    _full_parity(oracle, p, x, 1000, 2.0)


def test_constant_input_has_no_candidates(oracle):
    x = np.full((64, 5000), 77, np.uint8)
    p = make_plan(64, 1400.0, -1.0, 64e-6, [(0.0, 20.0, 20, 1), (0.0, 20.0, 4, 2)])
    out, snr, gpu_c, total, nsamp = run_gpu(p, x, 16, -1.0)
    assert total == 0
    for v in p.range_views(snr, nsamp):
        assert torch.all(v == 0)
    for r, v in enumerate(p.range_views(out, nsamp)):
        dec = p.ranges[r][3]
        assert torch.all(v == 77.0 * 64 * dec)


def test_saturated_input_exact():
    """Largest sums the plan allows (4096 ch x 255 x dec 8) stay exact."""
    x = np.full((4096, 6000), 255, np.uint8)
    p = Plan(4096, 1508.0, -0.0732421875, 64e-6, [(0.0, 1.0, 17, 8), (0.0, 0.3, 5, 1)])
    out, snr, gpu_c, total, nsamp = run_gpu(p, x, 8, 6.0)
    v = p.range_views(out, nsamp)
    assert torch.all(v[0] == 4096.0 * 255 * 8)
    assert torch.all(v[1] == 4096.0 * 255)
    assert total == 0


def test_empty_and_short_inputs(oracle):
    p = Plan(32, 1400.0, -4.0, 64e-6, [(0.0, 50.0, 10, 1), (0.0, 50.0, 10, 4)])
    lay = p.layout(1000)
    for nsamp in (0, 1, lay[0].maxshift, lay[0].maxshift + 1, 4 * lay[1].maxshift + 5):
        x = np.random.default_rng(nsamp).integers(0, 256, (32, max(nsamp, 1)), dtype=np.uint8)
        x = x[:, :nsamp]
        if nsamp == 0:
            info = p.query(0, 8)
            assert info.dd_elems >= 0 and info.dm_trial_samples == 0
            continue
        out, snr, gpu_c, total, n = run_gpu(p, x, 8, 3.0)
        pl, ys = oracle.dedisperse(x, 32, 1400.0, -4.0, 64e-6, p.ranges)
        for g, o in zip(p.range_views(out, n), ys):
            assert g.shape == o.shape
            assert np.array_equal(g.double().cpu().numpy(), o.astype(np.float64))


def test_candidate_capacity_overflow():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, (16, 4000), dtype=np.uint8)
    p = Plan(16, 1400.0, -1.0, 64e-6, [(0.0, 1.0, 8, 1)])
    out, snr, gpu_c, total, nsamp = run_gpu(p, x, 4, 0.5, capacity=3)
    assert total > 3 and len(gpu_c) == 3
    dd = p.dedisperse(x)
    arr, tot = p.sps_search(dd, 4, 0.5, capacity=3)
    assert tot == total and len(arr) == 3
    dd.close()


def test_host_path_matches_device_path_and_keeps_input(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(
        w, synth.pulses_single(),
        lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    pinned = torch.from_numpy(x).pin_memory()
    digest = hashlib.sha256(pinned.numpy().tobytes()).hexdigest()
    p = Plan.from_workload(w)
    out, snr, gpu_c, total, nsamp = run_gpu(p, x, w.max_width, w.threshold)
    dd = p.dedisperse(pinned.numpy())
    assert hashlib.sha256(pinned.numpy().tobytes()).hexdigest() == digest
    host_out = dd.to_tensor()
    for a, b in zip(p.range_views(host_out, nsamp), p.range_views(out, nsamp)):
        assert torch.equal(a, b)
    arr, tot = p.sps_search(dd, w.max_width, w.threshold)
    assert tot == total
    assert np.array_equal(arr, gpu_c)
    dd.close()


def test_bounded_wait_reports_timeout():
    """A staging copy that is never issued makes every CTA give up after the
    wait limit; the host reads AA_ERR_TIMEOUT and the next run is clean."""
    rng = np.random.default_rng(5)
    x = rng.integers(0, 256, (64, 6000), dtype=np.uint8)
    p = Plan(64, 1400.0, -1.0, 64e-6, [(0.0, 5.0, 16, 1)])
    d, nsamp = p.device_input(x)
    info = p.query(nsamp)
    ws = p.alloc_workspace(info.dedisp_ws_bytes)
    out = p.alloc_output(nsamp)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        abi.aa_debug_inject(2, 20_000_000)  # 20 ms
        abi.aa_debug_inject(1, 1)           # chunk 1 never staged
        p.dedisperse_device(d, nsamp, out=out, ws=ws)
        assert abi.aa_workspace_status(ws.data_ptr(), stream) == abi.AA_ERR_TIMEOUT
    finally:
        abi.aa_debug_inject(0, 0)
    p.dedisperse_device(d, nsamp, out=out, ws=ws)
    assert abi.aa_workspace_status(ws.data_ptr(), stream) == abi.AA_OK
    ref = p.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    assert torch.equal(p.range_views(out, nsamp)[0], p.range_views(ref, nsamp)[0])


def test_plan_create_destroy_no_leak():
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(100):
        p = Plan(256, 1500.0, -1.171875, 64e-6, [(0.0, 1.0, 256, 1)])
        p.bind()
        p.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (8 << 20)
