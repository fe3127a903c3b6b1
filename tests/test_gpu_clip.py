"""k-sigma clipped statistics (aa_plan_set_sps_clip) through the C ABI against
the oracle: full B(t) rows and candidate lists of data with a pulse and
broadband (zero-DM) spikes, on the 256-channel workload and on a ragged
decimated plan; the host path, the batched path and the plain statistics
after switching clipping off."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, oracle_candidates, run_gpu
from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Batch, Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _with_spikes(x, seed, n=12, amp=60):
    """Broadband spikes: +amp counts in every channel at n random samples."""
    x = x.astype(np.int64)
    t = np.random.default_rng(seed).integers(0, x.shape[1], n)
    x[:, t] += amp
    return np.clip(x, 0, 255).astype(np.uint8)


def _parity(oracle, plan, x, W, thr, clip):
    plan.set_sps_clip(*clip)
    out, snr, gpu_c, total, nsamp = run_gpu(plan, x, W, thr, 1 << 16)
    pl, ys = oracle.dedisperse(x, x.shape[0], plan.fch1, plan.foff, plan.tsamp, plan.ranges)
    n = 0
    for r, o in enumerate(ys):
        rows = {i: o[i] for i in range(o.shape[0])}
        solid, fragile, B = oracle_candidates(oracle, rows, W, thr, pl[r].dm_offset, r, clip=clip)
        check_snr_rows(plan.range_views(snr, nsamp)[r], rows, B)
        n += compare_candidate_lists(gpu_c[gpu_c["range"] == r], solid, fragile)
    return n, gpu_c


def test_clip_256_with_spikes(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(w, synth.pulses_single(),
                              lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1))
    x = _with_spikes(x.numpy(), 3)
    plan = Plan(w.nchans, w.fch1, w.foff, w.tsamp, list(w.ranges))
    n, clipped = _parity(oracle, plan, x, w.max_width, w.threshold, (48, 8))
    assert n > 0
    # switching clipping off gives the plain statistics back (a different list)
    n2, plain = _parity(oracle, plan, x, w.max_width, w.threshold, (0, 0))
    assert n2 > 0 and not np.array_equal(clipped, plain)


def test_clip_ragged_decimated(oracle):
    C, fch1, foff, ts, T = 100, 1400.0, -2.0, 64e-6, 20011
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (137.0, 5.0, 10, 3), (187.0, 8.0, 19, 8)]
    w = synth.Workload("ragged", C, fch1, foff, ts, T, tuple(ranges), 50, 5.0, 7)
    pulses = [synth.Pulse(30.0, 3000, 8, 25.0), synth.Pulse(160.0, 9000, 40, 12.0)]
    x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1))
    x = _with_spikes(x.numpy(), 4, n=30, amp=90)
    for clip in [(40, 1), (40, 3), (32, 64)]:  # k >= 2: iterated clipping keeps a stable core
        n, _ = _parity(oracle, Plan(C, fch1, foff, ts, ranges), x, 50, 5.0, clip)
        assert n > 0


def test_clip_host_and_batched_paths(oracle):
    C, fch1, foff, ts, T = 64, 1400.0, -4.0, 64e-6, 21001
    ranges = [(0.0, 4.0, 23, 1), (92.0, 6.0, 17, 2)]
    w = synth.Workload("clip-batch", C, fch1, foff, ts, T, tuple(ranges), 64, 5.0, 30)
    x = synth.make_filterbank(w, [synth.Pulse(8.0, T // 3, 6, 30.0)],
                              lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1))
    x = _with_spikes(x.numpy(), 5)
    plan = Plan(C, fch1, foff, ts, ranges)
    plan.set_sps_clip(40, 6)
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    cands, count, _ = plan.sps_search_device(out, nsamp, 64, 5.0, 1 << 16)
    torch.cuda.synchronize()
    dev = candidates_from_device(cands, count, 1 << 16)
    host, total = plan.sps_search(plan.dedisperse(x), 64, 5.0, capacity=1 << 16)
    assert total == int(count.item()) and np.array_equal(host, dev)
    b = Batch([plan, plan], [T, T], 64, 5.0, capacity=1 << 18)
    for i in range(2):
        b.input_view(i)[:, :T].copy_(torch.from_numpy(x))
    b.run()
    arr, _ = b.candidates()
    for i in range(2):
        a = arr[arr["reserved"] == i].copy()
        a["reserved"] = 0
        assert np.array_equal(a, dev)
