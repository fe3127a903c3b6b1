"""Decimated boxcar width ladder (aa_plan_set_sps_decimated) through the C
ABI against the oracle's decimated ladder (oracle_boxcar_dec): full B(t)
rows and candidate lists on a multi-range plan with wide pulses across
several tiles, the exact int64 tile path, a 4096-channel plan at W = 8192,
the W0 >= W case against the exhaustive search, and batches."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, run_gpu
from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Batch, Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _oracle_rows(oracle, y_rows, W, thr, dm_offset, r, W0):
    solid, fragile, B = {}, set(), {}
    for i, y in y_rows.items():
        c, b, wb, mu, sg = oracle.search_row(y, W, thr, dm_offset + i, r, dec_w0=W0)
        B[i] = (0, b, wb, mu, sg)
        for cc in c:
            (fragile.add((cc.dm_index, cc.t)) if cc.fragile
             else solid.__setitem__((cc.dm_index, cc.t), cc))
    return solid, fragile, B


def _parity(oracle, plan, x, W, thr, W0, rows=None):
    plan.set_sps_decimated(W0)
    out, snr, gpu_c, total, nsamp = run_gpu(plan, x, W, thr, 1 << 18)
    pl, ys = oracle.dedisperse(x, x.shape[0], plan.fch1, plan.foff, plan.tsamp, plan.ranges, rows=rows)
    n, widths = 0, set()
    for r, o in enumerate(ys):
        idx = range(o.shape[0]) if rows is None else rows[r]
        y_rows = {i: (o[i] if rows is None else o[k]) for k, i in enumerate(idx)}
        solid, fragile, B = _oracle_rows(oracle, y_rows, W, thr, pl[r].dm_offset, r, W0)
        check_snr_rows(plan.range_views(snr, nsamp)[r], y_rows, B)
        sel = {pl[r].dm_offset + i for i in y_rows}
        mine = gpu_c[gpu_c["range"] == r]
        n += compare_candidate_lists(mine, solid, fragile, lambda dm, t: dm in sel)
        widths |= {c.width for c in solid.values()}
    return n, widths


@pytest.mark.parametrize("W0", [16, 32])
def test_dec_ladder_multirange(oracle, W0):
    C, fch1, foff, ts, T = 100, 1400.0, -2.0, 64e-6, 20011
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (187.0, 8.0, 19, 8)]
    w = synth.Workload("dec", C, fch1, foff, ts, T, tuple(ranges), 1024, 5.0, 9)
    pulses = [synth.Pulse(30.0, 4090, 300, 6.0), synth.Pulse(160.0, 8188, 40, 12.0),
              synth.Pulse(250.0, 15000, 900, 4.0), synth.Pulse(10.0, 12000, 3, 40.0)]
    x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
    n, widths = _parity(oracle, Plan(C, fch1, foff, ts, ranges), x, 1024, 5.0, W0)
    assert n > 0
    assert any(wd > W0 for wd in widths), "no candidate from a decimated level"


def test_dec_ladder_exact_tile_path(oracle):
    C, nsamp = 4096, 9000
    x = np.zeros((C, nsamp), np.uint8)
    for b in range(0, nsamp, 128):
        if (b // 128) % 2 == 0:
            x[:, b:b + 64] = 255
    x[:, 5000:5003] = 200
    p = Plan(C, 1508.0, -0.0732421875, 64e-6, [(0.0, 0.0, 3, 1), (0.0, 0.5, 2, 2)])
    _parity(oracle, p, x, 300, 1.5, 16)


def test_dec_ladder_4096ch_w8192(oracle):
    w = synth.Workload("dec-ska", 4096, 1508.0, -0.0732421875, 64e-6, 1 << 16,
                       ((0.0, 0.1, 300, 1), (150.0, 0.2, 40, 2)), 8192, 6.0, 1)
    d1 = lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)
    pulses = [synth.Pulse(12.0, 9000, 2000, 3.0), synth.Pulse(20.0, 30000, 16, 12.0),
              synth.Pulse(160.0, 50000, 4000, 2.0)]
    x = synth.make_filterbank(w, pulses, d1).numpy()
    rows = [sorted(set(range(0, 300, 23)) | {119, 120, 199, 200, 299}), list(range(40))]
    n, widths = _parity(oracle, Plan.from_workload(w), x, 8192, 6.0, 32, rows=rows)
    assert n > 0 and max(widths) > 512


def test_base_widths_covering_w_equal_exhaustive(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(w, synth.pulses_single(),
                              lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    got = []
    for W0 in (0, 64):  # W = 64 <= W0: level 0 only
        p = Plan(w.nchans, w.fch1, w.foff, w.tsamp, list(w.ranges))
        p.set_sps_decimated(W0)
        d, nsamp = p.device_input(x)
        out = p.dedisperse_device(d, nsamp)
        snr = torch.full_like(out, float("nan"))
        cands, count, _ = p.sps_search_device(out, nsamp, 64, w.threshold, 1 << 16, snr_out=snr)
        torch.cuda.synchronize()
        got.append((candidates_from_device(cands, count, 1 << 16), p.range_views(snr, nsamp)[0].cpu()))
    assert np.array_equal(got[0][0], got[1][0]) and torch.equal(got[0][1], got[1][1])
    assert len(got[0][0]) > 0


@pytest.mark.parametrize("branches", [8, 0], ids=["branches", "persistent"])
def test_dec_ladder_in_batch(oracle, branches):
    C, fch1, foff, ts, W, thr = 128, 1500.0, -2.0, 64e-6, 512, 5.0
    specs = [([(0.0, 3.0, 40, 1), (120.0, 5.0, 9, 4)], 30011), ([(0.0, 1.0, 33, 1)], 17777)]
    plans, xs, alone = [], [], []
    for k, (ranges, T) in enumerate(specs):
        wk = synth.Workload(f"b{k}", C, fch1, foff, ts, T, tuple(ranges), W, thr, 30 + k)
        pulses = [synth.Pulse(ranges[0][0] + 6.0, T // 3, 200, 5.0), synth.Pulse(ranges[0][0] + 3.0, T // 2, 4, 30.0)]
        x = synth.make_filterbank(wk, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
        p = Plan(C, fch1, foff, ts, ranges)
        p.set_sps_decimated(16)
        d, n = p.device_input(x)
        out = p.dedisperse_device(d, n)
        cands, count, _ = p.sps_search_device(out, n, W, thr, 1 << 16)
        torch.cuda.synchronize()
        alone.append(candidates_from_device(cands, count, 1 << 16))
        plans.append(p)
        xs.append(x)
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
