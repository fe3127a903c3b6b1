"""Sparse boxcar width ladder (aa_plan_set_sps_ladder) through the C ABI
against the oracle's search over the same widths: full B(t) rows and
candidate lists on a multi-range plan with W = 1024, the exact int64 tile
path, the pruned and unpruned searches, and the ladder that keeps every
chunk (equal to the exhaustive search)."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, oracle_candidates, run_gpu
from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _parity(oracle, plan, x, W, thr, g16):
    plan.set_sps_ladder(g16)
    out, snr, gpu_c, total, nsamp = run_gpu(plan, x, W, thr, 1 << 16)  # also pruned vs unpruned
    pl, ys = oracle.dedisperse(x, x.shape[0], plan.fch1, plan.foff, plan.tsamp, plan.ranges)
    n = 0
    for r, o in enumerate(ys):
        rows = {i: o[i] for i in range(o.shape[0])}
        solid, fragile, B = {}, set(), {}
        for i, y in rows.items():
            c, b, wb, mu, sg = oracle.search_row(y, W, thr, pl[r].dm_offset + i, r,
                                                 wset=oracle.ladder_widths(W, g16))
            B[i] = (0, b, wb, mu, sg)
            for cc in c:
                (fragile.add((cc.dm_index, cc.t)) if cc.fragile
                 else solid.__setitem__((cc.dm_index, cc.t), cc))
        check_snr_rows(plan.range_views(snr, nsamp)[r], rows, B)
        n += compare_candidate_lists(gpu_c[gpu_c["range"] == r], solid, fragile)
    return n, gpu_c


def test_ladder_multirange(oracle):
    C, fch1, foff, ts, T = 100, 1400.0, -2.0, 64e-6, 20011
    ranges = [(0.0, 2.0, 37, 1), (74.0, 3.0, 21, 2), (187.0, 8.0, 19, 8)]
    w = synth.Workload("ladder", C, fch1, foff, ts, T, tuple(ranges), 1024, 5.0, 9)
    pulses = [synth.Pulse(30.0, 3000, 300, 6.0), synth.Pulse(160.0, 9000, 40, 12.0),
              synth.Pulse(250.0, 15000, 900, 4.0)]
    x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, ts, dm, 1)).numpy()
    for g16 in (24, 40):
        n, _ = _parity(oracle, Plan(C, fch1, foff, ts, ranges), x, 1024, 5.0, g16)
        assert n > 0


def test_ladder_exact_tile_path(oracle):
    C, nsamp = 4096, 9000
    x = np.zeros((C, nsamp), np.uint8)
    for b in range(0, nsamp, 128):
        if (b // 128) % 2 == 0:
            x[:, b:b + 64] = 255
    x[:, 5000:5003] = 200
    p = Plan(C, 1508.0, -0.0732421875, 64e-6, [(0.0, 0.0, 3, 1), (0.0, 0.5, 2, 2)])
    _parity(oracle, p, x, 300, 1.5, 20)


def test_all_chunks_equal_exhaustive(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(w, synth.pulses_single(),
                              lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    got = []
    for g16 in (0, 17):  # 17: chunks 0..17 = widths 1..288 >= W = 256
        p = Plan(w.nchans, w.fch1, w.foff, w.tsamp, list(w.ranges))
        p.set_sps_ladder(g16)
        d, nsamp = p.device_input(x)
        out = p.dedisperse_device(d, nsamp)
        snr = torch.full_like(out, float("nan"))
        cands, count, _ = p.sps_search_device(out, nsamp, 256, w.threshold, 1 << 16, snr_out=snr)
        torch.cuda.synchronize()
        got.append((candidates_from_device(cands, count, 1 << 16), p.range_views(snr, nsamp)[0].cpu()))
    assert np.array_equal(got[0][0], got[1][0]) and torch.equal(got[0][1], got[1][1])
