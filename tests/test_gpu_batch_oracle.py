"""The batched path (one CUDA graph over many beams, in its default form of
each beam's kernels on concurrent branches, and in the persistent work-queue
form) against the ORACLE, not against the single-beam GPU path.

Beams: the four small uneven beams of test_gpu_batch (64-128 channels,
decimations 1/2/4/8/16 with the dec-16 range among them), plus two beams of
the batched workload's shape: 1024 channels over the 300 MHz band, 2^17
samples, the 4096-channel plan's ranges clipped at DM 2100 with the
(2000, 2, ., dec 16) range above DM 2000, every range forced onto the grouped
strategy (so the 16-bit lanes' largest channel chunks run); and 4096 channels,
2^17 samples, ranges clipped at DM 700, every range on the direct strategy.

Dedispersion is compared bit-exactly (every row of the small beams, every
25th trial plus both ends of each range of the large ones); candidate lists
and SNRs on those rows are compared with the oracle's search of the same
series, away from fragile decisions.
"""
import numpy as np
import pytest
import torch

from gpu_common import compare_candidate_lists, oracle_candidates
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Batch, Plan

pytestmark = pytest.mark.gpu

SMALL = [
    (64, 1400.0, -4.0, 21001, [(0.0, 4.0, 23, 1), (92.0, 6.0, 17, 2)]),
    (128, 1500.0, -2.0, 30011, [(0.0, 3.0, 40, 1), (120.0, 5.0, 9, 4), (165.0, 9.0, 7, 16)]),
    (64, 1300.0, -3.0, 9000, [(10.0, 2.0, 5, 2)]),
    (96, 1450.0, -2.5, 17777, [(0.0, 1.0, 33, 1), (33.0, 2.0, 12, 8)]),
]
W, THR = 512, 6.0
STRIDE = 25


def _shape3(C, dm_max, index):
    """A beam of the batched workload's shape (300 MHz band, 2^17 samples)."""
    return synth.Workload(f"b3-{C}ch", C, 1508.0, -300.0 / C, 64e-6, 1 << 17,
                          synth.clipped_ska_ranges(dm_max), W, THR, index)


def _rows(ndm, every):
    if every <= 1:
        return list(range(ndm))
    return sorted(set(range(0, ndm, every)) | {ndm - 1})


@pytest.fixture(scope="module")
def batch_run(oracle):
    oracle.set_threads(0)
    beams = []  # (workload, plan, host data, row stride)
    for k, (C, fch1, foff, T, ranges) in enumerate(SMALL):
        w = synth.Workload(f"s{k}", C, fch1, foff, 64e-6, T, tuple(ranges), W, THR, 40 + k)
        pulses = [synth.Pulse(ranges[0][0] + ranges[0][1] * 2, T // 3, 6, 30.0),
                  synth.Pulse(ranges[-1][0] + ranges[-1][1] * 2, (2 * T) // 3, 24, 12.0)]
        d1 = lambda dm, C=C, fch1=fch1, foff=foff: oracle.shifts(C, fch1, foff, 64e-6, dm, 1)
        x = synth.make_filterbank(w, pulses, d1).numpy()
        beams.append((w, Plan(C, fch1, foff, 64e-6, ranges), x, 1))
    for (C, dm_max, strategy, idx) in [(1024, 2100.0, abi.AA_DEDISP_GROUPED, 50),
                                       (4096, 700.0, abi.AA_DEDISP_DIRECT, 51)]:
        w = _shape3(C, dm_max, idx)
        d1 = lambda dm, w=w: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)
        pulses = synth.pulses_ska(w, lambda dm: int(d1(dm).max()), n=4)
        x = synth.make_filterbank(w, pulses, d1).numpy()
        p = Plan.from_workload(w)
        for r in range(len(w.ranges)):
            info = abi.aa_plan_range(p.handle, w.nsamp, r)
            if strategy == abi.AA_DEDISP_GROUPED:
                assert info.grouped_available == 1, (C, r)
            p.set_strategy(r, strategy)
        beams.append((w, p, x, STRIDE))
    b = Batch([bm[1] for bm in beams], [bm[2].shape[1] for bm in beams], W, THR,
              capacity=1 << 22)
    assert b.info()[0] == 1  # one wave: every beam's series stay readable
    for i, (_, _, x, _) in enumerate(beams):
        b.input_view(i)[:, : x.shape[1]].copy_(torch.from_numpy(x))
    b.run()
    torch.cuda.synchronize()
    arr, total = b.candidates()
    assert total == len(arr)
    yield b, beams, arr
    b.close()
    for bm in beams:
        bm[1].close()


def test_dec16_and_grouped_ranges_present(batch_run):
    b, beams, arr = batch_run
    decs = {g.dec for (w, p, x, _) in beams for g in p.layout(x.shape[1])}
    assert 16 in decs and {1, 2, 4, 8} <= decs
    w, p, x, _ = beams[len(SMALL)]
    assert p.layout(x.shape[1])[-1].dec == 16
    for r in range(len(w.ranges)):
        assert abi.aa_plan_range(p.handle, x.shape[1], r).strategy == abi.AA_DEDISP_GROUPED


@pytest.mark.parametrize("beam", range(len(SMALL) + 2))
def test_batched_beam_equals_oracle(oracle, batch_run, beam):
    b, beams, arr = batch_run
    w, p, x, every = beams[beam]
    nsamp = x.shape[1]
    views = p.range_views(b.dd_view(beam), nsamp)
    opl = oracle.plan(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, nsamp)
    mine = arr[arr["reserved"] == beam]
    compared = 0
    for r, (g, v) in enumerate(zip(p.layout(nsamp), views)):
        assert g.length == opl[r].length
        if g.length <= 0:
            continue
        xr = oracle.range_input(x, g.dec)
        rows = _rows(g.ndm, every)
        got = v[rows].double().cpu().numpy()
        ys = {}
        for k, i in enumerate(rows):
            y = oracle.dedisperse_row(xr, opl[r].shifts[i], 0, g.length)
            assert np.array_equal(got[k], y.astype(np.float64)), (beam, r, i)
            ys[i] = y
        solid, fragile, _ = oracle_candidates(oracle, ys, W, THR, g.dm_offset, r)
        sel = set(g.dm_offset + i for i in rows)
        compared += compare_candidate_lists(mine[mine["range"] == r], solid, fragile,
                                            lambda dm, t: dm in sel)
    assert compared > 0, f"beam {beam}: no candidates compared"


def test_dd_view_refuses_overwritten_waves(oracle):
    """With one wave per beam only the last wave's series survive a run."""
    plans, xs = [], []
    for k, (C, fch1, foff, T, ranges) in enumerate(SMALL[:2]):
        plans.append(Plan(C, fch1, foff, 64e-6, ranges))
        xs.append(synth.noise_filterbank(C, T, seed=70 + k).numpy())
    b = Batch(plans, [x.shape[1] for x in xs], 64, THR, capacity=1 << 16, wave_budget=1)
    assert b.info()[0] == 2
    for i, x in enumerate(xs):
        b.input_view(i)[:, : x.shape[1]].copy_(torch.from_numpy(x))
    b.run()
    torch.cuda.synchronize()
    with pytest.raises(abi.AAError):
        b.dd_view(0)
    v = plans[1].range_views(b.dd_view(1), xs[1].shape[1])
    _, ys = oracle.dedisperse(xs[1], plans[1].nchans, plans[1].fch1, plans[1].foff, 64e-6,
                              plans[1].ranges)
    for g, o in zip(v, ys):
        assert np.array_equal(g.double().cpu().numpy(), o.astype(np.float64))
    b.close()


def test_persistent_form_equals_checked_form(batch_run):
    """The persistent work-queue form gives the candidates and the series of
    the default form checked against the oracle above (on every row)."""
    b, beams, arr = batch_run
    before = [[v.clone() for v in p.range_views(b.dd_view(i), x.shape[1])]
              for i, (_, p, x, _) in enumerate(beams)]
    b.set_branches(0)
    try:
        b.run()
        torch.cuda.synchronize()
        arr_p, total_p = b.candidates()
        assert total_p == len(arr) and np.array_equal(arr_p, arr)
        for i, (_, p, x, _) in enumerate(beams):
            after = p.range_views(b.dd_view(i), x.shape[1])
            assert all(torch.equal(u, v) for u, v in zip(before[i], after)), f"beam {i}"
    finally:
        b.set_branches(8)
