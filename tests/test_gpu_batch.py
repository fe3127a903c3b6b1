"""Batched beams (one CUDA graph: each beam's kernels on concurrent branches,
or persistent work-queue kernels per stage) against the same beams run one
at a time, and the autotuner."""
import os

import numpy as np
import pytest
import torch

from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Batch, Plan, candidates_from_device

pytestmark = pytest.mark.gpu

BEAMS = [
    (64, 1400.0, -4.0, 21001, [(0.0, 4.0, 23, 1), (92.0, 6.0, 17, 2)]),
    (128, 1500.0, -2.0, 30011, [(0.0, 3.0, 40, 1), (120.0, 5.0, 9, 4), (165.0, 9.0, 7, 16)]),
    (64, 1300.0, -3.0, 9000, [(10.0, 2.0, 5, 2)]),
    (96, 1450.0, -2.5, 17777, [(0.0, 1.0, 33, 1), (33.0, 2.0, 12, 8)]),
]
W, THR = 64, 5.0


def make_beams(oracle):
    plans, data = [], []
    for k, (C, fch1, foff, T, ranges) in enumerate(BEAMS):
        w = synth.Workload(f"b{k}", C, fch1, foff, 64e-6, T, tuple(ranges), W, THR, 20 + k)
        pulses = [synth.Pulse(ranges[0][0] + ranges[0][1] * 2, T // 3, 6, 30.0)]
        x = synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, fch1, foff, 64e-6, dm, 1))
        plans.append(Plan(C, fch1, foff, 64e-6, ranges))
        data.append(x.numpy())
    return plans, data


def single(plan, x):
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    cands, count, _ = plan.sps_search_device(out, nsamp, W, THR, 1 << 16)
    torch.cuda.synchronize()
    return candidates_from_device(cands, count, 1 << 16)


def batched(plans, data, budget=0):
    b = Batch(plans, [x.shape[1] for x in data], W, THR, capacity=1 << 18, wave_budget=budget)
    for i, x in enumerate(data):
        b.input_view(i)[:, : x.shape[1]].copy_(torch.from_numpy(x))
    b.run()
    arr, total = b.candidates()
    return b, arr, total


def split(arr, n):
    out = []
    for i in range(n):
        a = arr[arr["reserved"] == i].copy()
        a["reserved"] = 0
        out.append(a)
    return out


@pytest.mark.parametrize("budget", [0, 1], ids=["one-wave", "wave-per-beam"])
def test_batch_equals_beams_alone(oracle, budget):
    plans, data = make_beams(oracle)
    b, arr, total = batched(plans, data, budget)
    assert b.info()[0] == (1 if budget == 0 else len(BEAMS))
    per = split(arr, len(BEAMS))
    assert sum(len(a) for a in per) == total == len(arr)
    n_nonempty = 0
    for i, (p, x) in enumerate(zip(plans, data)):
        ref = single(p, x)
        assert np.array_equal(per[i], ref), f"beam {i}"
        n_nonempty += len(ref) > 0
    assert n_nonempty >= 3
    # a second replay of the graph gives the same list
    b.run()
    arr2, total2 = b.candidates()
    assert total2 == total and np.array_equal(arr2, arr)
    b.close()


@pytest.mark.parametrize("budget", [0, 1], ids=["one-wave", "wave-per-beam"])
@pytest.mark.parametrize("branches", [1, 3])
def test_branched_graph_equals_persistent(oracle, budget, branches):
    """Every graph form (8 branches at creation, 1 or 3 branches, the
    persistent work-queue kernels) finds the same candidates and the same
    dedispersed series; switching re-records the graph without touching the
    buffers."""
    plans, data = make_beams(oracle)
    b, arr, total = batched(plans, data, budget)
    b.set_branches(branches)
    b.run()
    arr_b, total_b = b.candidates()
    assert total_b == total and np.array_equal(arr_b, arr)
    for i, (p, x) in enumerate(zip(plans, data)):
        if b.info()[0] == 1 or i == len(BEAMS) - 1:  # series kept by the last wave only
            d, nsamp = p.device_input(x)
            ref = p.range_views(p.dedisperse_device(d, nsamp), nsamp)
            got = p.range_views(b.dd_view(i), nsamp)
            assert all(torch.equal(u, v) for u, v in zip(got, ref)), f"beam {i}"
    b.set_branches(0)
    b.run()
    arr_p, total_p = b.candidates()
    assert total_p == total and np.array_equal(arr_p, arr)
    with pytest.raises(Exception):
        b.set_branches(65)
    b.close()


def test_autotune_keeps_results_and_caches(tmp_path, oracle):
    C, fch1, foff, T, ranges = BEAMS[1]
    x = synth.noise_filterbank(C, T, seed=3).numpy()
    p0 = Plan(C, fch1, foff, 64e-6, ranges)
    d, nsamp = p0.device_input(x)
    ref = p0.dedisperse_device(d, nsamp).clone()
    cache = tmp_path / "tune.txt"
    p1 = Plan(C, fch1, foff, 64e-6, ranges)
    p1.autotune(nsamp, str(cache))
    assert cache.exists() and len(cache.read_text().strip().splitlines()) == len(ranges)
    out1 = p1.dedisperse_device(d, nsamp)
    p2 = Plan(C, fch1, foff, 64e-6, ranges)
    p2.autotune(nsamp, str(cache))  # served from the cache
    assert len(cache.read_text().strip().splitlines()) == len(ranges)
    out2 = p2.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    for a, b_, c in zip(p0.range_views(ref, nsamp), p1.range_views(out1, nsamp),
                        p2.range_views(out2, nsamp)):
        assert torch.equal(a, b_) and torch.equal(a, c)
