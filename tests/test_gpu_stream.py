"""Streaming server with continuous batching: chunk results are identical
alone and in the mix, match the oracle run on the same block, and the
dedispersed samples of each chunk's emitted region equal those of the whole
series."""
import numpy as np
import pytest
import torch

from gpu_common import compare_candidate_lists
from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Plan, Server

pytestmark = pytest.mark.gpu

C, FCH1, FOFF, TS = 64, 1400.0, -4.0, 64e-6
RANGES = [(0.0, 4.0, 20, 1), (80.0, 8.0, 10, 2)]
N, W, THR, NCHUNK, NBEAM = 4096, 32, 5.0, 5, 3


def series(oracle, b):
    w = synth.Workload(f"s{b}", C, FCH1, FOFF, TS, N * NCHUNK, tuple(RANGES), W, THR, 40 + b)
    pulses = [synth.Pulse(20.0 + 30 * b, 3000 + 5000 * b, 8, 25.0),
              synth.Pulse(100.0, 12000 + 1000 * b, 4, 30.0)]
    return synth.make_filterbank(w, pulses, lambda dm: oracle.shifts(C, FCH1, FOFF, TS, dm, 1)).numpy()


def run_server(plan, data, beams, order, max_slots):
    srv = Server(plan, NBEAM, N, W, THR, capacity=1 << 16, max_slots=max_slots)
    chunks = {}
    tickets = {}
    for (b, k) in order:
        if b not in beams:
            continue
        buf = np.ascontiguousarray(data[b][:, k * N:(k + 1) * N])
        chunks[(b, k)] = buf  # keep alive until completion
        tickets[(b, k)] = srv.submit(b, buf)
        srv.poll()
    srv.drain()
    out = {}
    for key, t in tickets.items():
        st, info, arr = srv.result(t)
        assert st == 0 and info.chunk == key[1] and info.beam == key[0]
        out[key] = (info, arr)
    stats = srv.stats()
    srv.close()
    return out, stats


@pytest.fixture(scope="module")
def streams(oracle):
    plan = Plan(C, FCH1, FOFF, TS, RANGES)
    data = [series(oracle, b) for b in range(NBEAM)]
    order = [(b, k) for k in range(NCHUNK) for b in range(NBEAM)]
    mix, stats = run_server(plan, data, set(range(NBEAM)), order, max_slots=4)
    return plan, data, mix, stats


def test_mix_equals_alone(streams):
    plan, data, mix, stats = streams
    assert stats.completed == NBEAM * NCHUNK and stats.max_in_flight >= 2
    for b in range(NBEAM):
        alone, _ = run_server(plan, data, {b}, [(b, k) for k in range(NCHUNK)], max_slots=1)
        for k in range(NCHUNK):
            assert np.array_equal(alone[(b, k)][1], mix[(b, k)][1]), (b, k)


def test_chunks_match_oracle_on_blocks(oracle, streams):
    plan, data, mix, stats = streams
    H = stats.history_nsamp
    opl = oracle.plan(C, FCH1, FOFF, TS, RANGES, N * NCHUNK)
    compared = 0
    for b in range(NBEAM):
        whole = oracle.dedisperse(data[b], C, FCH1, FOFF, TS, RANGES)[1]
        for k in range(NCHUNK):
            info, arr = mix[(b, k)]
            b0 = max(0, k * N - H)
            assert info.block_start == b0
            block = np.ascontiguousarray(data[b][:, b0:(k + 1) * N])
            bpl, bys = oracle.dedisperse(block, C, FCH1, FOFF, TS, RANGES)
            for r, (g, rng) in enumerate(zip(opl, RANGES)):
                dec = rng[3]
                lag = g.maxshift + W + 1
                lo, hi = max(0, k * N // dec - lag), (k + 1) * N // dec - lag
                if hi <= lo:
                    continue
                # block dedispersion == whole-series dedispersion on the region
                a, bb = lo - b0 // dec, hi - b0 // dec
                assert np.array_equal(bys[r][:, a:bb], whole[r][:, lo:hi])
                solid, fragile = {}, set()
                for i in range(g.ndm):
                    cands, *_ = oracle.search_row(bys[r][i], W, THR, g.dm_offset + i, r, a, bb)
                    for c in cands:
                        key = (c.dm_index, c.t + b0 // dec)
                        c.t += b0 // dec
                        (fragile.add(key) if c.fragile else solid.__setitem__(key, c))
                sel = arr[arr["range"] == r].copy()
                sel["reserved"] = 0
                compared += compare_candidate_lists(sel, solid, fragile)
    assert compared > 0
