"""Full-size 4096-channel, 2^20-sample, four-range plan with W = 8192, run
exactly as bench.py runs it.  The oracle checks dedispersion bit-exactly on
a strided subset of trials (every 25th trial of each range, both ends of each
range and the trials at the injected pulses' DMs: about 180 full rows), the
boxcar SNR B(t) and the candidate list over one full-length row per range
(the row at the range's strongest pulse, else its middle row) and over
2048-sample windows (around each pulse where one falls in the row) of every
other sampled row; every strong injected pulse must be detected near its DM
and arrival time.
The bench's post-processing runs on the same output: the device ordering must
equal a numpy sort of the records, and the 2-D peak filter must agree with the
oracle on sampled candidates."""
import numpy as np
import pytest
import torch

from gpu_common import check_snr_rows, compare_candidate_lists, oracle_candidates
from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device
from paper_1912_07704_gb300.synth import CANDIDATE_RECORD

pytestmark = pytest.mark.gpu

W = synth.SKA_4096


PEAK_DM_RADIUS, PEAK_T_RADIUS = 8, 256  # bench.py's 2-D peak window
post = {}


@pytest.fixture(scope="module")
def ska_run(oracle):
    oracle.set_threads(0)
    d1 = lambda dm: oracle.shifts(W.nchans, W.fch1, W.foff, W.tsamp, dm, 1)
    pulses = synth.pulses_ska(W, lambda dm: int(d1(dm).max()))
    plan = Plan.from_workload(W)
    pitch = plan.query(W.nsamp).in_pitch_min
    x = synth.make_filterbank(W, pulses, d1, device="cuda", pitch=pitch)
    nsamp = W.nsamp
    # the bench configuration: no B output
    out = plan.dedisperse_device(x, nsamp)
    cap = 1 << 25
    ws = plan.alloc_workspace(plan.query(nsamp, W.max_width).sps_ws_bytes)
    cands, count, _ = plan.sps_search_device(out, nsamp, W.max_width, W.threshold, cap, ws=ws)
    torch.cuda.synchronize()
    assert int(count.item()) <= cap, int(count.item())
    bench_cands = candidates_from_device(cands, count, cap)
    # device ordering and 2-D peaks, as bench.py runs them
    n = int(count.item())
    srt = plan.sps_order_device(nsamp, W.max_width, ws, cands, count, cap)
    peaks, npeaks = plan.peaks2d_device(nsamp, W.max_width, srt, count, cap, PEAK_DM_RADIUS,
                                        PEAK_T_RADIUS)
    torch.cuda.synchronize()
    dev_sorted = srt[: n * 16].cpu().numpy().view(CANDIDATE_RECORD)
    dev_peaks = peaks[: int(npeaks.item()) * 16].cpu().numpy().view(CANDIDATE_RECORD)
    del srt, peaks, ws
    # the same call with the optional B(t) output
    snr = torch.full_like(out, float("nan"))
    cands2, count2, _ = plan.sps_search_device(out, nsamp, W.max_width, W.threshold, cap,
                                               snr_out=snr)
    torch.cuda.synchronize()
    assert int(count2.item()) == int(count.item())
    snr_cands = candidates_from_device(cands2, count2, cap)
    xh = x[:, :nsamp].cpu().numpy()
    del x, cands, cands2
    torch.cuda.empty_cache()
    post["sorted"], post["peaks"] = dev_sorted, dev_peaks
    yield plan, xh, out, snr, bench_cands, snr_cands, pulses
    del out, snr
    torch.cuda.empty_cache()


def test_bench_and_snr_runs_agree(ska_run):
    plan, xh, out, snr, bc, sc, pulses = ska_run
    assert np.array_equal(bc, sc)


STRIDE = 25


def _pulse_row(g, p):
    i = int(round((p.dm - g.dm_lo) / g.dm_step)) if g.dm_step > 0 else 0
    return i if 0 <= i < g.ndm else None


def _sample_rows(lay, pulses, r):
    g = lay[r]
    rows = set(range(0, g.ndm, STRIDE)) | {g.ndm - 1}
    for p in pulses:
        i = _pulse_row(g, p)
        if i is not None:
            rows.add(i)
    return sorted(rows)


def _full_row(lay, pulses, r):
    """The row searched over its whole length: the strongest pulse's trial
    in this range, else the middle trial."""
    g = lay[r]
    best = None
    for p in pulses:
        i = _pulse_row(g, p)
        if i is not None and (best is None or p.amplitude * np.sqrt(p.n_w) > best[0]):
            best = (p.amplitude * np.sqrt(p.n_w), i)
    return best[1] if best else g.ndm // 2


def test_sampled_rows_parity(oracle, ska_run):
    plan, xh, out, snr, bc, sc, pulses = ska_run
    lay = plan.layout(W.nsamp)
    dd = plan.range_views(out, W.nsamp)
    sv = plan.range_views(snr, W.nsamp)
    opl = oracle.plan(W.nchans, W.fch1, W.foff, W.tsamp, W.ranges, W.nsamp)
    compared = checked_rows = 0
    for r, g in enumerate(lay):
        xr = oracle.range_input(xh, g.dec)
        rows = _sample_rows(lay, pulses, r)
        ys = {}
        for i in rows:
            y = oracle.dedisperse_row(xr, opl[r].shifts[i], 0, g.length)
            assert np.array_equal(dd[r][i].double().cpu().numpy(), y.astype(np.float64)), (r, i)
            ys[i] = y
        windows = {}
        full = _full_row(lay, pulses, r)
        for i in rows:
            lo, hi = 0, 2048
            for p in pulses:
                t = p.t0 // g.dec
                if abs(p.dm - (g.dm_lo + i * g.dm_step)) < 3 * max(g.dm_step, 1e-9) and t < g.length:
                    lo, hi = max(0, t - 1024), min(g.length, t + 1024)
            windows[i] = (lo, hi)
        windows[full] = (0, g.length)  # the whole series
        solid, fragile, B = oracle_candidates(oracle, ys, W.max_width, W.threshold,
                                              g.dm_offset, r, windows)
        check_snr_rows(sv[r], ys, B)
        glob = {g.dm_offset + i: windows[i] for i in rows}
        keep = lambda dm, t: dm in glob and glob[dm][0] <= t < glob[dm][1]
        compared += compare_candidate_lists(bc[bc["range"] == r], solid, fragile, keep)
        checked_rows += len(rows)
    assert compared > 0
    assert checked_rows >= 170


def test_strong_pulses_detected(ska_run):
    plan, xh, out, snr, bc, sc, pulses = ska_run
    lay = plan.layout(W.nsamp)
    checked = 0
    for p in pulses:
        if 4.0 * p.amplitude * np.sqrt(p.n_w) < 12.0:
            continue  # expected SNR too low to require a detection
        for r, g in enumerate(lay):
            hi = g.dm_lo + (g.ndm - 1) * g.dm_step
            if not (g.dm_lo <= p.dm <= hi + g.dm_step):
                continue
            t = p.t0 // g.dec
            sel = bc[(bc["range"] == r)
                     & (np.abs(g.dm_lo + (bc["dm_index"] - g.dm_offset) * g.dm_step - p.dm)
                        <= 2 * g.dm_step)
                     & (np.abs(bc["t"].astype(np.int64) - t) <= p.n_w // g.dec + 4)]
            assert len(sel) > 0, (p, r)
            checked += 1
    assert checked >= 5


def test_device_order_full_size(ska_run):
    bc = ska_run[4]
    assert bc.size > 1 << 20
    assert np.array_equal(post["sorted"], bc)


def test_peaks2d_full_size_sampled(oracle, ska_run):
    bc = ska_run[4]
    pk = post["peaks"]
    assert 0 < pk.size < bc.size
    key = lambda a: a["dm_index"].astype(np.int64) * (1 << 32) + a["t"].astype(np.int64)
    kb, kp = key(bc), key(pk)
    assert np.all(np.diff(kp) > 0)  # ordered, and a subset of the list below
    pos = np.searchsorted(kb, kp)
    assert np.array_equal(bc[pos], pk)
    rng = np.random.Generator(np.random.PCG64(77))
    idx = np.unique(np.concatenate([rng.integers(0, bc.size, 3000), pos[:200], pos[-200:],
                                    [int(np.argmax(bc["snr"]))]]))
    want = oracle.peaks2d(bc, PEAK_DM_RADIUS, PEAK_T_RADIUS, idx)
    got = np.isin(kb[idx], kp)
    assert np.array_equal(got, want)
    assert got[idx == int(np.argmax(bc["snr"]))].all()  # the strongest candidate survives
