"""Candidate post-processing on the device through the C ABI:
aa_sps_order_device (runs of the boxcar CTAs gathered into (dm_index, t)
order) against the host ordering and a numpy sort of the same records, and
aa_candidates_peaks2d_device (2-D DM-time peaks) against the oracle on seeded
synthetic candidate lists: ties, several ranges, radii from 0 to unbounded,
lists spanning several scan blocks, empty and truncated lists."""
import numpy as np
import pytest
import torch

from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device

pytestmark = pytest.mark.gpu


def _search(plan, x, W, thr, cap):
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    ws = plan.alloc_workspace(plan.query(nsamp, W).sps_ws_bytes)
    cands, count, _ = plan.sps_search_device(out, nsamp, W, thr, cap, ws=ws)
    return out, nsamp, ws, cands, count


def _ordered(plan, nsamp, W, ws, cands, count, cap):
    srt = plan.sps_order_device(nsamp, W, ws, cands, count, cap)
    torch.cuda.synchronize()
    n = min(int(count.item()), cap)
    return srt[: n * 16].cpu().numpy().view(synth.CANDIDATE_RECORD)


def _noise(C, T, seed):
    return np.random.default_rng(seed).integers(96, 160, size=(C, T), dtype=np.uint8)


def test_order_single_range_many_tiles():
    w = synth.PLAIN_256
    plan = Plan(w.nchans, w.fch1, w.foff, w.tsamp, list(w.ranges))
    x = _noise(w.nchans, w.nsamp, 21)
    cap = 1 << 20
    out, nsamp, ws, cands, count = _search(plan, x, 32, 3.0, cap)
    got = _ordered(plan, nsamp, 32, ws, cands, count, cap)
    total = int(count.item())
    assert 10000 < total <= cap
    ref = candidates_from_device(cands, count, cap)  # numpy sort of the same records
    assert np.array_equal(got, ref)
    host, htotal = plan.sps_search(plan.dedisperse(x), 32, 3.0, capacity=cap)
    assert htotal == total and np.array_equal(got, host)


def test_order_decimated_ranges_and_overflow():
    C, fch1, foff, ts, T = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    plan = Plan(C, fch1, foff, ts, ranges)
    x = _noise(C, T, 22)
    cap = 1 << 16
    out, nsamp, ws, cands, count = _search(plan, x, 64, 2.5, cap)
    got = _ordered(plan, nsamp, 64, ws, cands, count, cap)
    total = int(count.item())
    assert set(got["range"].tolist()) == {0, 1, 2, 3}
    assert np.array_equal(got, candidates_from_device(cands, count, cap))
    # capacity below the total: the stored records, ordered
    small = total // 3
    _, _, ws2, c2, n2 = _search(plan, x, 64, 2.5, small)
    got2 = _ordered(plan, nsamp, 64, ws2, c2, n2, small)
    assert int(n2.item()) == total and got2.size == small
    assert np.array_equal(got2, candidates_from_device(c2, n2, small))


def _peaks_gpu(plan, nsamp, W, f, cap, R, Tr, count=None):
    dev = torch.zeros(max(cap, 1) * 16, dtype=torch.uint8, device="cuda")
    if f.size:
        dev[: f.size * 16] = torch.from_numpy(f.view(np.uint8).copy()).cuda()
    n = torch.tensor([f.size if count is None else count], dtype=torch.int64, device="cuda")
    peaks, npeaks = plan.peaks2d_device(nsamp, W, dev, n, cap, R, Tr)
    torch.cuda.synchronize()
    k = int(npeaks.item())
    return peaks[: k * 16].cpu().numpy().view(synth.CANDIDATE_RECORD)


def _plan_field(seed, n_pulses, n_noise, q):
    C, fch1, foff, ts, T = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    plan = Plan(C, fch1, foff, ts, ranges)
    lay = plan.layout(T)
    f = synth.candidate_field([g.ndm for g in lay], [g.length for g in lay], n_pulses, n_noise,
                              seed, snr_quantum=q)
    return plan, T, f


@pytest.mark.parametrize("R,Tr,q", [(0, 0, 0.25), (1, 1, 0.25), (3, 12, 0.5), (8, 64, 0.0),
                                    (40, 500, 0.25), (10 ** 6, 10 ** 8, 0.5)])
def test_peaks2d_parity(oracle, R, Tr, q):
    plan, T, f = _plan_field(31, 60, 14000, q)
    assert f.size > 3 * 4096  # several scan blocks
    got = _peaks_gpu(plan, T, 64, f, f.size + 100, R, Tr)
    want = f[oracle.peaks2d(f, R, Tr)]
    assert np.array_equal(got, want)


def test_peaks2d_empty_and_truncated(oracle):
    plan, T, f = _plan_field(32, 10, 500, 0.25)
    assert _peaks_gpu(plan, T, 64, f[:0], 0, 2, 8).size == 0
    assert _peaks_gpu(plan, T, 64, f[:0], 64, 2, 8).size == 0
    # a count above the capacity: the first `capacity` records form the list
    cap = f.size // 2
    got = _peaks_gpu(plan, T, 64, f[:cap], cap, 2, 8, count=f.size + 7)
    assert np.array_equal(got, f[:cap][oracle.peaks2d(f[:cap], 2, 8)])


def test_order_then_peaks_on_search_output(oracle):
    """The two calls chained on a real search: the peaks of the ordered list
    equal the oracle's filter of the numpy-sorted records."""
    C, fch1, foff, ts, T = 203, 1400.0, -0.5, 64e-6, 9001
    ranges = [(0.0, 1.0, 35, 1), (35.0, 1.5, 18, 2), (62.0, 2.0, 21, 4), (104.0, 3.0, 5, 3)]
    plan = Plan(C, fch1, foff, ts, ranges)
    x = _noise(C, T, 23)
    cap = 1 << 16
    out, nsamp, ws, cands, count = _search(plan, x, 64, 3.0, cap)
    srt = plan.sps_order_device(nsamp, 64, ws, cands, count, cap)
    peaks, npeaks = plan.peaks2d_device(nsamp, 64, srt, count, cap, 3, 16)
    torch.cuda.synchronize()
    ref = candidates_from_device(cands, count, cap)
    k = int(npeaks.item())
    got = peaks[: k * 16].cpu().numpy().view(synth.CANDIDATE_RECORD)
    assert np.array_equal(got, ref[oracle.peaks2d(ref, 3, 16)])


def test_peaks2d_times_past_series_end(oracle):
    """Records with t beyond a range's series length (not produced by the
    search, but a valid list): the time index's last bucket is open-ended."""
    plan, T, f = _plan_field(33, 30, 5000, 0.25)
    f["t"] = f["t"] * 3 + 5
    f = f[np.lexsort((f["t"], f["dm_index"]))]
    for R, Tr in [(2, 40), (5, 700)]:
        got = _peaks_gpu(plan, T, 64, f, f.size, R, Tr)
        assert np.array_equal(got, f[oracle.peaks2d(f, R, Tr)])
