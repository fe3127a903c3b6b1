"""Oracle on the 256-channel single-beam workload: the injected pulse is
recovered at its DM, arrival time and width with the closed-form SNR, and
pure noise gives (almost) no candidates above 6 sigma."""
import numpy as np
import pytest

from paper_1912_07704_gb300 import synth


def _delays(o, w):
    return lambda dm: o.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)


@pytest.fixture(scope="module")
def plain_run(oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(w, synth.pulses_single(), _delays(oracle, w)).numpy()
    pl, ys = oracle.dedisperse(x, w.nchans, w.fch1, w.foff, w.tsamp, w.ranges)
    cands = []
    for i in range(pl[0].ndm):
        c, *_ = oracle.search_row(ys[0][i], w.max_width, w.threshold, i, 0)
        cands += c
    return w, pl, ys, cands


def test_pulse_recovered(plain_run):
    w, pl, ys, cands = plain_run
    best = max(cands, key=lambda c: c.snr)
    assert (pl[0].dms[best.dm_index], best.t, best.width) == (150.0, 8192, 16)
    # closed form with the pulse's own share of the series variance:
    # box height h = A*C = 10240 on n_w = 16 of L = 28658 samples, p = n_w/L,
    # noise variance C*16^2 = 65536; sigma^2 = 65536 + h^2 p (1-p);
    # SNR = n_w h (1-p) / (sqrt(n_w) sigma) = 116.2 (160 if the pulse did
    # not inflate sigma).  Noise moves it by about +-0.7 (1 sigma).
    C, A, n_w, L = 256, 40.0, 16, 32768 - 4110
    h, p = A * C, n_w / L
    sig = np.sqrt(C * 16.0**2 + h * h * p * (1 - p))
    expect = n_w * h * (1 - p) / (np.sqrt(n_w) * sig)
    assert abs(expect - 116.2) < 0.1
    assert abs(best.snr - expect) < 3.0


def test_pulse_candidate_only_near_pulse(plain_run):
    w, pl, ys, cands = plain_run
    solid = [c for c in cands if not c.fragile]
    # every candidate lies on the dispersed pulse track (arrival near 8192
    # once the DM error is accounted for), i.e. no noise detections
    assert all(abs(c.t - 8192) < 2500 for c in solid)
    dms = {pl[0].dms[c.dm_index] for c in solid}
    assert 150.0 in dms


def test_noise_only_false_positive_rate(oracle):
    w = synth.PLAIN_256
    x = synth.noise_filterbank(w.nchans, w.nsamp, seed=99).numpy()
    rows = [list(range(0, 256, 8))]
    pl, ys = oracle.dedisperse(x, w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, rows=rows)
    n = 0
    for k, i in enumerate(rows[0]):
        c, B, *_ = oracle.search_row(ys[0][k], w.max_width, w.threshold, i, 0)
        n += sum(1 for cc in c if not cc.fragile)
        assert np.isfinite(B).all()
    assert n <= 1
