"""Seeded synthetic filterbanks standing in for simulated SKA-like data.

The paper evaluates on "simulated SKA-like data" (abstract, Sec. 1) that is not
published; these generators produce data of that shape instead:

* noise: round(N(128, 16^2)) clipped to [0, 255], uint8, channels x time;
* dispersed box pulses: amplitude A added to the noise (before rounding and
  clipping) on samples [t0 + d_c, t0 + d_c + n_w) of every channel c.

The per-channel pulse delays d_c are INPUTS: this module computes no
dispersion delay and holds none of the search arithmetic.  Callers obtain the
delays from their own side (the library's plan in bench.py, the oracle in
tests).  Everything is seeded: torch.Generator for the noise (on the device
the data is made on), numpy PCG64 for the pulse parameters.

Workload presets mirror the configurations the library is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np
import torch

DATA_SEED = 1912
PULSE_SEED = 7704


@dataclass(frozen=True)
class Workload:
    name: str
    nchans: int
    fch1: float
    foff: float
    tsamp: float
    nsamp: int
    ranges: tuple  # ((dm_lo, dm_step, ndm, dec), ...)
    max_width: int
    threshold: float
    index: int  # 0-based position among the presets (seeds are offset by it)

    @property
    def data_seed(self) -> int:
        return DATA_SEED + self.index

    @property
    def pulse_seed(self) -> int:
        return PULSE_SEED + self.index


# 256 channels, 32768 samples, DM 0..255 step 1, widths 1..32, threshold 6.
PLAIN_256 = Workload("plain-256ch-32768", 256, 1500.0, -1.171875, 64e-6, 32768,
                     ((0.0, 1.0, 256, 1),), 32, 6.0, 0)
# 4096 channels, 2^20 samples, four DM ranges with decimation 1/2/4/8,
# widths 1..8192, threshold 6.
SKA_4096 = Workload("ska-4096ch-2^20", 4096, 1508.0, -0.0732421875, 64e-6, 1 << 20,
                    ((0.0, 0.1, 1500, 1), (150.0, 0.2, 750, 2), (300.0, 0.5, 600, 4),
                     (600.0, 1.0, 1400, 8)), 8192, 6.0, 1)


@dataclass
class Pulse:
    dm: float
    t0: int        # arrival sample at the top of the band
    n_w: int       # width in full-rate samples
    amplitude: float


def pulses_single(dm=150.0, t0=8192, n_w=16, amplitude=40.0) -> list:
    """The single 1 ms, +40 count pulse of the 256-channel workload."""
    return [Pulse(dm, t0, n_w, amplitude)]


def pulses_ska(w: Workload, max_delay: Callable[[float], int], n: int = 20,
               snr_range=(8.0, 150.0)) -> list:
    """n pulses: DM ~ U[50, 2000], width log-uniform 64 us .. 16 ms, and an
    amplitude set from a target matched-filter SNR ~ U[snr_range]:
    A = SNR * 16 / (sqrt(nchans) * sqrt(n_w)) counts (noise std 16 per
    channel-sample, box of n_w samples summed over all channels).  Start times
    are evenly spaced with jitter so that no two pulses overlap and every
    pulse ends before the series does.

    max_delay(dm) must return the largest per-channel delay (full-rate
    samples) of a pulse at that DM; it is supplied by the caller.
    """
    rng = np.random.Generator(np.random.PCG64(w.pulse_seed))
    dms = rng.uniform(50.0, 2000.0, n)
    widths_s = np.exp(rng.uniform(np.log(64e-6), np.log(16e-3), n))
    snrs = rng.uniform(snr_range[0], snr_range[1], n)
    n_w = np.maximum(1, np.rint(widths_s / w.tsamp)).astype(np.int64)
    amps = snrs * 16.0 / (np.sqrt(w.nchans) * np.sqrt(n_w))
    slot = w.nsamp // n
    out = []
    for i in range(n):
        span = int(max_delay(float(dms[i]))) + int(n_w[i])
        room = slot - span
        base = i * slot
        if room <= 0:
            # the dispersed pulse does not fit its slot: keep it at the slot start
            t0 = base
        else:
            t0 = base + int(rng.integers(0, room))
        if t0 + span >= w.nsamp:
            continue
        out.append(Pulse(float(dms[i]), int(t0), int(n_w[i]), float(amps[i])))
    return out


def make_filterbank(w: Workload, pulses: Sequence[Pulse],
                    delays: Callable[[float], np.ndarray],
                    device="cpu", pitch: int | None = None,
                    chunk_channels: int = 256) -> torch.Tensor:
    """uint8 tensor [nchans][pitch] (first nsamp columns valid, the rest 0).

    delays(dm) -> int array [nchans] of per-channel delays in full-rate
    samples (caller-supplied).
    """
    C, T = w.nchans, w.nsamp
    pitch = T if pitch is None else pitch
    assert pitch >= T
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.data_seed)
    out = torch.zeros((C, pitch), dtype=torch.uint8, device=dev)
    pul = [(p, np.asarray(delays(p.dm), dtype=np.int64)) for p in pulses]
    for c0 in range(0, C, chunk_channels):
        c1 = min(C, c0 + chunk_channels)
        v = torch.randn((c1 - c0, T), generator=gen, device=dev, dtype=torch.float32)
        v.mul_(16.0).add_(128.0)
        for p, d in pul:
            rows = np.repeat(np.arange(c1 - c0, dtype=np.int64), p.n_w)
            cols = (np.repeat(p.t0 + d[c0:c1], p.n_w)
                    + np.tile(np.arange(p.n_w, dtype=np.int64), c1 - c0))
            keep = cols < T
            if keep.any():
                ri = torch.from_numpy(rows[keep]).to(dev)
                ci = torch.from_numpy(cols[keep]).to(dev)
                val = torch.full((ri.numel(),), float(p.amplitude), device=dev)
                v.index_put_((ri, ci), val, accumulate=True)
        v.round_().clamp_(0.0, 255.0)
        out[c0:c1, :T] = v.to(torch.uint8)
    return out


def noise_filterbank(nchans: int, nsamp: int, seed: int, device="cpu",
                     mean=128.0, std=16.0) -> torch.Tensor:
    """Plain seeded noise, uint8 [nchans][nsamp]."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    v = torch.randn((nchans, nsamp), generator=gen, device=dev, dtype=torch.float32)
    return v.mul_(std).add_(mean).round_().clamp_(0.0, 255.0).to(torch.uint8)


# Differentiable form: 1024 channels over 300 MHz, 65536 float samples
# ~N(0, 1), 1024 trials DM 0..511.5 step 0.5, one pulse at DM 400.
ADJ_1024 = Workload("adjoint-1024ch-65536", 1024, 1508.0, -0.29296875, 64e-6, 65536,
                    ((0.0, 0.5, 1024, 1),), 0, 0.0, 3)
# its finite-difference check size: 256 channels, 4096 samples, DM 0..127.5
ADJ_256 = Workload("adjoint-256ch-4096", 256, 1508.0, -1.171875, 64e-6, 4096,
                   ((0.0, 0.5, 256, 1),), 0, 0.0, 4)


def float_filterbank(w: Workload, pulses: Sequence[Pulse],
                     delays: Callable[[float], np.ndarray], device="cpu",
                     noise: bool = True) -> torch.Tensor:
    """float32 [nchans][nsamp]: N(0, 1) noise (seeded) plus box pulses of
    amplitude A (delays supplied by the caller)."""
    dev = torch.device(device)
    C, T = w.nchans, w.nsamp
    if noise:
        gen = torch.Generator(device=dev)
        gen.manual_seed(w.data_seed)
        x = torch.randn((C, T), generator=gen, device=dev, dtype=torch.float32)
    else:
        x = torch.zeros((C, T), device=dev, dtype=torch.float32)
    for p in pulses:
        d = np.asarray(delays(p.dm), dtype=np.int64)
        rows = np.repeat(np.arange(C, dtype=np.int64), p.n_w)
        cols = np.repeat(p.t0 + d, p.n_w) + np.tile(np.arange(p.n_w, dtype=np.int64), C)
        keep = cols < T
        ri = torch.from_numpy(rows[keep]).to(dev)
        ci = torch.from_numpy(cols[keep]).to(dev)
        x.index_put_((ri, ci), torch.full((ri.numel(),), float(p.amplitude), device=dev),
                     accumulate=True)
    return x


def channel_weights(nchans: int, seed: int, device="cpu") -> torch.Tensor:
    """Per-channel weights ~U[0.5, 1.5] (seeded)."""
    gen = torch.Generator(device=torch.device(device))
    gen.manual_seed(seed)
    return torch.rand(nchans, generator=gen, device=device, dtype=torch.float32) + 0.5


def clipped_ska_ranges(dm_max: float) -> tuple:
    """The 4096-channel plan's DM ranges clipped at dm_max, plus
    (2000, 2, ., dec 16) above DM 2000."""
    out = []
    for (lo, step, ndm, dec) in SKA_4096.ranges + ((2000.0, 2.0, 1 << 30, 16),):
        if lo >= dm_max:
            break
        n = min(ndm, int(np.ceil((dm_max - lo) / step)))
        out.append((lo, step, n, dec))
    return tuple(out)


def batched_beams(n: int = 32, seed: int = PULSE_SEED + 2) -> list:
    """Uneven beams: channels 1024 or 4096 over the same 300 MHz band,
    lengths U{2^17..2^20}, DM_max ~ U[500, 3000] with clipped plans."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beams = []
    for i in range(n):
        C = int(rng.choice([1024, 4096]))
        T = int(rng.integers(1 << 17, (1 << 20) + 1))
        dm_max = float(rng.uniform(500.0, 3000.0))
        foff = -300.0 / C
        beams.append(Workload(f"beam{i}-{C}ch-{T}", C, 1508.0, foff, 64e-6, T,
                              clipped_ska_ranges(dm_max), 8192, 6.0, 10 + i))
    return beams


def small_beams(n: int = 128, seed: int = PULSE_SEED + 3) -> list:
    """Many short beams (a multi-beam receiver's blocks of a few seconds):
    channels 512 or 1024 over the same 300 MHz band, lengths U{2^15..2^16},
    DM_max ~ U[100, 400] with clipped plans."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beams = []
    for i in range(n):
        C = int(rng.choice([512, 1024]))
        T = int(rng.integers(1 << 15, (1 << 16) + 1))
        dm_max = float(rng.uniform(100.0, 400.0))
        foff = -300.0 / C
        beams.append(Workload(f"short{i}-{C}ch-{T}", C, 1508.0, foff, 64e-6, T,
                              clipped_ska_ranges(dm_max), 8192, 6.0, 300 + i))
    return beams


# Record layout of a single-pulse candidate (16 bytes, the library's format).
CANDIDATE_RECORD = np.dtype([("dm_index", "<u4"), ("t", "<u4"), ("width", "<u2"),
                             ("range", "u1"), ("reserved", "u1"), ("snr", "<f4")])


def candidate_field(range_ndm: Sequence[int], range_len: Sequence[int], n_pulses: int,
                    n_noise: int, seed: int, snr_quantum: float = 0.0,
                    threshold: float = 6.0) -> np.ndarray:
    """Seeded synthetic candidate list with the structure of a single-pulse
    search's output, sorted by (dm_index, t), one record per (dm_index, t).

    * pulses: a range r, a centre trial and time, a peak SNR U[8, 40] and a
      half-extent h U{1..40} trials; trial c+k carries a record at
      t_c + round(slope*k) (slope U[-3, 3]) with SNR falling linearly to
      the threshold at |k| = h + 1, plus 0-3 weaker side records per trial at
      gaps U{2..24} samples;
    * noise: uniform (range, trial, t) with SNR threshold + Exp(0.5);
    * snr_quantum > 0 rounds every SNR to a multiple of it (equal SNRs);
    * dm_index is global: the ranges' trials concatenated in order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    offs = np.concatenate([[0], np.cumsum(range_ndm)]).astype(np.int64)
    recs = []  # (dm_global, t, width, range, snr)

    def add(r, d, t, snr):
        if 0 <= d < range_ndm[r] and 0 <= t < range_len[r]:
            recs.append((int(offs[r] + d), int(t), int(rng.integers(1, 64)), r, float(snr)))

    live = [r for r in range(len(range_ndm)) if range_ndm[r] > 0 and range_len[r] > 0]
    for _ in range(n_pulses if live else 0):
        r = int(rng.choice(live))
        c = int(rng.integers(0, range_ndm[r]))
        tc = int(rng.integers(0, range_len[r]))
        peak = rng.uniform(8.0, 40.0)
        h = int(rng.integers(1, 41))
        slope = rng.uniform(-3.0, 3.0)
        for k in range(-h, h + 1):
            s = threshold + (peak - threshold) * (1.0 - abs(k) / (h + 1)) + rng.normal(0, 0.3)
            t = tc + int(round(slope * k))
            add(r, c + k, t, s)
            for _ in range(int(rng.integers(0, 4))):
                add(r, c + k, t + int(rng.choice([-1, 1])) * int(rng.integers(2, 25)),
                    threshold + rng.uniform(0.0, 1.0) * (s - threshold))
    for _ in range(n_noise if live else 0):
        r = int(rng.choice(live))
        add(r, int(rng.integers(0, range_ndm[r])), int(rng.integers(0, range_len[r])),
            threshold + rng.exponential(0.5))
    out = np.zeros(len(recs), dtype=CANDIDATE_RECORD)
    if recs:
        a = np.array(recs, dtype=np.float64)
        out["dm_index"] = a[:, 0].astype(np.uint32)
        out["t"] = a[:, 1].astype(np.uint32)
        out["width"] = a[:, 2].astype(np.uint16)
        out["range"] = a[:, 3].astype(np.uint8)
        snr = a[:, 4]
        if snr_quantum > 0:
            snr = np.round(snr / snr_quantum) * snr_quantum
        out["snr"] = snr.astype(np.float32)
    # one record per (dm_index, t): the first drawn
    key = out["dm_index"].astype(np.int64) * (1 << 32) + out["t"].astype(np.int64)
    _, first = np.unique(key, return_index=True)
    out = out[np.sort(first)]
    return out[np.lexsort((out["t"], out["dm_index"]))]
