"""Python face of the CPU oracle (``aa_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it.  It shares no code with the CUDA path.

The C file holds the arithmetic (FP64 delays/statistics/SNR, exact int64
sums); this module only marshals numpy arrays and assembles the per-range
plan and candidate lists in the same plain terms:

* plan (brute-force DM grid, per-range decimation): DM_i = dm_lo + i*dm_step,
  shifts in decimated samples, L_r = floor(T/dec_r) - max shift;
* dedispersion, boxcar SNR and thresholded local maxima as in the C header;
* candidate fragility: a candidate whose decision hinges on a margin smaller
  than the FP32/FP64 disagreement allowed for the GPU path is flagged so that
  list comparisons can exclude it on both sides.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Margins that make a candidate "fragile" (FP32 GPU vs FP64 oracle may decide
# differently): distance of B to the threshold, and the margins of the local
# maximum comparisons and of the width argmax.
FRAGILE_THR = 1e-3
FRAGILE_CMP = 2e-4


def build(force: bool = False) -> str:
    """Compile aa_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        vp = ctypes.c_void_p
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_f_top.argtypes = [f64, f64, i32]
        L.oracle_f_top.restype = f64
        L.oracle_shifts.argtypes = [i32, f64, f64, f64, f64, i32, vp]
        L.oracle_shifts.restype = i32
        L.oracle_decimate.argtypes = [vp, i32, i64, i64, i32, vp, i64]
        L.oracle_decimate.restype = None
        L.oracle_dedisperse.argtypes = [vp, i32, i32, i64, vp, i64, i64, vp]
        L.oracle_dedisperse.restype = None
        L.oracle_moments.argtypes = [vp, i64, ctypes.POINTER(f64), ctypes.POINTER(f64)]
        L.oracle_moments.restype = None
        L.oracle_subband_rel.argtypes = [i32, f64, f64, f64, f64, i32, i32, vp]
        L.oracle_subband_rel.restype = None
        L.oracle_fdmt_delays.argtypes = [i32, f64, f64, i64, vp]
        L.oracle_fdmt_delays.restype = None
        L.oracle_moments_clipped.argtypes = [vp, i64, i32, i32, ctypes.POINTER(f64),
                                             ctypes.POINTER(f64), ctypes.POINTER(i64)]
        L.oracle_moments_clipped.restype = None
        L.oracle_boxcar.argtypes = [vp, i64, f64, f64, i32, i64, i64, vp, vp, vp]
        L.oracle_boxcar_widths.argtypes = [vp, i64, f64, f64, i32, vp, i64, i64, vp, vp, vp]
        L.oracle_boxcar_widths.restype = None
        L.oracle_boxcar.restype = None
        L.oracle_boxcar_dec.argtypes = [vp, i64, f64, f64, i32, i32, i64, i64, vp, vp, vp, vp]
        L.oracle_boxcar_dec.restype = ctypes.c_int
        L.oracle_peaks.argtypes = [vp, i64, f64, vp, i64]
        L.oracle_peaks.restype = i64
        L.oracle_forward_f64.argtypes = [vp, i32, i64, vp, vp, i64, vp]
        L.oracle_forward_f64.restype = None
        L.oracle_adjoint_f64.argtypes = [vp, i32, i64, vp, vp, i32, vp, i64, vp, vp]
        L.oracle_adjoint_f64.restype = None
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count in use."""
    return int(lib().oracle_set_threads(int(n)))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ----------------------------------------------------------------------------
# Plan
# ----------------------------------------------------------------------------

def shifts(nchans: int, fch1: float, foff: float, tsamp: float, dm: float, dec: int = 1):
    """Per-channel integer delays for one DM, in decimated samples."""
    out = np.empty(nchans, dtype=np.int32)
    lib().oracle_shifts(nchans, fch1, foff, tsamp, float(dm), int(dec), _ptr(out))
    return out


def shifts_near_half(nchans, fch1, foff, tsamp, dm, dec=1) -> int:
    out = np.empty(nchans, dtype=np.int32)
    return int(lib().oracle_shifts(nchans, fch1, foff, tsamp, float(dm), int(dec), _ptr(out)))


@dataclass
class OracleRange:
    dm_lo: float
    dm_step: float
    ndm: int
    dec: int
    dms: np.ndarray = field(repr=False)
    shifts: np.ndarray = field(repr=False)  # [ndm][nchans] int32
    maxshift: int = 0
    nsamp_dec: int = 0
    length: int = 0
    dm_offset: int = 0


def plan(nchans, fch1, foff, tsamp, ranges, nsamp):
    """Per-range DM list, shift table, max shift and output length."""
    out = []
    off = 0
    for (dm_lo, dm_step, ndm, dec) in ranges:
        dms = np.array([dm_lo + i * dm_step for i in range(ndm)], dtype=np.float64)
        tab = np.stack([shifts(nchans, fch1, foff, tsamp, d, dec) for d in dms]) if ndm else \
            np.zeros((0, nchans), np.int32)
        ms = int(tab.max()) if ndm else 0
        nd = nsamp // dec
        out.append(OracleRange(dm_lo, dm_step, ndm, dec, dms, tab, ms, nd, max(0, nd - ms), off))
        off += ndm
    return out


# ----------------------------------------------------------------------------
# Dedispersion
# ----------------------------------------------------------------------------

def decimate(x: np.ndarray, dec: int) -> np.ndarray:
    """uint8 [C][T] -> uint16 [C][T//dec], summing dec samples."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    C, T = x.shape
    nd = T // dec
    out = np.empty((C, nd), dtype=np.uint16)
    lib().oracle_decimate(_ptr(x), C, T, T, int(dec), _ptr(out), nd)
    return out


def dedisperse_row(xr: np.ndarray, shift_row: np.ndarray, t0: int, t1: int) -> np.ndarray:
    """y[t] for t in [t0, t1) of one DM trial; xr is uint8 or uint16 [C][T_r]."""
    xr = np.ascontiguousarray(xr)
    assert xr.dtype in (np.uint8, np.uint16)
    C, Tr = xr.shape
    sh = np.ascontiguousarray(shift_row, dtype=np.int32)
    assert t0 >= 0 and t1 >= t0
    if t1 > t0:
        assert t1 - 1 + int(sh.max()) < Tr, "window reads past the end of the series"
    out = np.zeros(max(0, t1 - t0), dtype=np.int64)
    lib().oracle_dedisperse(_ptr(xr), xr.itemsize, C, Tr, _ptr(sh), int(t0), int(t1), _ptr(out))
    return out


def range_input(x: np.ndarray, dec: int) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint8) if dec == 1 else decimate(x, dec)


def dedisperse(x, nchans, fch1, foff, tsamp, ranges, rows=None):
    """Full dedispersion: list (per range) of int64 [ndm_r][L_r] (or the listed rows)."""
    C, T = x.shape
    assert C == nchans
    pl = plan(nchans, fch1, foff, tsamp, ranges, T)
    res = []
    for r, rg in enumerate(pl):
        xr = range_input(x, rg.dec)
        sel = range(rg.ndm) if rows is None else rows[r]
        res.append(np.stack([dedisperse_row(xr, rg.shifts[i], 0, rg.length) for i in sel])
                   if len(sel) else np.zeros((0, rg.length), np.int64))
    return pl, res


# ----------------------------------------------------------------------------
# Single-pulse search
# ----------------------------------------------------------------------------

def moments(y: np.ndarray):
    y = np.ascontiguousarray(y, dtype=np.int64)
    mu, sg = ctypes.c_double(), ctypes.c_double()
    lib().oracle_moments(_ptr(y), y.size, ctypes.byref(mu), ctypes.byref(sg))
    return mu.value, sg.value


def moments_clipped(y: np.ndarray, c16: int, max_iters: int):
    """(mu, sigma, kept) of iterative k-sigma clipping, k = c16/16."""
    y = np.ascontiguousarray(y, dtype=np.int64)
    mu, sg, nk = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    lib().oracle_moments_clipped(_ptr(y), y.size, int(c16), int(max_iters), ctypes.byref(mu),
                                 ctypes.byref(sg), ctypes.byref(nk))
    return mu.value, sg.value, nk.value


def row_moments(y: np.ndarray, clip=None):
    """Plain moments, or clipped ones for clip = (c16, max_iters) with
    max_iters > 0."""
    if clip and clip[1] > 0:
        mu, sg, _ = moments_clipped(y, clip[0], clip[1])
        return mu, sg
    return moments(y)


def ladder_widths(W: int, g16: int) -> np.ndarray:
    """Widths 1..W taking part in the sparse width ladder with growth g16/16:
    width chunks of 16 (chunk c = widths 16c+1 .. 16c+16); chunks 0-3 always,
    then c_0 = 4 and c_{n+1} = max(c_n + 1, ceil(c_n * g16 / 16))."""
    nch = -(-W // 16)
    on = np.zeros(nch, bool)
    on[:min(4, nch)] = True
    c = 4
    while c < nch:
        on[c] = True
        c = max(c + 1, -(-(c * g16) // 16))
    return np.repeat(on, 16)[:W]


def boxcar(y: np.ndarray, mu: float, sigma: float, W: int, t0: int = 0, t1: int | None = None,
           wset: np.ndarray | None = None, dec_w0: int | None = None):
    """(B, wbest, margin) for t in [t0, t1); wset: optional bool mask of the
    widths 1..W taking part; dec_w0: the decimated width ladder with W0 =
    dec_w0 base widths (oracle_boxcar_dec), instead of every width."""
    y = np.ascontiguousarray(y, dtype=np.int64)
    n = y.size
    t1 = n if t1 is None else t1
    m = max(0, t1 - t0)
    B = np.empty(m, np.float64)
    wb = np.empty(m, np.int32)
    mg = np.empty(m, np.float64)
    if dec_w0:
        assert wset is None
        return boxcar_dec(y, mu, sigma, W, dec_w0, t0, t1)[:3]
    if m and wset is None:
        lib().oracle_boxcar(_ptr(y), n, float(mu), float(sigma), int(W), int(t0), int(t1),
                            _ptr(B), _ptr(wb), _ptr(mg))
    elif m:
        ws = np.ascontiguousarray(wset, dtype=np.uint8)
        assert ws.size == W
        lib().oracle_boxcar_widths(_ptr(y), n, float(mu), float(sigma), int(W), _ptr(ws), int(t0),
                                   int(t1), _ptr(B), _ptr(wb), _ptr(mg))
    return B, wb, mg


def boxcar_dec(y: np.ndarray, mu: float, sigma: float, W: int, W0: int, t0: int = 0,
               t1: int | None = None):
    """(B, wbest, margin, start of the maximising window) of the decimated
    width ladder with W0 base widths (oracle_boxcar_dec) for t in [t0, t1)."""
    assert W0 >= 2 and W0 % 2 == 0
    y = np.ascontiguousarray(y, dtype=np.int64)
    n = y.size
    t1 = n if t1 is None else t1
    m = max(0, t1 - t0)
    B = np.empty(m, np.float64)
    wb = np.empty(m, np.int32)
    mg = np.empty(m, np.float64)
    sb = np.empty(m, np.int64)
    if m and lib().oracle_boxcar_dec(_ptr(y), n, float(mu), float(sigma), int(W), int(W0), int(t0),
                                     int(t1), _ptr(B), _ptr(wb), _ptr(mg), _ptr(sb)) != 0:
        raise MemoryError("oracle_boxcar_dec: prefix sums")
    return B, wb, mg, sb


def peaks_thr(B: np.ndarray, thr: float) -> np.ndarray:
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.empty(B.size, np.int64)
    n = lib().oracle_peaks(_ptr(B), B.size, float(thr), _ptr(out), B.size)
    return out[:n].copy()


@dataclass
class Candidate:
    dm_index: int  # global DM-trial index (ranges concatenated)
    t: int         # sample index in that range's (decimated) series
    width: int     # boxcar width in samples of that range
    range: int
    snr: float
    fragile: bool = False


def search_row(y: np.ndarray, W: int, thr: float, dm_index: int, rng: int,
               t_lo: int = 0, t_hi: int | None = None, clip=None, wset=None, dec_w0=None):
    """Candidates of one DM series with t in [t_lo, t_hi).

    Returns (candidates, B, wbest, mu, sigma) with B/wbest over [t_lo, t_hi).
    clip = (c16, max_iters) takes mu, sigma from iterative k-sigma clipping;
    wset restricts the widths (bool mask over 1..W, e.g. ladder_widths);
    dec_w0 selects the decimated width ladder with that many base widths.
    Rows with sigma == 0 have B = 0 and no candidates.  Near-decision entries
    (|B - thr| < FRAGILE_THR, neighbour or width-argmax margin < FRAGILE_CMP)
    are flagged fragile; entries just below the threshold that could flip
    into the list are returned as fragile too.
    """
    y = np.ascontiguousarray(y, dtype=np.int64)
    n = y.size
    t_hi = n if t_hi is None else min(t_hi, n)
    mu, sigma = row_moments(y, clip)
    a, b = max(0, t_lo - 1), min(n, t_hi + 1)
    if dec_w0:
        B, wb, mg, sb = boxcar_dec(y, mu, sigma, W, dec_w0, a, b)
    else:
        B, wb, mg = boxcar(y, mu, sigma, W, a, b, wset)
        sb = np.arange(a, b, dtype=np.int64)  # every window starts at its own t
    cands = []
    if sigma == 0.0 or t_hi <= t_lo:
        return cands, B[t_lo - a:t_hi - a], wb[t_lo - a:t_hi - a], mu, sigma
    # The peak decision is oracle_peaks on B over [a, b): a window end is the
    # series end (a missing neighbour, -inf) or lies outside [t_lo, t_hi),
    # so every t in [t_lo, t_hi) is decided with its true neighbours.
    peak_set = set((peaks_thr(B, thr) + a).tolist())
    # only samples within FRAGILE_THR of the threshold or above can matter
    near_idx = np.nonzero(B[t_lo - a:t_hi - a] >= thr - FRAGILE_THR)[0] + t_lo
    for t in near_idx.tolist():
        k = t - a
        v = B[k]
        left = B[k - 1] if t > 0 else -np.inf
        right = B[k + 1] if t + 1 < n else -np.inf
        is_peak = t in peak_set
        # a neighbour holding the same window (a decimated-ladder plateau) is
        # equal by construction on both sides, not a near decision
        same_l = t > 0 and k > 0 and sb[k - 1] == sb[k] and wb[k - 1] == wb[k]
        same_r = t + 1 < n and k + 1 < len(B) and sb[k + 1] == sb[k] and wb[k + 1] == wb[k]
        near = (abs(v - thr) < FRAGILE_THR or (abs(v - left) < FRAGILE_CMP and not same_l)
                or (abs(v - right) < FRAGILE_CMP and not same_r))
        if is_peak or near:
            fragile = near or mg[k] < FRAGILE_CMP
            cands.append(Candidate(dm_index, t, int(wb[k]), rng, float(v), bool(fragile)))
    return cands, B[t_lo - a:t_hi - a], wb[t_lo - a:t_hi - a], mu, sigma


# ----------------------------------------------------------------------------
# Sub-band dedispersion (approximate; exact integer sums of approximated delays)
# ----------------------------------------------------------------------------

def subband_rel(nchans, fch1, foff, tsamp, dm, dec, band) -> np.ndarray:
    """Delay of every channel relative to its band's reference channel."""
    out = np.empty(nchans, dtype=np.int32)
    lib().oracle_subband_rel(int(nchans), float(fch1), float(foff), float(tsamp), float(dm),
                             int(dec), int(band), _ptr(out))
    return out


def subband_delays(nchans, fch1, foff, tsamp, rng: OracleRange, band, coarse):
    """Effective delay table [ndm][nchans] of the sub-band form and the
    largest stage delays (rmax, s2max).

    Channel c of trial i (coarse trial j = i // coarse, middle trial
    i_j = j*coarse + (n_j - 1)//2) is taken at s(c_b, i) + r(c, D_j): the
    reference channel's own delay at the fine DM plus the channel's delay
    relative to the reference at the coarse DM D_j = DM_{i_j}.
    """
    ndm = rng.ndm
    cref = np.array([min((c // band) * band + band - 1, nchans - 1) if foff > 0 else (c // band) * band
                     for c in range(nchans)], dtype=np.int64)
    eff = np.zeros((ndm, nchans), dtype=np.int64)
    rmax = 0
    for j in range((ndm + coarse - 1) // coarse):
        i0 = j * coarse
        nj = min(coarse, ndm - i0)
        ij = i0 + (nj - 1) // 2
        rel = subband_rel(nchans, fch1, foff, tsamp, rng.dms[ij], rng.dec, band).astype(np.int64)
        rmax = max(rmax, int(rel.max()))
        for i in range(i0, i0 + nj):
            eff[i] = rng.shifts[i][cref] + rel
    s2max = int(rng.shifts[:, np.unique(cref)].max()) if ndm else 0
    return eff, rmax, s2max


def dedisperse_subband(x, nchans, fch1, foff, tsamp, rng: OracleRange, band, coarse):
    """y[i][t] = sum_c xr[c][t + eff(i, c)], t < nsamp_dec - (rmax + s2max)."""
    eff, rmax, s2max = subband_delays(nchans, fch1, foff, tsamp, rng, band, coarse)
    xr = range_input(x, rng.dec)
    L = max(0, rng.nsamp_dec - (rmax + s2max))
    out = np.zeros((rng.ndm, L), dtype=np.int64)
    for i in range(rng.ndm):
        if L:
            out[i] = dedisperse_row(xr, eff[i].astype(np.int32), 0, L)
    return out, eff, rmax, s2max


# ----------------------------------------------------------------------------
# FDMT-style tree dedispersion (approximate; exact integer sums of the
# delays the tree's splits give)
# ----------------------------------------------------------------------------

def fdmt_delays(nchans, fch1, foff, D) -> np.ndarray:
    """Per-channel delays of the tree for a whole-band delay of D samples."""
    out = np.empty(nchans, dtype=np.int32)
    lib().oracle_fdmt_delays(int(nchans), float(fch1), float(foff), int(D), _ptr(out))
    return out


def fdmt_bottom(nchans, foff) -> int:
    """The lowest-frequency channel (the one whose delay is the band's)."""
    return nchans - 1 if foff < 0 else 0


def fdmt_table(nchans, fch1, foff, rng: OracleRange) -> np.ndarray:
    """Delay table [ndm][nchans] of the tree form of a range: trial i takes
    the whole-band delay D_i = s(bottom channel, i) of the brute-force plan."""
    b = fdmt_bottom(nchans, foff)
    if rng.ndm == 0:
        return np.zeros((0, nchans), np.int32)
    return np.stack([fdmt_delays(nchans, fch1, foff, int(rng.shifts[i][b])) for i in range(rng.ndm)])


def dedisperse_fdmt(x, nchans, fch1, foff, tsamp, rng: OracleRange):
    """y[i][t] = sum_c xr[c][t + e_i(c)], t < L (the brute-force length:
    the bottom channel keeps its brute-force delay)."""
    tab = fdmt_table(nchans, fch1, foff, rng)
    xr = range_input(x, rng.dec)
    out = np.zeros((rng.ndm, rng.length), dtype=np.int64)
    for i in range(rng.ndm):
        if rng.length:
            out[i] = dedisperse_row(xr, tab[i], 0, rng.length)
    return out, tab


# ----------------------------------------------------------------------------
# Differentiable form (per-channel float weights), FP64
# ----------------------------------------------------------------------------

def forward_f64(x: np.ndarray, w: np.ndarray, shift_table: np.ndarray, L: int) -> np.ndarray:
    """y[d][t] = sum_c w_c x[c][t + s(c,d)] for every row of shift_table [D][C]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    C, T = x.shape
    out = np.zeros((shift_table.shape[0], max(L, 0)), np.float64)
    for d in range(shift_table.shape[0]):
        sh = np.ascontiguousarray(shift_table[d], dtype=np.int32)
        if L > 0:
            assert L - 1 + int(sh.max()) < T
            row = np.empty(L, np.float64)
            lib().oracle_forward_f64(_ptr(x), C, T, _ptr(w), _ptr(sh), L, _ptr(row))
            out[d] = row
    return out


def adjoint_f64(x: np.ndarray, w: np.ndarray, shift_table: np.ndarray, gy: np.ndarray):
    """(gx [C][T], gw [C]) of <gy, y(x, w)> (transpose of the forward)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    gy = np.ascontiguousarray(gy, dtype=np.float64)
    C, T = x.shape
    D, L = gy.shape
    sh = np.ascontiguousarray(shift_table, dtype=np.int32)
    gx = np.zeros((C, T), np.float64)
    gw = np.zeros(C, np.float64)
    if L > 0:
        lib().oracle_adjoint_f64(_ptr(x), C, T, _ptr(w), _ptr(sh), D, _ptr(gy), L, _ptr(gx),
                                 _ptr(gw))
    return gx, gw


def mse_f64(x, w, shift_table, L, template) -> float:
    y = forward_f64(x, w, shift_table, L)
    return float(np.mean((y - template) ** 2)) if y.size else 0.0


# ----------------------------------------------------------------------------
# 2-D DM-time peak filter over a candidate list (post-processing of the
# single-pulse search, Sec. 1: boxcar filters with peak finding)
# ----------------------------------------------------------------------------

def _beaten(dm, t, snr, c_dm, c_t, c_snr):
    """Mask of the records that beat candidate c: a larger SNR, or the same
    SNR and a smaller (dm_index, t) pair."""
    smaller_key = (dm < c_dm) | ((dm == c_dm) & (t < c_t))
    return (snr > c_snr) | ((snr == c_snr) & smaller_key)


def peaks2d(recs: np.ndarray, dm_radius: int, t_radius: int, idx=None) -> np.ndarray:
    """Keep-mask of the 2-D peak filter for the records `idx` (default all).

    recs: structured array with fields dm_index, t, range, snr (any order; the
    SNRs are compared as stored, float32).  Candidate c is kept iff no other
    record of the same range within +-dm_radius trials and +-t_radius samples
    beats it.  Brute force per candidate; when recs is sorted by dm_index the
    records are first narrowed to the candidate's DM window with a binary
    search (a plain lookup), otherwise every record is examined.
    """
    dm = recs["dm_index"].astype(np.int64)
    t = recs["t"].astype(np.int64)
    rg = recs["range"].astype(np.int64)
    snr = recs["snr"].astype(np.float32)
    n = dm.size
    idx = np.arange(n) if idx is None else np.asarray(idx, dtype=np.int64)
    by_dm = n < 2 or bool(np.all(dm[1:] >= dm[:-1]))
    keep = np.ones(idx.size, bool)
    for k, i in enumerate(idx.tolist()):
        if by_dm:
            a = int(np.searchsorted(dm, dm[i] - dm_radius, side="left"))
            b = int(np.searchsorted(dm, dm[i] + dm_radius, side="right"))
        else:
            a, b = 0, n
        sl = slice(a, b)
        near = ((rg[sl] == rg[i]) & (np.abs(dm[sl] - dm[i]) <= dm_radius)
                & (np.abs(t[sl] - t[i]) <= t_radius))
        near[i - a] = False  # a candidate does not suppress itself
        beat = near & _beaten(dm[sl], t[sl], snr[sl], dm[i], t[i], snr[i])
        keep[k] = not bool(beat.any())
    return keep
