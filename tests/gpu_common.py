"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and compare it with the oracle."""
from __future__ import annotations

import numpy as np
import torch

from paper_1912_07704_gb300.api import Plan, candidates_from_device

SNR_TOL = 1e-4  # absolute SNR tolerance against the FP64 oracle


def run_gpu(plan: Plan, x, W: int, thr: float, capacity: int = 1 << 16, want_snr=True):
    """Dedisperse + search on the GPU.  Returns (flat dd, flat snr, sorted
    candidates, total count, nsamp).  With want_snr the search runs twice:
    with the B(t) output (exhaustive widths) and without it (width blocks
    bounded below the threshold skipped); both candidate lists must agree."""
    d, nsamp = plan.device_input(x)
    out = plan.dedisperse_device(d, nsamp)
    snr = torch.full_like(out, float("nan")) if want_snr else None
    cands, count, snr = plan.sps_search_device(out, nsamp, W, thr, capacity, snr_out=snr)
    torch.cuda.synchronize()
    total = int(count.item())
    got = candidates_from_device(cands, count, capacity)
    if want_snr:
        c2, n2, _ = plan.sps_search_device(out, nsamp, W, thr, capacity)
        torch.cuda.synchronize()
        assert int(n2.item()) == total
        if total <= capacity:  # on overflow, which records are stored is unspecified
            assert np.array_equal(candidates_from_device(c2, n2, capacity), got)
    return out, snr, got, total, nsamp


def oracle_candidates(oracle, rows_y, W, thr, dm_offset, rng, windows=None, clip=None):
    """Oracle candidate dict {(dm, t): Candidate} and fragile key set for the
    given rows {row_index: int64 series}; windows {row: (t_lo, t_hi)};
    clip = (c16, max_iters) for k-sigma clipped statistics."""
    solid, fragile, B = {}, set(), {}
    for i, y in rows_y.items():
        lo, hi = windows[i] if windows else (0, y.size)
        c, b, wb, mu, sg = oracle.search_row(y, W, thr, dm_offset + i, rng, lo, hi, clip=clip)
        B[i] = (lo, b, wb, mu, sg)
        for cc in c:
            key = (cc.dm_index, cc.t)
            if cc.fragile:
                fragile.add(key)
            else:
                solid[key] = cc
    return solid, fragile, B


def compare_candidate_lists(gpu, solid, fragile, keep=lambda dm, t: True):
    """Candidate lists equal away from fragile decisions; SNR within tolerance."""
    g = {(int(c["dm_index"]), int(c["t"])): c for c in gpu if keep(int(c["dm_index"]), int(c["t"]))}
    missing = [k for k in solid if k not in g]
    extra = [k for k in g if k not in solid and k not in fragile]
    assert not missing, f"oracle candidates missing on GPU: {missing[:10]}"
    assert not extra, f"GPU candidates not in oracle list: {extra[:10]}"
    for k, oc in solid.items():
        gc = g[k]
        assert int(gc["range"]) == oc.range, k
        assert abs(float(gc["snr"]) - oc.snr) <= SNR_TOL, (k, float(gc["snr"]), oc.snr)
        assert int(gc["width"]) == oc.width, (k, int(gc["width"]), oc.width)
    return len(solid)


def check_snr_rows(snr_view: torch.Tensor, rows: dict, B: dict):
    """GPU B(t) against the oracle's for the listed rows/windows."""
    worst = 0.0
    for i in rows:
        lo, b, *_ = B[i]
        g = snr_view[i, lo:lo + b.size].double().cpu().numpy()
        d = np.abs(g - b)
        worst = max(worst, float(d.max()) if d.size else 0.0)
        assert d.size == 0 or d.max() <= SNR_TOL, (i, float(d.max()), int(d.argmax()) + lo)
    return worst
