"""Throughput of the dedispersion + single-pulse-search hot path.

One step = decimation + dedispersion of every DM range + the single-pulse
search (statistics, exhaustive boxcar widths 1..W, peak finding, widths) on
the 4096-channel, 2^20-sample (67.1 s) SKA-like plan (4250 DM trials over four
ranges with decimation 1/2/4/8, W = 8192), input resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank searches its
own beam (independent data, same plan; weak scaling, no data-path
collective); value = all ranks' DM-trial samples / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trial samples/s (4096-ch SKA-like plan, dedispersion + single-pulse search)"
UNIT = "DM-trial samples/s"
SM_MAX_MHZ_DEFAULT = 2070.0
# Minimal lane instructions per boxcar width-sample on sm_103a: running-sum
# add, normalising FMA, and half of a three-input max.
BOXCAR_OPS_PER_WS = 2.5


def workload(name: str):
    from paper_1912_07704_gb300 import synth
    import dataclasses
    if name == "ska":
        return synth.SKA_4096
    if name == "ska-small":
        # same channels, plan and widths, 2^17 samples: the profiling case
        return dataclasses.replace(synth.SKA_4096, name="ska-4096ch-2^17", nsamp=1 << 17)
    raise ValueError(name)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_totals(seconds: float, units: float):
    """Whole-job (time, units) over all ranks: the slowest rank's time and the
    sum of the units every rank processed.  Ranks work on independent beams, so
    this is the only cross-rank exchange (host-side, gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, units
    tt = torch.tensor([seconds], dtype=torch.float64)
    uu = torch.tensor([units], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def build_input(plan, w, device):
    """Seeded synthetic filterbank on the device (pulse delays from the
    library's own plan arithmetic, one single-DM plan per pulse)."""
    from paper_1912_07704_gb300 import synth
    from paper_1912_07704_gb300.api import Plan

    def delays(dm):
        with Plan(w.nchans, w.fch1, w.foff, w.tsamp, [(float(dm), 0.0, 1, 1)]) as p1:
            return p1.shifts(0)[0]

    pulses = synth.pulses_ska(w, lambda dm: int(delays(dm).max()))
    pitch = plan.query(w.nsamp).in_pitch_min
    return synth.make_filterbank(w, pulses, delays, device=device, pitch=pitch)


# DRAM bytes per launch of the dominant kernels, from one ncu capture of the
# small SKA-like case (2^17 samples, same plan) scaled to the full launch by its
# output samples (traffic grows in proportion: input and output both scale with
# the series length).  Each entry names the capture it comes from; set it to None
# when the kernel changes until it is captured again.
NCU_TRAFFIC = {
    ("dedisperse_u8", "grouped"): {
        "small_read_bytes": 542_687_232, "small_write_bytes": 740_074_496,
        "small_output_samples": 1500 * 128687,
        "capture": "profiles/dedisperse_grouped_u8_ska-4096ch-2^17.md"},
    ("sps_boxcar", "pruned"): {
        "small_read_bytes": 947_282_688, "small_write_bytes": 42_682_624,
        "small_output_samples": 1500 * 128687,
        "capture": "profiles/sps_boxcar_ska-4096ch-2^17.md"},
}


def workload_algorithmics(plan, w):
    from paper_1912_07704_gb300 import abi
    lay = plan.layout(w.nsamp)
    dm_samples = sum(g.ndm * g.length for g in lay)
    adds, executed = {}, {}
    for r, g in enumerate(lay):
        key = "dedisperse_u8" if g.dec == 1 else "dedisperse_u16"
        a = g.ndm * g.length * w.nchans
        adds[key] = adds.get(key, 0) + a
        # the grouped strategy executes (pre-sum adds + group adds) / direct adds of them
        info = abi.aa_plan_range(plan.handle, w.nsamp, r)
        executed[key] = executed.get(key, 0) + a * (info.grouped_work if info.strategy else 1.0)
    # width-samples: sum over rows and start times of min(W, L - t)
    ws = 0
    for g in lay:
        L, W = g.length, w.max_width
        full = max(0, L - W + 1) * W
        tail = sum(range(1, min(W, L)))  # t > L-W: L-t widths
        ws += g.ndm * (full + tail)
    in_bytes = w.nchans * w.nsamp
    dd_bytes = 4 * dm_samples
    return dict(dm_samples=dm_samples, adds=adds, executed_adds=executed, width_samples=ws,
                in_bytes=in_bytes, dd_bytes=dd_bytes, lay=lay)


def subband_bands(dec: int) -> int:
    """Bench sub-band width: as wide as 16-bit partial sums allow, at most 64."""
    return min(64, 65535 // (255 * dec) // 8 * 8)


SUBBAND_COARSE = 16


def strided_rows(ndm: int, count: int, k: int = 0) -> list:
    """Trial indices of one range for an oracle sample: `count` trials
    evenly spaced over [0, ndm) including both ends; with count = 1, the
    k-th of a sequence that strides over the range (successive k land on
    trials far apart, so K steps of one trial cover the range evenly)."""
    if ndm <= 0:
        return []
    if count > 1:
        return sorted(set(np.linspace(0, ndm - 1, count).round().astype(int).tolist()))
    # golden-ratio stride: k -> frac(k * 0.618...) * ndm
    return [int((k * 0.6180339887498949) % 1.0 * ndm)]


def run_oracle_sample(w, x_host, rows_per_range: int, threads: int, subband: bool = False,
                      k: int = 0, fdmt: bool = False):
    """Oracle (CPU) on a bounded sample: `rows_per_range` full-length DM trials
    of every range, strided over the range (see strided_rows; k selects the
    trial of a one-trial sample), decimated inputs prepared outside the timed
    part and amortised over all trials; with `subband`, the oracle's sub-band
    form (the same sum at the effective delays).  Returns (DM-trial samples,
    seconds, cores, desc)."""
    from oracle import oracle as o
    cores = o.set_threads(threads)
    pl = o.plan(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, w.nsamp)
    if subband:  # effective delays and lengths of the sub-band form
        for g in pl:
            eff, rmax, s2max = o.subband_delays(w.nchans, w.fch1, w.foff, w.tsamp, g,
                                                subband_bands(g.dec), SUBBAND_COARSE)
            g.shifts = eff.astype(np.int32)
            g.length = max(0, g.nsamp_dec - (rmax + s2max))
    if fdmt:  # effective delays of the tree form (same lengths)
        for g in pl:
            g.shifts = o.fdmt_table(w.nchans, w.fch1, w.foff, g)
    t_dec = 0.0
    inputs = []
    for g in pl:
        t = time.perf_counter()
        inputs.append(o.range_input(x_host, g.dec))
        t_dec += time.perf_counter() - t
    ntrials = sum(g.ndm for g in pl)
    samples, t_rows, nrows = 0, 0.0, 0
    for g, xr in zip(pl, inputs):
        for i in strided_rows(g.ndm, rows_per_range, k):
            t = time.perf_counter()
            y = o.dedisperse_row(xr, g.shifts[i], 0, g.length)
            o.search_row(y, w.max_width, w.threshold, g.dm_offset + int(i), 0)
            t_rows += time.perf_counter() - t
            samples += g.length
            nrows += 1
    secs = t_rows + t_dec * nrows / ntrials
    how = ("evenly spaced over each range incl. both ends" if rows_per_range > 1 else
           "a different trial per step, striding over each range")
    desc = (f"{rows_per_range} full-length DM trial(s) per range ({nrows} of {ntrials}; {how}), "
            f"time extrapolated to all trials by output samples, decimation time amortised "
            f"over all trials" + (", sub-band form" if subband else "")
            + (", FDMT tree form" if fdmt else ""))
    return samples, secs, cores, desc


def bench_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1912_07704_gb300 import synth
    import torch
    w = workload(args.workload)
    from oracle import oracle as o
    d1 = lambda dm: o.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)
    pulses = synth.pulses_ska(w, lambda dm: int(d1(dm).max()))
    x = synth.make_filterbank(w, pulses, d1, device="cpu").numpy()
    threads = os.cpu_count() or 1
    for j in range(args.warmup):
        run_oracle_sample(w, x, 1, threads, k=args.steps + j)
    tot_s, tot_t, cores, desc = 0, 0.0, 1, ""
    for j in range(args.steps):
        s, t, cores, desc = run_oracle_sample(w, x, 1, threads, k=j)
        tot_s += s
        tot_t += t
    v = tot_s / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _strategy_name(info) -> str:
    if info.strategy == 3:
        return (f"FDMT tree ({info.fdmt_depths} depths, largest {info.fdmt_max_rows} rows, "
                f"{info.fdmt_work:.4f} of the direct adds)")
    if info.strategy == 2:
        return (f"subband (bands of {info.subband_channels} ch, coarse trials of "
                f"{info.subband_coarse_trials}, {info.subband_work:.3f} of the direct adds, "
                f"max delay {info.maxshift})")
    return "grouped" if info.strategy == 1 else "direct"


def bench_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1912_07704_gb300 import abi, synth
    from paper_1912_07704_gb300.api import Plan, candidates_from_device

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("gloo")
    w = workload(args.workload)
    plan = Plan.from_workload(w)
    if args.strategy == "subband":
        # bands as wide as the 16-bit partial sums allow (at most 64 channels),
        # coarse trials of 16 fine trials
        for r, rg in enumerate(w.ranges):
            plan.set_subband(r, subband_bands(rg[3]), SUBBAND_COARSE)
    elif args.strategy == "fdmt":
        for r in range(len(w.ranges)):
            plan.set_fdmt(r)
    elif args.strategy != "auto":
        for r in range(len(w.ranges)):
            plan.set_strategy(r, abi.AA_DEDISP_GROUPED if args.strategy == "grouped"
                              else abi.AA_DEDISP_DIRECT)
    if args.sps_clip:
        c16, iters = (int(v) for v in args.sps_clip.split(","))
        plan.set_sps_clip(c16, iters)
    if args.sps_ladder:
        plan.set_sps_ladder(args.sps_ladder)
    if args.sps_dec:
        plan.set_sps_decimated(args.sps_dec)
    plan.bind(local)
    info = plan.query(w.nsamp, w.max_width)
    x = build_input(plan, w, "cuda")
    if ws > 1:  # independent beam per rank: perturb the data deterministically
        x[:, : w.nsamp].add_(rank).clamp_(max=255)
    nsamp = w.nsamp
    cap = 1 << 25
    cands = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    if args.fused:
        # dedispersion and search in stripes of trials, statistics summed by
        # the dedispersion kernels: no [ndm][L] series of the whole plan
        fused_bytes, sps_off = plan.fused_ws_bytes(nsamp, w.max_width, args.stripe)
        ws_fused = plan.alloc_workspace(fused_bytes)
        ws_sps = ws_fused[sps_off:]
        device_bytes = fused_bytes

        def step():
            plan.search_fused_device(x, nsamp, w.max_width, w.threshold, cap, args.stripe,
                                     ws=ws_fused, cands=cands, count=count)
    else:
        out = plan.alloc_output(nsamp)
        ws_dd = plan.alloc_workspace(info.dedisp_ws_bytes)
        ws_sps = plan.alloc_workspace(info.sps_ws_bytes)
        device_bytes = info.dd_elems * 4 + info.dedisp_ws_bytes + info.sps_ws_bytes

        def step():
            plan.dedisperse_device(x, nsamp, out=out, ws=ws_dd)
            plan.sps_search_device(out, nsamp, w.max_width, w.threshold, cap, ws=ws_sps,
                                   cands=cands, count=count)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    alg = workload_algorithmics(plan, w)
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    clocks.start()
    abi.aa_profile_enable(True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    abi.aa_profile_enable(False)
    prof = abi.profile_snapshot()
    clk = clocks.stop()
    t, units = job_totals(ev0.elapsed_time(ev1) / 1e3, alg["dm_samples"] * args.steps)
    ncand = int(count.item())
    value = units / t
    step_s = t / args.steps
    launches = sum(v[0] for v in prof.values())

    # end to end through the host-buffer pipeline of the C ABI: every step
    # uploads its block from page-locked host memory and reads its ordered
    # candidate list back; two blocks in flight, so step k+1's upload and
    # step k's read-back overlap the searches
    e2e = None
    if not args.no_e2e:
        from paper_1912_07704_gb300.api import Pipeline
        host = torch.empty((w.nchans, nsamp), dtype=torch.uint8, pin_memory=True)
        host.copy_(x[:, :nsamp])
        hn = host.numpy()
        depth = 2
        pl = Pipeline(plan, nsamp, w.max_width, w.threshold, cap, depth=depth)

        def run_blocks(n):
            d2h, pending = 0, []
            for _ in range(n):
                pending.append(pl.submit(hn))
                if len(pending) == depth:
                    arr, total = pl.wait(pending.pop(0))
                    d2h += 16 + arr.nbytes  # status words + records
                    del arr
            for t in pending:
                arr, total = pl.wait(t)
                d2h += 16 + arr.nbytes
                del arr
            return d2h

        run_blocks(max(3, args.warmup))  # page-locked result blocks reach steady state
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        d2h = run_blocks(args.steps)
        torch.cuda.synchronize()
        te, units_e = job_totals(time.perf_counter() - t0, alg["dm_samples"] * args.steps)
        pl.close()
        e2e = {"value": units_e / te, "unit": UNIT,
               "h2d_bytes_per_step": w.nchans * nsamp,
               "d2h_bytes_per_step": int(d2h / args.steps),
               "path": f"aa_pipeline_submit / aa_pipeline_wait, {depth} blocks in flight, "
                       "page-locked host input"}

    # roofline of the dominant kernel, from the live event timings
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", SM_MAX_MHZ_DEFAULT))
    # lane peak from the device the bench ran on: its SM count x 128 integer /
    # FP32 lanes per SM x the measured maximum SM clock
    sm_count = int(torch.cuda.get_device_properties(local).multi_processor_count)
    lane_peak = sm_count * 128 * sm_max * 1e6  # lane instructions / s
    kern = {}
    for name, (n, ms) in prof.items():
        if n:
            kern[name] = {"launches": n, "ms_per_step": ms / args.steps,
                          "share": ms / max(1e-9, sum(v[1] for v in prof.values()))}
    box_s = prof["sps_boxcar"][1] / 1e3 / args.steps
    u8_s = prof["dedisperse_u8"][1] / 1e3 / args.steps
    u16_s = prof["dedisperse_u16"][1] / 1e3 / args.steps
    if box_s > 0:
        kern["sps_boxcar"]["gws_per_s"] = alg["width_samples"] / box_s / 1e9
    for key, s in (("dedisperse_u8", u8_s), ("dedisperse_u16", u16_s)):
        if s > 0:
            kern[key]["gadds_per_s"] = alg["adds"][key] / s / 1e9
            kern[key]["executed_gadds_per_s"] = alg["executed_adds"][key] / s / 1e9
    evaluated = abi.aa_sps_workspace_work(ws_sps.data_ptr(), stream.cuda_stream)
    if box_s > 0:
        kern["sps_boxcar"]["evaluated_width_samples"] = evaluated
        kern["sps_boxcar"]["exhaustive_width_samples"] = alg["width_samples"]
        kern["sps_boxcar"]["gws_evaluated_per_s"] = evaluated / box_s / 1e9
    dominant = max(kern, key=lambda k: kern[k]["ms_per_step"])

    def traffic(key):
        """DRAM bytes per launch of `key` from its ncu capture, scaled to this
        workload's launches by output samples (None without a matching capture)."""
        lay = alg["lay"]
        if key == "sps_boxcar":
            ent, rows = NCU_TRAFFIC.get(("sps_boxcar", "pruned")), lay
        else:
            sel = [r for r, g in enumerate(lay) if (g.dec == 1) == (key == "dedisperse_u8")]
            strat = {("grouped" if abi.aa_plan_range(plan.handle, nsamp, r).strategy else "direct")
                     for r in sel}
            ent = NCU_TRAFFIC.get((key, strat.pop())) if len(strat) == 1 else None
            rows = [lay[r] for r in sel]
        if ent is None or not rows:
            return None, None
        samples = sum(g.ndm * g.length for g in rows)
        scale = samples / ent["small_output_samples"]
        per_launch = (ent["small_read_bytes"] + ent["small_write_bytes"]) * scale / len(rows)
        return per_launch, f"ncu capture {ent['capture']}, scaled x{scale:.2f} by output samples"

    if dominant == "dedisperse_fdmt":
        # HBM-bound gather-adds: every row of every tree depth reads two rows
        # and writes one (32-bit; leaves are 8/16-bit input rows, counted as 4
        # bytes: an upper estimate); rows = fdmt_work x ndm x nchans per range
        fd_s = kern[dominant]["ms_per_step"] / 1e3
        nbytes = 0.0
        for r, g in enumerate(alg["lay"]):
            info = abi.aa_plan_range(plan.handle, nsamp, r)
            if info.strategy == 3:
                nbytes += info.fdmt_work * g.ndm * w.nchans * g.nsamp_dec * 12
        nl = kern[dominant]["launches"] / max(args.steps, 1)
        achieved = nbytes / fd_s
        hbm_peak = float(peaks.get("hbm_gbs", 6678.2)) * 1e9
        roof = {"kernel": dominant, "bound": "hbm", "achieved": achieved / 1e9, "peak": hbm_peak / 1e9,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "traffic_source": "no capture of the tree kernels",
                "algorithmic_bytes_per_launch": nbytes / max(nl, 1),
                "ops": "per tree row: two rows read and one written, 4 bytes a sample "
                       "(rows = fdmt_work x ndm x nchans); peak = measured HBM copy bandwidth"}
    elif dominant == "sps_boxcar":
        achieved = BOXCAR_OPS_PER_WS * evaluated / box_s
        tb, tnote = traffic("sps_boxcar")
        roof = {"kernel": "sps_boxcar", "bound": "alu", "sm_count": sm_count, "achieved": achieved / 1e9,
                "peak": lane_peak / 1e9, "unit": "Gop/s", "frac": achieved / lane_peak,
                "traffic": tb, "traffic_source": tnote,
                "ops": f"{BOXCAR_OPS_PER_WS} lane instructions per evaluated width-sample "
                       f"(device-counted; blocks bounded below threshold skipped); peak = "
                       f"{sm_count} SMs (device query) x 128 lanes x {sm_max:.0f} MHz"}
    else:
        key = dominant
        s = kern[key]["ms_per_step"] / 1e3
        achieved = alg["adds"].get(key, 0) / s
        executed = alg["executed_adds"].get(key, 0) / s
        tb, tnote = traffic(key)
        nl = kern[key]["launches"] / max(args.steps, 1)
        alg_bytes = sum((w.nchans * g.nsamp_dec * (1 if g.dec == 1 else 2) + 4 * g.ndm * g.length)
                        for g in alg["lay"] if (g.dec == 1) == (key == "dedisperse_u8")) / max(nl, 1)
        roof = {"kernel": key, "bound": "alu", "sm_count": sm_count, "achieved": achieved / 1e9,
                "peak": lane_peak / 1e9, "unit": "Gop/s", "frac": achieved / lane_peak,
                "traffic": tb, "traffic_source": tnote, "algorithmic_bytes_per_launch": alg_bytes,
                "executed_gops": executed / 1e9, "executed_frac": executed / lane_peak,
                "ops": "algorithmic channel-adds (sum over trials of nchans x L) per second; "
                       "executed_* counts the adds the chosen strategy performs (grouped: "
                       "pre-sum adds + group adds); peak = 1 add per lane per clock "
                       f"({sm_count} SMs (device query) x 128 lanes x {sm_max:.0f} MHz)"}
    hbm = float(peaks.get("hbm_gbs", 6678.2))
    eff_in_gbs = alg["dm_samples"] * w.nchans / step_s / 1e9

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        xh = x[:, :nsamp].cpu().numpy()
        s, secs, cores, desc = run_oracle_sample(w, xh, 3, os.cpu_count() or 1,
                                                 subband=args.strategy == "subband",
                                                 fdmt=args.strategy == "fdmt")
        cpu = {"value": s / secs, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": (METRIC.replace("dedispersion", "sub-band dedispersion (approximate)")
                       if args.strategy == "subband" else
                       METRIC.replace("dedispersion", "FDMT tree dedispersion (approximate)")
                       if args.strategy == "fdmt" else METRIC),
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8->int32 (dedispersion), f32 (SNR)",
            "data": "synthetic",
            "config": {"workload": w.name, "nchans": w.nchans, "nsamp": w.nsamp,
                       "dm_trials": sum(g.ndm for g in alg["lay"]), "max_width": w.max_width,
                       "threshold": w.threshold, "parallelism": f"beams x{ws}",
                       "statistics": (f"k-sigma clipped, k = {args.sps_clip.split(',')[0]}/16, "
                                      f"<= {args.sps_clip.split(',')[1]} passes"
                                      if args.sps_clip else "plain mean and sigma"),
                       "widths": (f"sparse ladder, growth {args.sps_ladder}/16 (approximate)"
                                  if args.sps_ladder else
                                  f"decimated ladder, {args.sps_dec} base widths (approximate)"
                                  if args.sps_dec else "every width 1..W"),
                       "dedispersion": [_strategy_name(abi.aa_plan_range(plan.handle, nsamp, r))
                                        for r in range(len(w.ranges))],
                       "l2": (f"inputs larger than L2 ({alg['in_bytes'] / 1e9:.2f} GB filterbank, "
                              f"{alg['dd_bytes'] / 1e9:.2f} GB dedispersed)"),
                       "mode": (f"fused: stripes of {args.stripe or 256} trials, statistics summed "
                                "by the dedispersion kernels" if args.fused else
                                "dedisperse all ranges, then search"),
                       "device_bytes": {"input": alg["in_bytes"], "work": device_bytes,
                                        "candidates": cap * 16}},
            "rtf": (w.nsamp * w.tsamp) / step_s,
            "hbm": {"effective_input_gbs": eff_in_gbs, "frac_of_measured": eff_in_gbs / hbm,
                    "algorithmic_gbs": (alg["in_bytes"] + alg["dd_bytes"]) / step_s / 1e9,
                    "peak_gbs": hbm},
            "roofline": roof,
            "kernels": kern,
            "candidates": ncand,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _time_cuda(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def bench_adjoint(args):
    """Differentiable form (1024 ch, 65536 float samples, 1024 trials): float
    forward, fused MSE loss, loss + gradients (chunked recomputation), next
    to the plain uint8 path on the same plan shape."""
    import torch
    from paper_1912_07704_gb300 import synth
    from paper_1912_07704_gb300.api import Plan
    w = synth.ADJ_1024
    plan = Plan.from_workload(w)
    plan.bind()
    lay = plan.layout(w.nsamp)[0]

    def delays(dm):
        with Plan(w.nchans, w.fch1, w.foff, w.tsamp, [(float(dm), 0.0, 1, 1)]) as p1:
            return p1.shifts(0)[0]

    pulse = [synth.Pulse(400.0, w.nsamp // 4, 16, 1.0)]
    x = synth.float_filterbank(w, pulse, delays, device="cuda")
    wt = synth.channel_weights(w.nchans, w.data_seed + 100, device="cuda")
    tmpl = plan.f32_forward(synth.float_filterbank(w, pulse, delays, device="cuda", noise=False),
                            torch.ones_like(wt))
    y = plan.alloc_output(w.nsamp)
    t_fwd = _time_cuda(lambda: plan.f32_forward(x, wt, out=y), args.steps, args.warmup)
    t_loss = _time_cuda(lambda: plan.f32_mse(x, wt, tmpl), args.steps, args.warmup)
    t_grad = _time_cuda(lambda: plan.f32_mse(x, wt, tmpl, grad=True), args.steps, args.warmup)
    xq = (x * 16 + 128).round().clamp(0, 255).to(torch.uint8)
    dq, nsamp = plan.device_input(xq)
    out = plan.alloc_output(nsamp)
    wsd = plan.alloc_workspace(plan.query(nsamp).dedisp_ws_bytes)
    t_u8 = _time_cuda(lambda: plan.dedisperse_device(dq, nsamp, out=out, ws=wsd), args.steps,
                      args.warmup)
    fma = lay.ndm * lay.length * w.nchans
    line = {"metric": "differentiable dedispersion: loss + gradients per second", "workload": w.name,
            "unit": "ms", "steps": args.steps, "warmup": args.warmup,
            "f32_forward_ms": t_fwd, "mse_loss_ms": t_loss, "mse_loss_and_grad_ms": t_grad,
            "u8_dedisperse_same_plan_ms": t_u8,
            "forward_tflops": 2 * fma / t_fwd / 1e9, "grad_over_forward": t_grad / t_fwd,
            "dm_trial_samples": lay.ndm * lay.length}
    print(json.dumps(line), flush=True)


def bench_batched(args):
    """Batched beams in one CUDA graph vs the beams run one after another
    through the single-beam path, same GPU, same results.  `batched`: 32
    uneven beams (1024/4096 ch, 2^17..2^20 samples, DM_max 500..3000);
    `batched-small`: 128 short beams (512/1024 ch, 2^15..2^16 samples,
    DM_max 100..400)."""
    import torch
    from paper_1912_07704_gb300 import synth
    from paper_1912_07704_gb300.api import Batch, Plan
    small = args.workload == "batched-small"
    beams = synth.small_beams(128) if small else synth.batched_beams(32)
    plans = [Plan.from_workload(w) for w in beams]
    for p in plans:
        p.bind()
    batch = Batch(plans, [w.nsamp for w in beams], 8192, 6.0, capacity=1 << 28)
    dm_samples = 0
    for i, (w, p) in enumerate(zip(beams, plans)):
        def delays(dm, w=w):
            with Plan(w.nchans, w.fch1, w.foff, w.tsamp, [(float(dm), 0.0, 1, 1)]) as p1:
                return p1.shifts(0)[0]
        pulses = synth.pulses_ska(w, lambda dm: int(delays(dm).max()), n=4)
        x = synth.make_filterbank(w, pulses, delays, device="cuda")
        batch.input_view(i)[:, : w.nsamp].copy_(x)
        del x
        dm_samples += p.query(w.nsamp).dm_trial_samples
    torch.cuda.synchronize()
    forms = {}
    arr, total = None, None
    for k in [int(v) for v in args.batch_branches.split(",")]:
        batch.set_branches(k)
        forms[k] = _time_cuda(batch.run, args.steps, args.warmup)
        arr_k, total_k = batch.candidates()
        if arr is None:
            arr, total = arr_k, total_k
        else:
            # past the capacity the stored subset depends on arrival order: totals only
            same = total_k == total and (total > (1 << 28) or
                                         (len(arr_k) == len(arr) and bool((arr_k == arr).all())))
            assert same, f"graph form {k} found other candidates ({total_k} vs {total})"
    best = int(args.batch_branches.split(",")[0])  # the reported form: the first listed
    t_batch = forms[best]
    nwaves, nbytes = batch.info()
    # the same beams through the single-beam path, one after another
    info = [p.query(w.nsamp, 8192) for p, w in zip(plans, beams)]
    out = torch.empty(max(i.dd_elems for i in info), dtype=torch.float32, device="cuda")
    wsd = torch.empty(max(i.dedisp_ws_bytes for i in info), dtype=torch.uint8, device="cuda")
    wss = torch.empty(max(i.sps_ws_bytes for i in info), dtype=torch.uint8, device="cuda")
    cands = torch.empty((1 << 25) * 16, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    views = [batch.input_view(i) for i in range(len(beams))]

    def one_by_one():
        for i, (p, w) in enumerate(zip(plans, beams)):
            p.dedisperse_device(views[i], w.nsamp, out=out, ws=wsd)
            p.sps_search_device(out, w.nsamp, 8192, 6.0, 1 << 25, ws=wss, cands=cands, count=count)

    t_single = _time_cuda(one_by_one, args.steps, args.warmup)
    line = {"metric": "batched beams: DM-trial samples/s",
            "workload": "128 short beams" if small else "32 uneven beams",
            "unit": "DM-trial samples/s", "steps": args.steps, "warmup": args.warmup,
            "batched_value": dm_samples / (t_batch / 1e3),
            "single_beam_sum_value": dm_samples / (t_single / 1e3),
            "batched_ms": t_batch, "single_beams_ms": t_single, "speedup": t_single / t_batch,
            "batched_form": "persistent work queues" if best == 0 else f"{best} graph branches",
            "ms_by_form": {("persistent" if k == 0 else f"branches_{k}"): v for k, v in forms.items()},
            "waves": nwaves, "batch_device_bytes": nbytes, "dm_trial_samples": dm_samples,
            "candidates": total}
    print(json.dumps(line), flush=True)


def bench_stream(args):
    """16 beams of 4096 channels streamed in 2^16-sample chunks arriving as
    Poisson processes at 1.2x real time (per beam), searched by the
    continuous-batching server; then the same chunks submitted in lockstep
    (saturated) for the sustained real-time factor."""
    import dataclasses
    import time as _t
    import torch
    from paper_1912_07704_gb300 import synth
    from paper_1912_07704_gb300.api import Plan, Server
    base = synth.SKA_4096
    nbeams, N, nchunk = 16, 1 << 16, args.stream_chunks
    plan = Plan.from_workload(base)
    plan.bind()

    def delays(dm):
        with Plan(base.nchans, base.fch1, base.foff, base.tsamp, [(float(dm), 0.0, 1, 1)]) as p1:
            return p1.shifts(0)[0]

    series = []
    for b in range(nbeams):
        w = dataclasses.replace(base, nsamp=N * nchunk, index=100 + b)
        pulses = synth.pulses_ska(w, lambda dm: int(delays(dm).max()), n=2)
        series.append(synth.make_filterbank(w, pulses, delays, device="cuda"))
    host = [[torch.empty((base.nchans, N), dtype=torch.uint8, pin_memory=True) for _ in range(2)]
            for _ in range(nbeams)]
    chunk_s = N * base.tsamp
    rng = np.random.Generator(np.random.PCG64(base.pulse_seed + 5))
    events = []
    for b in range(nbeams):
        t = 0.0
        for k in range(nchunk):
            t += rng.exponential(chunk_s / 1.2)
            events.append((t, b, k))
    events.sort()

    def run(lockstep: bool):
        srv = Server(plan, nbeams, N, base.max_width, base.threshold, capacity=1 << 22, max_slots=8)
        tickets = {}
        t0 = srv.clock()
        order = sorted(events, key=lambda e: (e[2], e[1])) if lockstep else events
        for (ta, b, k) in order:
            if not lockstep:
                while srv.clock() < t0 + ta:
                    srv.poll()
                    _t.sleep(0.0005)
            prev = tickets.get((b, k - 2))
            while prev is not None and srv.result(prev)[0] == 1:  # buffer still in use
                srv.poll()
                _t.sleep(0.0005)
            buf = host[b][k % 2]
            buf.copy_(series[b][:, k * N:(k + 1) * N])
            tickets[(b, k)] = srv.submit(b, buf.numpy())
            srv.poll()
        srv.drain()
        st = srv.stats()
        ncand = sum(len(srv.result(t)[2]) for t in tickets.values())
        srv.close()
        return st, ncand

    st_rt, ncand = run(lockstep=False)
    st_sat, _ = run(lockstep=True)
    data_s = nbeams * nchunk * chunk_s
    # per-slot device work area of the two search paths (the server runs the
    # fused one), and the slots a 48 GiB budget would admit with each
    from paper_1912_07704_gb300 import abi as _abi
    block = st_rt.history_nsamp + N
    qi = plan.query(block, base.max_width)
    unfused = qi.dd_elems * 4 + qi.dedisp_ws_bytes + qi.sps_ws_bytes
    fused, _ = _abi.aa_search_fused_ws_bytes(plan.handle, block, base.max_width, 0)
    resident = 2 * nbeams * base.nchans * plan.query(block).in_pitch_min
    per_slot = lambda work: work + (1 << 22) * 16 + 4096
    budget = 48 << 30
    line = {"metric": "streaming serve: chunk latency and sustained real-time factor",
            "workload": f"{nbeams} beams x {base.nchans} ch, 2^16-sample chunks, 1.2x real-time Poisson",
            "chunks": nbeams * nchunk, "history_nsamp": st_rt.history_nsamp, "slots": st_rt.slots,
            "max_in_flight": st_rt.max_in_flight,
            "latency_p50_s": st_rt.latency_p50, "latency_p99_s": st_rt.latency_p99,
            "latency_max_s": st_rt.latency_max, "rtf_at_1.2x_arrivals": data_s / st_rt.span,
            "saturated_rtf": data_s / st_sat.span, "saturated_latency_p99_s": st_sat.latency_p99,
            "candidates": ncand,
            "slot_work_bytes": {"fused": fused, "unfused": unfused},
            "slots_in_48GiB_budget": {"fused": (budget - resident) // per_slot(fused),
                                      "unfused": (budget - resident) // per_slot(unfused)}}
    print(json.dumps(line), flush=True)


def bench_cornerturn(args):
    """Corner turn of a time-major 4096-channel x 2^20-sample block (the
    filterbank-file input path) into channel-major rows: HBM-bound, one byte
    read and one written per sample."""
    import torch
    from paper_1912_07704_gb300 import abi
    C, T = 4096, 1 << 20
    tm = torch.randint(0, 256, (T, C), dtype=torch.uint8, device="cuda")
    out = torch.empty((C, T), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    run = lambda: abi.aa_corner_turn_device(tm.data_ptr(), T, C, C, out.data_ptr(), T,
                                            stream.cuda_stream)
    for _ in range(args.warmup):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3 / args.steps
    ok = bool(torch.equal(out[:, :4096].cpu(), tm[:4096].cpu().T))
    hbm = float(load_peaks().get("hbm_gbs", 6678.2))
    gbs = 2 * C * T / s / 1e9
    print(json.dumps({"metric": "corner turn: bytes moved per second", "workload": "4096ch x 2^20",
                      "unit": "GB/s", "value": gbs, "ms": s * 1e3, "frac_of_measured_hbm": gbs / hbm,
                      "peak_gbs": hbm, "steps": args.steps, "warmup": args.warmup,
                      "sampled_check": ok}), flush=True)


def bench_postprocess(args):
    """Candidate post-processing of the 4096-channel SKA-like search output:
    device ordering of the boxcar CTAs' runs into (dm_index, t) order, then
    the 2-D DM-time peak filter (+-8 trials, +-256 samples).  The search runs
    once, untimed; each timed step orders and filters the whole list."""
    import torch
    from paper_1912_07704_gb300 import abi, synth
    from paper_1912_07704_gb300.api import Plan

    w = synth.SKA_4096
    plan = Plan.from_workload(w)
    plan.bind(0)
    info = plan.query(w.nsamp, w.max_width)
    x = build_input(plan, w, "cuda")
    nsamp, cap, R, Tr = w.nsamp, 1 << 25, 8, 256
    out = plan.alloc_output(nsamp)
    ws = plan.alloc_workspace(info.sps_ws_bytes)
    cands, count, _ = plan.sps_search_device(plan.dedisperse_device(x, nsamp, out=out), nsamp,
                                             w.max_width, w.threshold, cap, ws=ws)
    del x
    srt = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    peaks = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    npeaks = torch.zeros(1, dtype=torch.int64, device="cuda")
    tmp = plan.postprocess_scratch(nsamp, w.max_width, cap)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    order = lambda: plan.sps_order_device(nsamp, w.max_width, ws, cands, count, cap, out=srt,
                                          tmp=tmp)
    filt = lambda: plan.peaks2d_device(nsamp, w.max_width, srt, count, cap, R, Tr, out=peaks,
                                       npeaks=npeaks, tmp=tmp)
    for _ in range(args.warmup):
        order()
        filt()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_order = t_filt = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        ev[0].record(stream)
        order()
        ev[1].record(stream)
        flush.fill_(2)
        ev[2].record(stream)
        filt()
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_order += ev[0].elapsed_time(ev[1]) / args.steps
        t_filt += ev[2].elapsed_time(ev[3]) / args.steps
    n = min(int(count.item()), cap)
    k = int(npeaks.item())
    lay = plan.layout(nsamp)
    slots = sum(g.ndm * -(-g.length // 4094) for g in lay)
    # algorithmic bytes: ordering reads and writes every record once plus the
    # run headers (24 B) and a count/source/destination entry (3 x 8 B, written
    # and read) per boxcar CTA; the filter reads every record once, writes and
    # scans an 8-byte flag per record and writes the kept records
    b_order = 32 * n + slots * (24 + 2 * 24)
    b_filt = 16 * n + 3 * 8 * n + 16 * k + 16 * n
    hbm = float(load_peaks().get("hbm_gbs", 6678.2))
    tot_ms = t_order + t_filt
    print(json.dumps({
        "metric": "candidates post-processed per second (device ordering + 2-D peaks)",
        "value": n / (tot_ms / 1e3), "unit": "candidates/s", "steps": args.steps,
        "warmup": args.warmup, "workload": "ska-4096ch-2^20 search output, W=8192, thr 6",
        "candidates": n, "peaks": k, "dm_radius": R, "t_radius": Tr,
        "order_ms": t_order, "peaks2d_ms": t_filt, "l2": "flushed before each call",
        "roofline": {"order": {"bound": "hbm", "achieved": b_order / t_order / 1e6, "peak": hbm,
                               "unit": "GB/s", "frac": b_order / t_order / 1e6 / hbm},
                     "peaks2d": {"bound": "hbm", "achieved": b_filt / t_filt / 1e6, "peak": hbm,
                                 "unit": "GB/s", "frac": b_filt / t_filt / 1e6 / hbm}}}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["ska", "ska-small", "adjoint", "batched", "batched-small", "stream",
                                           "cornerturn", "postprocess"],
                    default="ska")
    ap.add_argument("--stream-chunks", type=int, default=6)
    ap.add_argument("--strategy", choices=["auto", "direct", "grouped", "subband", "fdmt"],
                    default="auto",
                    help="dedispersion strategy of every range (auto: the plan's choice; "
                         "subband / fdmt: the approximate two-stage / tree sums, a different "
                         "metric)")
    ap.add_argument("--sps-clip", default="",
                    help="C16,ITERS: k-sigma clipped statistics (k = C16/16), e.g. 48,4")
    ap.add_argument("--batch-branches", default="8,0",
                    help="batched workloads: graph forms to time (0 = persistent work-queue kernels, "
                         "k = each beam's kernels on k concurrent branches); the first is reported "
                         "(8 = the library's default), the others are listed beside it")
    ap.add_argument("--sps-dec", type=int, default=0,
                    help="W0: decimated boxcar width ladder with W0 base widths (approximate), e.g. 32")
    ap.add_argument("--sps-ladder", type=int, default=0,
                    help="G16: sparse boxcar width ladder of growth G16/16 (approximate), e.g. 24")
    ap.add_argument("--fused", action="store_true",
                    help="fused dedispersion -> search in stripes of trials (no full series buffer)")
    ap.add_argument("--stripe", type=int, default=0, help="trials per stripe of --fused (0: 256)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "adjoint":
        bench_adjoint(args)
    elif args.workload in ("batched", "batched-small"):
        bench_batched(args)
    elif args.workload == "stream":
        bench_stream(args)
    elif args.workload == "cornerturn":
        bench_cornerturn(args)
    elif args.workload == "postprocess":
        bench_postprocess(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
