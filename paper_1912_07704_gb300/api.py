"""Pythonic face of the C ABI (torch supplies device memory and streams).

Every computation runs in libaa_gb300.so; this module only allocates torch
buffers of the sizes the plan requests (arXiv:1912.07704 Sec. 2.3: memory is
requested before it is allocated) and passes raw pointers.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import abi


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class RangeLayout:
    ndm: int
    dec: int
    maxshift: int
    dm_offset: int
    dm_lo: float
    dm_step: float
    nsamp_dec: int
    length: int
    pitch: int
    row_offset: int

    @property
    def dms(self) -> np.ndarray:
        return np.array([self.dm_lo + i * self.dm_step for i in range(self.ndm)])


class Plan:
    """A bound-on-demand dedispersion + single-pulse search plan."""

    def __init__(self, nchans: int, fch1: float, foff: float, tsamp: float, ranges):
        ranges = [tuple(r) for r in ranges]
        arr = (abi.aa_dm_range * len(ranges))(
            *[abi.aa_dm_range(float(a), float(b), int(n), int(d)) for (a, b, n, d) in ranges])
        desc = abi.aa_plan_desc(int(nchans), float(fch1), float(foff), float(tsamp), len(ranges),
                                ctypes.cast(arr, ctypes.POINTER(abi.aa_dm_range)))
        self.handle = abi.aa_plan_create(desc)
        self.nchans = int(nchans)
        self.fch1, self.foff, self.tsamp = float(fch1), float(foff), float(tsamp)
        self.ranges = ranges

    @classmethod
    def from_workload(cls, w) -> "Plan":
        return cls(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges)

    @classmethod
    def from_filterbank(cls, header, ranges) -> "Plan":
        """Plan for the channels and sampling of a filterbank file header
        (abi.aa_fil_header, see read_filterbank)."""
        return cls(header.nchans, header.fch1_mhz, header.foff_mhz, header.tsamp_s, ranges)

    # lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            abi.aa_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # strategy ---------------------------------------------------------------
    def query(self, nsamp: int, max_width: int = 0) -> abi.aa_plan_info:
        return abi.aa_plan_query(self.handle, nsamp, max_width)

    def layout(self, nsamp: int) -> list:
        out = []
        for r in range(len(self.ranges)):
            i = abi.aa_plan_range(self.handle, nsamp, r)
            out.append(RangeLayout(i.ndm, i.dec, i.maxshift, i.dm_offset, i.dm_lo, i.dm_step,
                                   i.nsamp_dec, i.length, i.pitch, i.row_offset))
        return out

    def shifts(self, r: int) -> np.ndarray:
        return abi.aa_plan_shifts(self.handle, r, self.ranges[r][2], self.nchans)

    def set_sps_clip(self, c16: int, max_iters: int) -> None:
        """k-sigma clipped statistics for later searches (k = c16/16,
        max_iters passes; 0 = plain mean and sigma)."""
        abi.aa_plan_set_sps_clip(self.handle, c16, max_iters)

    def set_sps_ladder(self, growth_x16: int) -> None:
        """Sparse boxcar width ladder for later searches (0: every width)."""
        abi.aa_plan_set_sps_ladder(self.handle, growth_x16)

    def set_sps_decimated(self, base_widths: int) -> None:
        """Decimated boxcar width ladder for later searches (0: every width)."""
        abi.aa_plan_set_sps_decimated(self.handle, base_widths)

    def set_subband(self, r: int, band_channels: int, coarse_trials: int) -> None:
        """Sub-band dedispersion (an approximation) for range r."""
        abi.aa_plan_set_subband(self.handle, r, band_channels, coarse_trials)

    def set_fdmt(self, r: int) -> None:
        """FDMT-style tree dedispersion (an approximation) for range r."""
        abi.aa_plan_set_fdmt(self.handle, r)

    def set_strategy(self, r: int, strategy: int) -> None:
        """Dedispersion strategy of range r: abi.AA_DEDISP_DIRECT or
        abi.AA_DEDISP_GROUPED (same result, different grouping of the sums)."""
        abi.aa_plan_set_strategy(self.handle, r, strategy)

    def autotune(self, nsamp_probe: int, cache_path=None):
        """Pick the dedispersion tile shapes of every range by timing them on
        the bound device (see aa_plan_autotune)."""
        self.bind()
        abi.aa_plan_autotune(self.handle, nsamp_probe, cache_path)

    def bind(self, device=None):
        dev = torch.cuda.current_device() if device is None else int(device)
        abi.aa_plan_bind(self.handle, dev)

    # device path --------------------------------------------------------------
    def device_input(self, x) -> tuple:
        """Copy/pad a [nchans][nsamp] uint8 array to a device tensor whose row
        pitch meets the library's 16-byte rule.  Returns (tensor, nsamp)."""
        t = torch.as_tensor(x)
        assert t.dtype == torch.uint8 and t.dim() == 2 and t.shape[0] == self.nchans
        nsamp = t.shape[1]
        pitch = self.query(nsamp).in_pitch_min
        d = torch.zeros((self.nchans, pitch), dtype=torch.uint8, device="cuda")
        d[:, :nsamp].copy_(t, non_blocking=False)
        return d, nsamp

    def alloc_output(self, nsamp: int) -> torch.Tensor:
        return torch.empty(self.query(nsamp).dd_elems, dtype=torch.float32, device="cuda")

    def alloc_workspace(self, nbytes: int) -> torch.Tensor:
        return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")

    def dedisperse_device(self, d_in: torch.Tensor, nsamp: int, out=None, ws=None,
                          stream=None) -> torch.Tensor:
        self.bind()
        info = self.query(nsamp)
        out = self.alloc_output(nsamp) if out is None else out
        ws = self.alloc_workspace(info.dedisp_ws_bytes) if ws is None else ws
        assert out.numel() >= info.dd_elems and ws.numel() >= info.dedisp_ws_bytes
        abi.aa_dedisperse_device(self.handle, d_in.data_ptr(), nsamp, d_in.stride(0),
                                 out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return out

    def sps_search_device(self, dd: torch.Tensor, nsamp: int, max_width: int, threshold: float,
                          capacity: int = 1 << 20, snr_out=None, ws=None, cands=None, count=None,
                          stream=None):
        """Returns (cands uint8 tensor [capacity*16], count uint64 tensor [1], snr_out)."""
        self.bind()
        info = self.query(nsamp, max_width)
        ws = self.alloc_workspace(info.sps_ws_bytes) if ws is None else ws
        cands = (torch.empty(max(capacity, 1) * 16, dtype=torch.uint8, device="cuda")
                 if cands is None else cands)
        count = torch.zeros(1, dtype=torch.int64, device="cuda") if count is None else count
        abi.aa_sps_search_device(self.handle, nsamp, dd.data_ptr(), max_width, threshold,
                                 cands.data_ptr(), capacity, count.data_ptr(),
                                 0 if snr_out is None else snr_out.data_ptr(),
                                 ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return cands, count, snr_out

    def fused_ws_bytes(self, nsamp: int, max_width: int, stripe_trials: int = 0) -> tuple:
        """(workspace bytes, byte offset of the search workspace inside it) of
        search_fused_device."""
        return abi.aa_search_fused_ws_bytes(self.handle, nsamp, max_width, stripe_trials)

    def search_fused_device(self, x: torch.Tensor, nsamp: int, max_width: int, threshold: float,
                            capacity: int = 1 << 20, stripe_trials: int = 0, snr_out=None,
                            ws=None, cands=None, count=None, stream=None):
        """Dedispersion + search in stripes of trials (see aa_search_fused_device):
        returns (cands, count, ws); the search workspace for sps_order_device is
        ws[fused_ws_bytes(...)[1]:]."""
        self.bind()
        assert x.dtype == torch.uint8 and x.is_cuda and x.dim() == 2 and x.stride(1) == 1
        nbytes, _ = self.fused_ws_bytes(nsamp, max_width, stripe_trials)
        ws = self.alloc_workspace(nbytes) if ws is None else ws
        cands = (torch.empty(max(capacity, 1) * 16, dtype=torch.uint8, device="cuda")
                 if cands is None else cands)
        count = torch.zeros(1, dtype=torch.int64, device="cuda") if count is None else count
        abi.aa_search_fused_device(self.handle, x.data_ptr(), nsamp, x.stride(0), max_width,
                                   threshold, stripe_trials, cands.data_ptr(), capacity,
                                   count.data_ptr(), 0 if snr_out is None else snr_out.data_ptr(),
                                   ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return cands, count, ws

    def postprocess_scratch(self, nsamp: int, max_width: int, capacity: int) -> torch.Tensor:
        """Device scratch for sps_order_device / peaks2d_device."""
        self.bind()
        n = abi.aa_postprocess_ws_bytes(self.handle, nsamp, max_width, capacity)
        return torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")

    def sps_order_device(self, nsamp: int, max_width: int, ws: torch.Tensor, cands: torch.Tensor,
                         count: torch.Tensor, capacity: int, out=None, tmp=None, stream=None):
        """Candidates of the search that used workspace `ws`, in (dm_index, t)
        order, into `out` (uint8 [capacity*16]); returns `out`."""
        self.bind()
        out = (torch.empty(max(capacity, 1) * 16, dtype=torch.uint8, device="cuda")
               if out is None else out)
        tmp = self.postprocess_scratch(nsamp, max_width, capacity) if tmp is None else tmp
        abi.aa_sps_order_device(self.handle, nsamp, max_width, ws.data_ptr(), cands.data_ptr(),
                                count.data_ptr(), capacity, out.data_ptr(), tmp.data_ptr(),
                                tmp.numel(), _stream_handle(stream))
        return out

    def peaks2d_device(self, nsamp: int, max_width: int, sorted_cands: torch.Tensor,
                       count: torch.Tensor, capacity: int, dm_radius: int, t_radius: int,
                       out=None, npeaks=None, tmp=None, stream=None):
        """2-D DM-time peaks of an ordered list; returns (out, npeaks)."""
        self.bind()
        out = (torch.empty(max(capacity, 1) * 16, dtype=torch.uint8, device="cuda")
               if out is None else out)
        npeaks = torch.zeros(1, dtype=torch.int64, device="cuda") if npeaks is None else npeaks
        tmp = self.postprocess_scratch(nsamp, max_width, capacity) if tmp is None else tmp
        abi.aa_candidates_peaks2d_device(self.handle, nsamp, max_width, sorted_cands.data_ptr(),
                                         count.data_ptr(), capacity, dm_radius, t_radius,
                                         out.data_ptr(), npeaks.data_ptr(), tmp.data_ptr(),
                                         tmp.numel(), _stream_handle(stream))
        return out, npeaks

    # differentiable form ------------------------------------------------------
    def f32_forward(self, x: torch.Tensor, w: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """y = sum_c w_c x[c][t + s(c,d)] for float x [nchans][>= nsamp] (row
        stride = pitch); returns the flat output buffer (layout of the u8 path)."""
        self.bind()
        nsamp = x.shape[1]
        out = self.alloc_output(nsamp) if out is None else out
        abi.aa_dedisperse_f32_device(self.handle, x.data_ptr(), nsamp, x.stride(0), w.data_ptr(),
                                     out.data_ptr(), _stream_handle(stream))
        return out

    def f32_adjoint(self, x: torch.Tensor, w: torch.Tensor, gy: torch.Tensor, stream=None):
        self.bind()
        nsamp = x.shape[1]
        gx = torch.empty_like(x)
        gw = torch.empty_like(w)
        ws = self.alloc_workspace(self.query(nsamp).f32_ws_bytes)
        abi.aa_dedisperse_f32_adjoint_device(self.handle, x.data_ptr(), nsamp, x.stride(0),
                                             w.data_ptr(), gy.data_ptr(), gx.data_ptr(),
                                             gw.data_ptr(), ws.data_ptr(), ws.numel(),
                                             _stream_handle(stream))
        return gx, gw

    def f32_mse(self, x: torch.Tensor, w: torch.Tensor, template: torch.Tensor, grad=False,
                stream=None):
        """(loss [float64 scalar tensor], gx or None, gw or None)."""
        self.bind()
        nsamp = x.shape[1]
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = self.alloc_workspace(self.query(nsamp).f32_ws_bytes)
        gx = torch.empty_like(x) if grad else None
        gw = torch.empty_like(w) if grad else None
        abi.aa_dedisperse_f32_mse_device(self.handle, x.data_ptr(), nsamp, x.stride(0),
                                         w.data_ptr(), template.data_ptr(), loss.data_ptr(),
                                         gx.data_ptr() if grad else 0,
                                         gw.data_ptr() if grad else 0,
                                         ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return loss[0], gx, gw

    def range_views(self, flat: torch.Tensor, nsamp: int) -> list:
        """[ndm_r][L_r] views of a flat output buffer, one per range."""
        views = []
        for g in self.layout(nsamp):
            v = flat[g.row_offset:g.row_offset + g.ndm * g.pitch].view(g.ndm, g.pitch)
            views.append(v[:, :g.length])
        return views

    # host-buffer path (library-owned results) ------------------------------
    def dedisperse(self, host, stream=None) -> "DDResult":
        h = host if isinstance(host, np.ndarray) else host.numpy()
        assert h.dtype == np.uint8 and h.ndim == 2 and h.shape[0] == self.nchans
        assert h.strides[1] == 1
        res = abi.aa_dedisperse(self.handle, h.ctypes.data, h.shape[1], h.strides[0],
                                _stream_handle(stream))
        return DDResult(self, res)

    def sps_search(self, dd: "DDResult", max_width: int, threshold: float,
                   capacity: int = 1 << 20, stream=None):
        """Sorted candidate records (numpy structured array) and the total found."""
        h, st = abi.aa_sps_search(self.handle, dd.handle, max_width, threshold, capacity,
                                  _stream_handle(stream))
        return _candidates_array(h)


class _DeviceArray:
    """Zero-copy description of a library-owned float buffer."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


class DDResult:
    """Library-owned dedispersed output (device memory)."""

    def __init__(self, plan: Plan, handle: int):
        self.plan = plan
        self.handle = handle

    def view(self) -> tuple:
        return abi.aa_dd_result_view(self.handle)

    def to_tensor(self) -> torch.Tensor:
        """Copy of the output buffer as a torch tensor (for inspection/tests)."""
        ptr, nsamp = self.view()
        n = self.plan.query(nsamp).dd_elems
        return torch.as_tensor(_DeviceArray(ptr, n), device="cuda").clone()

    def close(self):
        if self.handle:
            abi.aa_dd_result_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def candidates_from_device(cands: torch.Tensor, count: torch.Tensor, capacity: int) -> np.ndarray:
    """Device candidate buffer -> sorted numpy structured array."""
    n = min(int(count.item()), capacity)
    raw = cands[: n * 16].cpu().numpy()
    arr = raw.view(abi.CANDIDATE_DTYPE).copy()
    order = np.lexsort((arr["t"], arr["dm_index"]))
    return arr[order]


class _CandidatesOwner:
    """Destroys a library candidate list when the last numpy view of it goes."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            abi.aa_candidates_destroy(self.h)
        except Exception:
            pass


def _candidates_array(h) -> tuple:
    """Zero-copy numpy view (structured records) of a library candidate list,
    and the total found; the list is freed with the last view."""
    try:
        ptr, stored, total = abi.aa_candidates_view(h)
    except Exception:
        abi.aa_candidates_destroy(h)
        raise
    if not stored:
        abi.aa_candidates_destroy(h)
        return np.zeros(0, dtype=abi.CANDIDATE_DTYPE), total
    nbytes = stored * abi.CANDIDATE_DTYPE.itemsize
    buf = (ctypes.c_char * nbytes).from_address(ptr)
    buf.owner = _CandidatesOwner(h)
    return np.frombuffer(buf, dtype=abi.CANDIDATE_DTYPE, count=stored), total


class Pipeline:
    """Host-buffer pipeline over same-sized blocks (see aa_pipeline_create):
    submit() queues a block of uint8 [nchans][>= nsamp] host memory (keep it
    unchanged until its wait() returns), wait() returns its sorted candidate
    records and the total found.  Uploads and read-backs overlap the search
    of the neighbouring blocks."""

    def __init__(self, plan: Plan, nsamp: int, max_width: int, threshold: float,
                 capacity: int = 1 << 20, depth: int = 2):
        plan.bind()
        self.plan = plan
        self.nsamp = int(nsamp)
        self.handle = abi.aa_pipeline_create(plan.handle, nsamp, max_width, threshold, capacity,
                                             depth)
        self._held = {}

    def submit(self, host) -> int:
        h = host if isinstance(host, np.ndarray) else host.numpy()
        assert h.dtype == np.uint8 and h.ndim == 2 and h.shape[0] == self.plan.nchans
        assert h.strides[1] == 1 and h.shape[1] >= self.nsamp
        t = abi.aa_pipeline_submit(self.handle, h.ctypes.data, h.strides[0])
        self._held[t] = h  # the library reads it until wait(t)
        return t

    def wait(self, ticket: int):
        try:
            h, st = abi.aa_pipeline_wait(self.handle, ticket)
        finally:
            self._held.pop(ticket, None)
        return _candidates_array(h)

    def close(self):
        if getattr(self, "handle", None):
            abi.aa_pipeline_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several beams searched by one CUDA graph (see aa_batch_create and
    aa_batch_set_branches).  The plans must outlive the batch."""

    def __init__(self, plans, nsamps, max_width, threshold, capacity=1 << 24, wave_budget=0):
        for p in plans:
            p.bind()
        self.plans = list(plans)
        self.nsamps = [int(n) for n in nsamps]
        self.handle = abi.aa_batch_create([p.handle for p in plans], self.nsamps, max_width,
                                          threshold, capacity, wave_budget)

    def input_view(self, beam: int) -> torch.Tensor:
        """The library-owned device input of a beam as a uint8 tensor
        [nchans][pitch] (zero-copy)."""
        ptr, pitch = abi.aa_batch_input(self.handle, beam)
        C = self.plans[beam].nchans

        class _U8:
            __cuda_array_interface__ = {"shape": (C, pitch), "typestr": "|u1",
                                        "data": (ptr, False), "version": 3, "strides": None}
        return torch.as_tensor(_U8(), device="cuda")

    def dd_view(self, beam: int) -> torch.Tensor:
        """The beam's dedispersed series after a completed run (beams of the
        last wave only), as a float32 tensor of the plan's dd_elems (zero-copy,
        layout of Plan.dedisperse_device; split it with Plan.range_views)."""
        ptr = abi.aa_batch_dd_view(self.handle, beam)
        n = self.plans[beam].query(self.nsamps[beam]).dd_elems

        class _F32:
            __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4",
                                        "data": (ptr, False), "version": 3, "strides": None}
        return torch.as_tensor(_F32(), device="cuda")

    def info(self) -> tuple:
        return abi.aa_batch_info(self.handle)

    def set_branches(self, branches: int):
        """0: persistent work-queue kernels per stage; k >= 1: each beam's own
        kernels on k concurrent graph branches (see aa_batch_set_branches)."""
        abi.aa_batch_set_branches(self.handle, int(branches))

    def run(self, stream=None):
        abi.aa_batch_run(self.handle, _stream_handle(stream))

    def candidates(self, stream=None):
        """Sorted records (beam in the `reserved` field) and the total found."""
        h, st = abi.aa_batch_candidates(self.handle, _stream_handle(stream))
        return _candidates_array(h)

    def close(self):
        if getattr(self, "handle", None):
            abi.aa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Streaming continuous-batching search server (see aa_server_create)."""

    def __init__(self, plan, nbeams, chunk_nsamp, max_width, threshold, capacity=1 << 20,
                 budget=0, max_slots=8):
        plan.bind()
        self.plan = plan
        self.chunk_nsamp = int(chunk_nsamp)
        self.handle = abi.aa_server_create(plan.handle, nbeams, chunk_nsamp, max_width, threshold,
                                           capacity, budget, max_slots)

    def submit(self, beam: int, host_chunk: np.ndarray, arrival=None) -> int:
        """Queue the next chunk of a beam; host_chunk (uint8 [nchans][>= N],
        unit stride rows) must stay valid until the chunk completes."""
        assert host_chunk.dtype == np.uint8 and host_chunk.strides[1] == 1
        t = abi.aa_server_clock() if arrival is None else arrival
        return abi.aa_server_submit(self.handle, beam, host_chunk.ctypes.data,
                                    host_chunk.strides[0], t)

    def poll(self) -> tuple:
        return abi.aa_server_poll(self.handle)

    def drain(self):
        abi.aa_server_drain(self.handle)

    def result(self, ticket: int):
        """(status, aa_chunk_info, candidates array or None)."""
        st, info, h = abi.aa_server_result(self.handle, ticket)
        arr = None
        if h:
            arr, _ = _candidates_array(h)
        return st, info, arr

    def stats(self):
        return abi.aa_server_stats(self.handle)

    @staticmethod
    def clock() -> float:
        return abi.aa_server_clock()

    def close(self):
        if getattr(self, "handle", None):
            abi.aa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -- filterbank files ------------------------------------------------------------

def read_filterbank(path, t0: int = 0, nsamp: int | None = None, pinned: bool = True):
    """Header and time samples [t0, t0 + nsamp) of an 8-bit SIGPROC filterbank
    file, as (abi.aa_fil_header, uint8 tensor [nsamp][nchans]) in host memory
    (pinned by default, ready for an asynchronous copy)."""
    h = abi.aa_fil_read_header(path)
    n = h.nsamples - t0 if nsamp is None else int(nsamp)
    buf = torch.empty((max(n, 0), h.nchans), dtype=torch.uint8,
                      pin_memory=pinned and torch.cuda.is_available())
    abi.aa_fil_read_block(path, h, t0, n, buf.data_ptr())
    return h, buf


def corner_turn(tm: torch.Tensor, pitch: int | None = None, stream=None) -> torch.Tensor:
    """Device corner turn of a time-major uint8 block [nsamp][nchans] into a
    channel-major [nchans][pitch] tensor (pitch >= nsamp, default nsamp rounded
    up to 16, the dedispersion input's row alignment)."""
    assert tm.is_cuda and tm.dtype == torch.uint8 and tm.dim() == 2
    nsamp, nchans = tm.shape
    pitch = (nsamp + 15) // 16 * 16 if pitch is None else int(pitch)
    out = torch.zeros((nchans, pitch), dtype=torch.uint8, device=tm.device)
    abi.aa_corner_turn_device(tm.data_ptr(), nsamp, nchans, tm.stride(0), out.data_ptr(), pitch,
                              _stream_handle(stream))
    return out
