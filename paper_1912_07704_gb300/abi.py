"""ctypes binding of include/aa_dedisp.h: one Python function per C entry
point, same names, argument marshalling only.

The shared library is loaded from this package directory (built by
``paper_1912_07704_gb300.build``).  There is no fallback: if the library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaa_gb300.so")

AA_OK = 0
AA_PENDING = 1
AA_WARN_CAND_OVERFLOW = 2
AA_ERR_CONFIG = -1
AA_ERR_NOMEM = -2
AA_ERR_CUDA = -3
AA_ERR_TIMEOUT = -4
AA_ERR_STATE = -5
AA_ERR_ARG = -6


class aa_dm_range(ctypes.Structure):
    _fields_ = [("dm_lo", ctypes.c_double), ("dm_step", ctypes.c_double),
                ("ndm", ctypes.c_int32), ("dec", ctypes.c_int32)]


class aa_plan_desc(ctypes.Structure):
    _fields_ = [("nchans", ctypes.c_int32), ("fch1_mhz", ctypes.c_double),
                ("foff_mhz", ctypes.c_double), ("tsamp_s", ctypes.c_double),
                ("nranges", ctypes.c_int32), ("ranges", ctypes.POINTER(aa_dm_range))]


class aa_range_info(ctypes.Structure):
    _fields_ = [("ndm", ctypes.c_int32), ("dec", ctypes.c_int32), ("maxshift", ctypes.c_int32),
                ("dm_offset", ctypes.c_int32), ("dm_lo", ctypes.c_double),
                ("dm_step", ctypes.c_double), ("nsamp_dec", ctypes.c_int64),
                ("length", ctypes.c_int64), ("pitch", ctypes.c_int64),
                ("row_offset", ctypes.c_int64), ("tile_dms", ctypes.c_int32),
                ("tile_samples", ctypes.c_int32), ("stage_channels", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("span_max", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("strategy", ctypes.c_int32),
                ("grouped_available", ctypes.c_int32), ("grouped_work", ctypes.c_double),
                ("subband_channels", ctypes.c_int32), ("subband_coarse_trials", ctypes.c_int32),
                ("subband_work", ctypes.c_double), ("fdmt_depths", ctypes.c_int32),
                ("fdmt_max_rows", ctypes.c_int32), ("fdmt_work", ctypes.c_double)]


class aa_plan_info(ctypes.Structure):
    _fields_ = [("nchans", ctypes.c_int32), ("nranges", ctypes.c_int32),
                ("ndm_total", ctypes.c_int32), ("ready", ctypes.c_int32),
                ("device", ctypes.c_int32), ("max_width", ctypes.c_int32),
                ("nsamp", ctypes.c_int64), ("in_pitch_min", ctypes.c_int64),
                ("dd_elems", ctypes.c_int64), ("dedisp_ws_bytes", ctypes.c_int64),
                ("sps_ws_bytes", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("host_path_bytes", ctypes.c_int64), ("dm_trial_samples", ctypes.c_int64),
                ("dm_max", ctypes.c_double), ("f32_ws_bytes", ctypes.c_int64)]


class aa_fil_header(ctypes.Structure):
    _fields_ = [("nchans", ctypes.c_int32), ("nbits", ctypes.c_int32), ("nifs", ctypes.c_int32),
                ("data_type", ctypes.c_int32), ("telescope_id", ctypes.c_int32),
                ("machine_id", ctypes.c_int32), ("fch1_mhz", ctypes.c_double),
                ("foff_mhz", ctypes.c_double), ("tsamp_s", ctypes.c_double),
                ("tstart_mjd", ctypes.c_double), ("header_bytes", ctypes.c_int64),
                ("nsamples", ctypes.c_int64), ("source_name", ctypes.c_char * 80)]


class aa_candidate(ctypes.Structure):
    _fields_ = [("dm_index", ctypes.c_uint32), ("t", ctypes.c_uint32),
                ("width", ctypes.c_uint16), ("range", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8), ("snr", ctypes.c_float)]


class aa_chunk_info(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("status", ctypes.c_int32), ("chunk", ctypes.c_int64),
                ("block_start", ctypes.c_int64), ("total", ctypes.c_int64),
                ("arrival", ctypes.c_double), ("admitted", ctypes.c_double),
                ("done", ctypes.c_double)]


class aa_server_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("slots", ctypes.c_int32), ("max_in_flight", ctypes.c_int32),
                ("history_nsamp", ctypes.c_int64), ("latency_p50", ctypes.c_double),
                ("latency_p99", ctypes.c_double), ("latency_max", ctypes.c_double),
                ("span", ctypes.c_double)]


CANDIDATE_DTYPE = np.dtype([("dm_index", "<u4"), ("t", "<u4"), ("width", "<u2"),
                            ("range", "u1"), ("reserved", "u1"), ("snr", "<f4")])
assert CANDIDATE_DTYPE.itemsize == ctypes.sizeof(aa_candidate) == 16

_P = ctypes.c_void_p
_I32, _I64, _F32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
_SIG = {
    "aa_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "aa_last_error": (ctypes.c_char_p, []),
    "aa_plan_create": (ctypes.c_int, [ctypes.POINTER(aa_plan_desc), ctypes.POINTER(_P)]),
    "aa_plan_destroy": (None, [_P]),
    "aa_plan_bind": (ctypes.c_int, [_P, ctypes.c_int]),
    "aa_plan_query": (ctypes.c_int, [_P, _I64, _I32, ctypes.POINTER(aa_plan_info)]),
    "aa_plan_range": (ctypes.c_int, [_P, _I64, _I32, ctypes.POINTER(aa_range_info)]),
    "aa_plan_shifts": (ctypes.c_int, [_P, _I32, _P, _I64]),
    "aa_dedisperse_device": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P, ctypes.c_size_t, _P]),
    "aa_sps_search_device": (ctypes.c_int, [_P, _I64, _P, _I32, _F32, _P, _I64, _P, _P, _P,
                                            ctypes.c_size_t, _P]),
    "aa_workspace_status": (ctypes.c_int, [_P, _P]),
    "aa_sps_workspace_work": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I64)]),
    "aa_dedisperse": (ctypes.c_int, [_P, _P, _I64, _I64, _P, ctypes.POINTER(_P)]),
    "aa_dd_result_view": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "aa_dd_result_destroy": (None, [_P]),
    "aa_sps_search": (ctypes.c_int, [_P, _P, _I32, _F32, _I64, _P, ctypes.POINTER(_P)]),
    "aa_candidates_view": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64),
                                          ctypes.POINTER(_I64)]),
    "aa_candidates_destroy": (None, [_P]),
    "aa_search_fused_ws_bytes": (ctypes.c_int, [_P, _I64, _I32, _I32, ctypes.POINTER(ctypes.c_size_t),
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "aa_search_fused_device": (ctypes.c_int, [_P, _P, _I64, _I64, _I32, _F32, _I32, _P, _I64, _P, _P,
                                              _P, ctypes.c_size_t, _P]),
    "aa_pipeline_create": (ctypes.c_int, [_P, _I64, _I32, _F32, _I64, _I32, ctypes.POINTER(_P)]),
    "aa_pipeline_submit": (ctypes.c_int, [_P, _P, _I64, ctypes.POINTER(_I64)]),
    "aa_pipeline_wait": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_P)]),
    "aa_pipeline_destroy": (None, [_P]),
    "aa_debug_inject": (ctypes.c_int, [_I32, _I64]),
    "aa_fil_read_header": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(aa_fil_header)]),
    "aa_fil_read_block": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(aa_fil_header), _I64, _I64, _P]),
    "aa_corner_turn_device": (ctypes.c_int, [_P, _I64, _I32, _I64, _P, _I64, _P]),
    "aa_plan_set_sps_clip": (ctypes.c_int, [_P, _I32, _I32]),
    "aa_plan_set_subband": (ctypes.c_int, [_P, _I32, _I32, _I32]),
    "aa_plan_set_fdmt": (ctypes.c_int, [_P, _I32]),
    "aa_plan_effective_shifts": (ctypes.c_int, [_P, _I32, _P, _I64]),
    "aa_plan_set_sps_ladder": (ctypes.c_int, [_P, _I32]),
    "aa_plan_set_sps_decimated": (ctypes.c_int, [_P, _I32]),
    "aa_postprocess_ws_bytes": (ctypes.c_int, [_P, _I64, _I32, _I64,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "aa_sps_order_device": (ctypes.c_int, [_P, _I64, _I32, _P, _P, _P, _I64, _P, _P,
                                           ctypes.c_size_t, _P]),
    "aa_candidates_peaks2d_device": (ctypes.c_int, [_P, _I64, _I32, _P, _P, _I64, _I32, _I32, _P,
                                                    _P, _P, ctypes.c_size_t, _P]),
    "aa_sps_search_device_noalloc": (ctypes.c_int, [_P, _I64, _P, _I32, _F32, _P, _I64, _P, _P,
                                                    _P]),
    "aa_dedisperse_f32_device": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P, _P]),
    "aa_dedisperse_f32_adjoint_device": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P, _P, _P, _P,
                                                        ctypes.c_size_t, _P]),
    "aa_dedisperse_f32_mse_device": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P, _P, _P, _P, _P,
                                                    ctypes.c_size_t, _P]),
    "aa_plan_autotune": (ctypes.c_int, [_P, _I64, ctypes.c_char_p]),
    "aa_plan_set_strategy": (ctypes.c_int, [_P, _I32, _I32]),
    "aa_batch_create": (ctypes.c_int, [_P, _P, _I32, _I32, _F32, _I64, _I64, ctypes.POINTER(_P)]),
    "aa_batch_destroy": (None, [_P]),
    "aa_batch_input": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "aa_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "aa_batch_dd_view": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_P)]),
    "aa_batch_run": (ctypes.c_int, [_P, _P]),
    "aa_batch_set_branches": (ctypes.c_int, [_P, _I32]),
    "aa_batch_candidates": (ctypes.c_int, [_P, _P, ctypes.POINTER(_P)]),
    "aa_server_create": (ctypes.c_int, [_P, _I32, _I64, _I32, _F32, _I64, _I64, _I32,
                                        ctypes.POINTER(_P)]),
    "aa_server_destroy": (None, [_P]),
    "aa_server_submit": (ctypes.c_int, [_P, _I32, _P, _I64, ctypes.c_double, ctypes.POINTER(_I64)]),
    "aa_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "aa_server_drain": (ctypes.c_int, [_P]),
    "aa_server_result": (ctypes.c_int, [_P, _I64, ctypes.POINTER(aa_chunk_info), ctypes.POINTER(_P)]),
    "aa_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(aa_server_report)]),
    "aa_server_clock": (ctypes.c_double, []),
    "aa_profile_enable": (ctypes.c_int, [_I32]),
    "aa_profile_read": (ctypes.c_int, [_I32, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)]),
    "aa_profile_kernel_name": (ctypes.c_char_p, [_I32]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libaa_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1912_07704_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_names() -> list:
    return list(_SIG)


class AAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = lib().aa_last_error().decode(errors="replace")
        super().__init__(f"{where}: {status_str(status)}" + (f" ({detail})" if detail else ""))


def status_str(s: int) -> str:
    return lib().aa_status_str(int(s)).decode()


def check(status: int, where: str, ok=(AA_OK,)) -> int:
    if status not in ok:
        raise AAError(status, where)
    return status


# -- thin wrappers: same names as the C entry points --------------------------

def aa_status_str(s):
    return status_str(s)


def aa_last_error():
    return lib().aa_last_error().decode(errors="replace")


def aa_plan_create(desc: aa_plan_desc) -> int:
    h = ctypes.c_void_p()
    check(lib().aa_plan_create(ctypes.byref(desc), ctypes.byref(h)), "aa_plan_create")
    return h.value


def aa_plan_destroy(plan: int) -> None:
    lib().aa_plan_destroy(plan)


def aa_plan_bind(plan: int, device: int) -> None:
    check(lib().aa_plan_bind(plan, int(device)), "aa_plan_bind")


def aa_plan_query(plan: int, nsamp: int, max_width: int = 0) -> aa_plan_info:
    info = aa_plan_info()
    check(lib().aa_plan_query(plan, int(nsamp), int(max_width), ctypes.byref(info)), "aa_plan_query")
    return info


def aa_plan_range(plan: int, nsamp: int, r: int) -> aa_range_info:
    info = aa_range_info()
    check(lib().aa_plan_range(plan, int(nsamp), int(r), ctypes.byref(info)), "aa_plan_range")
    return info


def aa_plan_shifts(plan: int, r: int, ndm: int, nchans: int) -> np.ndarray:
    out = np.empty((ndm, nchans), np.int32)
    check(lib().aa_plan_shifts(plan, int(r), out.ctypes.data, out.size), "aa_plan_shifts")
    return out


def aa_dedisperse_device(plan, d_in, nsamp, in_pitch, d_out, d_ws, ws_bytes, stream) -> None:
    check(lib().aa_dedisperse_device(plan, d_in, int(nsamp), int(in_pitch), d_out, d_ws,
                                     int(ws_bytes), stream), "aa_dedisperse_device")


def aa_sps_search_device(plan, nsamp, d_dd, max_width, threshold, d_cands, capacity, d_count,
                         d_snr_out, d_ws, ws_bytes, stream) -> None:
    check(lib().aa_sps_search_device(plan, int(nsamp), d_dd, int(max_width), float(threshold),
                                     d_cands, int(capacity), d_count, d_snr_out, d_ws,
                                     int(ws_bytes), stream), "aa_sps_search_device")


def aa_workspace_status(d_ws, stream) -> int:
    return lib().aa_workspace_status(d_ws, stream)


def aa_dedisperse(plan, host_ptr, nsamp, host_pitch, stream) -> int:
    h = ctypes.c_void_p()
    check(lib().aa_dedisperse(plan, host_ptr, int(nsamp), int(host_pitch), stream,
                              ctypes.byref(h)), "aa_dedisperse")
    return h.value


def aa_dd_result_view(res) -> tuple:
    p, n = ctypes.c_void_p(), ctypes.c_int64()
    check(lib().aa_dd_result_view(res, ctypes.byref(p), ctypes.byref(n)), "aa_dd_result_view")
    return p.value, n.value


def aa_dd_result_destroy(res) -> None:
    lib().aa_dd_result_destroy(res)


def aa_sps_search(plan, dd, max_width, threshold, capacity, stream) -> tuple:
    h = ctypes.c_void_p()
    st = check(lib().aa_sps_search(plan, dd, int(max_width), float(threshold), int(capacity),
                                   stream, ctypes.byref(h)), "aa_sps_search",
               ok=(AA_OK, AA_WARN_CAND_OVERFLOW))
    return h.value, st


def aa_candidates_view(c) -> tuple:
    p, stored, total = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().aa_candidates_view(c, ctypes.byref(p), ctypes.byref(stored), ctypes.byref(total)),
          "aa_candidates_view")
    return p.value, stored.value, total.value


def aa_candidates_destroy(c) -> None:
    lib().aa_candidates_destroy(c)


def aa_search_fused_ws_bytes(plan, nsamp, max_width, stripe_trials=0) -> tuple:
    b, off = ctypes.c_size_t(), ctypes.c_size_t()
    check(lib().aa_search_fused_ws_bytes(plan, int(nsamp), int(max_width), int(stripe_trials),
                                         ctypes.byref(b), ctypes.byref(off)),
          "aa_search_fused_ws_bytes")
    return b.value, off.value


def aa_search_fused_device(plan, d_in, nsamp, in_pitch, max_width, threshold, stripe_trials,
                           d_cands, capacity, d_count, d_snr_out, d_ws, ws_bytes, stream) -> int:
    return check(lib().aa_search_fused_device(plan, d_in, int(nsamp), int(in_pitch), int(max_width),
                                              float(threshold), int(stripe_trials), d_cands,
                                              int(capacity), d_count, d_snr_out, d_ws, int(ws_bytes),
                                              stream),
                 "aa_search_fused_device")


def aa_pipeline_create(plan, nsamp, max_width, threshold, capacity, depth) -> int:
    h = ctypes.c_void_p()
    check(lib().aa_pipeline_create(plan, int(nsamp), int(max_width), float(threshold),
                                   int(capacity), int(depth), ctypes.byref(h)),
          "aa_pipeline_create")
    return h.value


def aa_pipeline_submit(pipeline, host_ptr: int, host_pitch: int) -> int:
    t = ctypes.c_int64()
    check(lib().aa_pipeline_submit(pipeline, host_ptr, int(host_pitch), ctypes.byref(t)),
          "aa_pipeline_submit", ok=(AA_PENDING,))
    return t.value


def aa_pipeline_wait(pipeline, ticket: int) -> tuple:
    h = ctypes.c_void_p()
    st = check(lib().aa_pipeline_wait(pipeline, int(ticket), ctypes.byref(h)), "aa_pipeline_wait",
               ok=(AA_OK, AA_WARN_CAND_OVERFLOW))
    return h.value, st


def aa_pipeline_destroy(pipeline) -> None:
    lib().aa_pipeline_destroy(pipeline)


def aa_debug_inject(what: int, value: int = 0) -> None:
    check(lib().aa_debug_inject(int(what), int(value)), "aa_debug_inject")


def aa_fil_read_header(path: str) -> aa_fil_header:
    h = aa_fil_header()
    check(lib().aa_fil_read_header(str(path).encode(), ctypes.byref(h)), "aa_fil_read_header")
    return h


def aa_fil_read_block(path: str, h: aa_fil_header, t0: int, nsamp: int, host_ptr: int) -> None:
    check(lib().aa_fil_read_block(str(path).encode(), ctypes.byref(h), int(t0), int(nsamp),
                                  host_ptr), "aa_fil_read_block")


def aa_corner_turn_device(d_tm: int, nsamp: int, nchans: int, tm_stride: int, d_cm: int,
                          cm_pitch: int, stream: int = 0) -> None:
    check(lib().aa_corner_turn_device(d_tm, int(nsamp), int(nchans), int(tm_stride), d_cm,
                                      int(cm_pitch), stream), "aa_corner_turn_device")


def aa_plan_set_sps_ladder(plan, growth_x16: int) -> None:
    check(lib().aa_plan_set_sps_ladder(plan, int(growth_x16)), "aa_plan_set_sps_ladder")


def aa_plan_set_sps_decimated(plan, base_widths: int) -> None:
    check(lib().aa_plan_set_sps_decimated(plan, base_widths), "aa_plan_set_sps_decimated")


def aa_plan_effective_shifts(plan, r: int, ndm: int, nchans: int):
    import numpy as np
    out = np.empty((ndm, nchans), dtype=np.int32)
    check(lib().aa_plan_effective_shifts(plan, int(r), out.ctypes.data, out.size),
          "aa_plan_effective_shifts")
    return out


def aa_plan_set_fdmt(plan, r: int) -> None:
    check(lib().aa_plan_set_fdmt(plan, int(r)), "aa_plan_set_fdmt")


def aa_plan_set_subband(plan, r: int, band_channels: int, coarse_trials: int) -> None:
    check(lib().aa_plan_set_subband(plan, int(r), int(band_channels), int(coarse_trials)),
          "aa_plan_set_subband")


def aa_plan_set_sps_clip(plan, c16: int, max_iters: int) -> None:
    check(lib().aa_plan_set_sps_clip(plan, int(c16), int(max_iters)), "aa_plan_set_sps_clip")


def aa_postprocess_ws_bytes(plan, nsamp: int, max_width: int, capacity: int) -> int:
    out = ctypes.c_size_t(0)
    check(lib().aa_postprocess_ws_bytes(plan, int(nsamp), int(max_width), int(capacity),
                                        ctypes.byref(out)), "aa_postprocess_ws_bytes")
    return out.value


def aa_sps_order_device(plan, nsamp, max_width, d_sps_ws, d_cands, d_count, capacity, d_sorted,
                        d_tmp, tmp_bytes, stream=0) -> None:
    check(lib().aa_sps_order_device(plan, int(nsamp), int(max_width), d_sps_ws, d_cands, d_count,
                                    int(capacity), d_sorted, d_tmp, int(tmp_bytes), stream),
          "aa_sps_order_device")


def aa_candidates_peaks2d_device(plan, nsamp, max_width, d_sorted, d_count, capacity, dm_radius,
                                 t_radius, d_peaks, d_npeaks, d_tmp, tmp_bytes, stream=0) -> None:
    check(lib().aa_candidates_peaks2d_device(plan, int(nsamp), int(max_width), d_sorted, d_count,
                                             int(capacity), int(dm_radius), int(t_radius), d_peaks,
                                             d_npeaks, d_tmp, int(tmp_bytes), stream),
          "aa_candidates_peaks2d_device")


def aa_profile_enable(on: bool) -> None:
    check(lib().aa_profile_enable(1 if on else 0), "aa_profile_enable")


def aa_profile_read(kernel: int) -> tuple:
    n, ms = ctypes.c_int64(), ctypes.c_double()
    check(lib().aa_profile_read(int(kernel), ctypes.byref(n), ctypes.byref(ms)), "aa_profile_read")
    return n.value, ms.value


def aa_profile_kernel_name(kernel: int):
    r = lib().aa_profile_kernel_name(int(kernel))
    return None if r is None else r.decode()


def profile_snapshot() -> dict:
    """{kernel name: (launches, total ms)} for every library kernel."""
    out, k = {}, 0
    while True:
        name = aa_profile_kernel_name(k)
        if name is None:
            return out
        out[name] = aa_profile_read(k)
        k += 1


def aa_sps_search_device_noalloc(plan, nsamp, d_dd, max_width, threshold, d_cands, capacity,
                                 d_count, d_snr_out, stream) -> int:
    """Returns the status code (callers check it: AA_ERR_ARG means the
    search needs more scratch than the built-in area holds)."""
    return lib().aa_sps_search_device_noalloc(plan, int(nsamp), d_dd, int(max_width),
                                              float(threshold), d_cands, int(capacity), d_count,
                                              d_snr_out, stream)


def aa_dedisperse_f32_device(plan, d_x, nsamp, x_pitch, d_w, d_y, stream) -> None:
    check(lib().aa_dedisperse_f32_device(plan, d_x, int(nsamp), int(x_pitch), d_w, d_y, stream),
          "aa_dedisperse_f32_device")


def aa_dedisperse_f32_adjoint_device(plan, d_x, nsamp, x_pitch, d_w, d_gy, d_gx, d_gw, d_ws,
                                     ws_bytes, stream) -> None:
    check(lib().aa_dedisperse_f32_adjoint_device(plan, d_x, int(nsamp), int(x_pitch), d_w, d_gy,
                                                 d_gx, d_gw, d_ws, int(ws_bytes), stream),
          "aa_dedisperse_f32_adjoint_device")


def aa_dedisperse_f32_mse_device(plan, d_x, nsamp, x_pitch, d_w, d_tmpl, d_loss, d_gx, d_gw,
                                 d_ws, ws_bytes, stream) -> None:
    check(lib().aa_dedisperse_f32_mse_device(plan, d_x, int(nsamp), int(x_pitch), d_w, d_tmpl,
                                             d_loss, d_gx, d_gw, d_ws, int(ws_bytes), stream),
          "aa_dedisperse_f32_mse_device")


AA_DEDISP_DIRECT = 0
AA_DEDISP_GROUPED = 1
AA_DEDISP_SUBBAND = 2
AA_DEDISP_FDMT = 3


def aa_plan_set_strategy(plan, r: int, strategy: int) -> None:
    check(lib().aa_plan_set_strategy(plan, int(r), int(strategy)), "aa_plan_set_strategy")


def aa_plan_autotune(plan, nsamp_probe: int, cache_path=None) -> None:
    check(lib().aa_plan_autotune(plan, int(nsamp_probe),
                                 None if cache_path is None else str(cache_path).encode()),
          "aa_plan_autotune")


def aa_batch_create(plans, nsamps, max_width, threshold, capacity, wave_budget=0) -> int:
    n = len(plans)
    parr = (ctypes.c_void_p * n)(*plans)
    narr = (ctypes.c_int64 * n)(*[int(v) for v in nsamps])
    h = ctypes.c_void_p()
    check(lib().aa_batch_create(parr, narr, n, int(max_width), float(threshold), int(capacity),
                                int(wave_budget), ctypes.byref(h)), "aa_batch_create")
    return h.value


def aa_batch_destroy(batch) -> None:
    lib().aa_batch_destroy(batch)


def aa_batch_input(batch, beam: int) -> tuple:
    p, pitch = ctypes.c_void_p(), ctypes.c_int64()
    check(lib().aa_batch_input(batch, int(beam), ctypes.byref(p), ctypes.byref(pitch)),
          "aa_batch_input")
    return p.value, pitch.value


def aa_batch_dd_view(batch, beam: int) -> int:
    p = ctypes.c_void_p()
    check(lib().aa_batch_dd_view(batch, int(beam), ctypes.byref(p)), "aa_batch_dd_view")
    return p.value


def aa_batch_info(batch) -> tuple:
    nw, nb = ctypes.c_int32(), ctypes.c_int64()
    check(lib().aa_batch_info(batch, ctypes.byref(nw), ctypes.byref(nb)), "aa_batch_info")
    return nw.value, nb.value


def aa_batch_run(batch, stream) -> None:
    check(lib().aa_batch_run(batch, stream), "aa_batch_run")


def aa_batch_set_branches(batch, branches: int) -> None:
    check(lib().aa_batch_set_branches(batch, branches), "aa_batch_set_branches")


def aa_batch_candidates(batch, stream) -> tuple:
    h = ctypes.c_void_p()
    st = check(lib().aa_batch_candidates(batch, stream, ctypes.byref(h)), "aa_batch_candidates",
               ok=(AA_OK, AA_WARN_CAND_OVERFLOW))
    return h.value, st


def aa_server_create(plan, nbeams, chunk_nsamp, max_width, threshold, capacity, budget=0,
                     max_slots=8) -> int:
    h = ctypes.c_void_p()
    check(lib().aa_server_create(plan, int(nbeams), int(chunk_nsamp), int(max_width),
                                 float(threshold), int(capacity), int(budget), int(max_slots),
                                 ctypes.byref(h)), "aa_server_create")
    return h.value


def aa_server_destroy(server) -> None:
    lib().aa_server_destroy(server)


def aa_server_submit(server, beam, host_ptr, host_pitch, arrival) -> int:
    t = ctypes.c_int64()
    check(lib().aa_server_submit(server, int(beam), host_ptr, int(host_pitch), float(arrival),
                                 ctypes.byref(t)), "aa_server_submit", ok=(AA_PENDING,))
    return t.value


def aa_server_poll(server) -> tuple:
    n = ctypes.c_int32()
    st = check(lib().aa_server_poll(server, ctypes.byref(n)), "aa_server_poll",
               ok=(AA_OK, AA_PENDING))
    return st, n.value


def aa_server_drain(server) -> None:
    check(lib().aa_server_drain(server), "aa_server_drain")


def aa_server_result(server, ticket, want_candidates=True) -> tuple:
    info = aa_chunk_info()
    h = ctypes.c_void_p()
    st = lib().aa_server_result(server, int(ticket), ctypes.byref(info),
                                ctypes.byref(h) if want_candidates else None)
    if st not in (AA_OK, AA_PENDING, AA_WARN_CAND_OVERFLOW):
        raise AAError(st, "aa_server_result")
    return st, info, h.value


def aa_server_stats(server) -> aa_server_report:
    s = aa_server_report()
    check(lib().aa_server_stats(server, ctypes.byref(s)), "aa_server_stats")
    return s


def aa_server_clock() -> float:
    return lib().aa_server_clock()


def aa_sps_workspace_work(d_ws, stream) -> int:
    v = ctypes.c_int64()
    check(lib().aa_sps_workspace_work(d_ws, stream, ctypes.byref(v)), "aa_sps_workspace_work")
    return v.value
