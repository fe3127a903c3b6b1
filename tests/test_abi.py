"""C ABI checks that need no GPU: the library loads, exports every entry
point of include/aa_dedisp.h, and its host-side plan logic (validation, FP64
delay tables, per-range lengths, memory requests) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

from paper_1912_07704_gb300 import abi
from paper_1912_07704_gb300.api import Plan
from paper_1912_07704_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "aa_dedisp.h")


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(aa_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 18
    L = abi.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(abi.exported_names()) == names


def test_status_strings():
    for code in (0, 1, 2, -1, -2, -3, -4, -5, -6):
        assert abi.status_str(code).startswith("AA_")
    assert abi.status_str(99) == "AA_UNKNOWN_STATUS"


def test_destroy_null_is_noop():
    abi.aa_plan_destroy(None)
    abi.aa_dd_result_destroy(None)
    abi.aa_candidates_destroy(None)


BAD = [
    dict(nchans=0), dict(tsamp=0.0), dict(tsamp=-1e-3), dict(foff=0.0), dict(fch1=-5.0),
    dict(fch1=100.0, foff=-1.0, nchans=200),            # lowest channel <= 0 MHz
    dict(ranges=[]), dict(ranges=[(0.0, 1.0, 0, 1)]), dict(ranges=[(0.0, 1.0, 4, 0)]),
    dict(ranges=[(0.0, 1.0, 4, 17)]), dict(ranges=[(-1.0, 1.0, 4, 1)]),
    dict(ranges=[(0.0, -1.0, 4, 1)]), dict(nchans=8192, ranges=[(0.0, 1.0, 4, 16)]),
]


@pytest.mark.parametrize("bad", BAD, ids=[str(b) for b in BAD])
def test_invalid_plans_are_rejected(bad):
    kw = dict(nchans=64, fch1=1400.0, foff=-1.0, tsamp=64e-6, ranges=[(0.0, 1.0, 8, 1)])
    kw.update(bad)
    with pytest.raises(abi.AAError) as e:
        Plan(kw["nchans"], kw["fch1"], kw["foff"], kw["tsamp"], kw["ranges"])
    assert e.value.status in (abi.AA_ERR_CONFIG, abi.AA_ERR_ARG)
    assert abi.aa_last_error() != ""


@pytest.mark.parametrize("w", [synth.PLAIN_256, synth.SKA_4096], ids=lambda w: w.name)
def test_plan_matches_oracle(oracle, w):
    p = Plan.from_workload(w)
    opl = oracle.plan(w.nchans, w.fch1, w.foff, w.tsamp, w.ranges, w.nsamp)
    lay = p.layout(w.nsamp)
    for r, (g, o) in enumerate(zip(lay, opl)):
        assert (g.ndm, g.dec, g.maxshift, g.length, g.dm_offset) == \
            (o.ndm, o.dec, o.maxshift, o.length, o.dm_offset)
        assert np.array_equal(p.shifts(r), o.shifts)
        assert g.pitch % 64 == 0 and g.pitch >= max(g.length, 1)
    info = p.query(w.nsamp, w.max_width)
    assert info.dm_trial_samples == sum(o.ndm * o.length for o in opl)
    assert info.ready == 0 and info.device == -1
    assert info.in_pitch_min % 16 == 0 and info.in_pitch_min >= w.nsamp
    assert info.dd_elems == sum(g.ndm * g.pitch for g in lay)
    p.close()


def test_ragged_and_empty_lengths():
    p = Plan(100, 1400.0, -2.0, 64e-6, [(0.0, 3.0, 37, 1), (100.0, 5.0, 9, 3)])
    for nsamp in (0, 1, 50, 12345):
        lay = p.layout(nsamp)
        for g in lay:
            assert g.length == max(0, nsamp // g.dec - g.maxshift)
    assert p.query(0).dm_trial_samples == 0


def test_query_does_not_touch_device():
    p = Plan.from_workload(synth.SKA_4096)
    info = p.query(1 << 20, 8192)
    # bytes requested before allocation: output, scratch and the delay tables
    assert info.dd_elems * 4 > 9e9
    assert info.table_bytes >= 4250 * 4096 * 4
    assert info.sps_ws_bytes >= 4250 * 8192 * 8
    p.close()


def test_postprocess_scratch_and_argument_checks():
    p = Plan(100, 1400.0, -2.0, 64e-6, [(0.0, 3.0, 37, 1), (100.0, 5.0, 9, 3)])
    small = abi.aa_postprocess_ws_bytes(p.handle, 5000, 16, 1000)
    large = abi.aa_postprocess_ws_bytes(p.handle, 5000, 16, 1 << 20)
    assert 256 < small < large
    # 16 bytes per candidate (keep flag and work-queue entry) plus the scan's share
    assert 16 * (1 << 20) <= large - small + 16 * 1000 < 17 * (1 << 20)
    assert abi.aa_postprocess_ws_bytes(p.handle, 0, 16, 0) >= 256
    for args in [(5000, 0, 10), (-1, 16, 10), (5000, 16, -1)]:
        with pytest.raises(abi.AAError):
            abi.aa_postprocess_ws_bytes(p.handle, *args)
    with pytest.raises(abi.AAError):  # NULL device pointers are rejected before any launch
        abi.aa_sps_order_device(p.handle, 5000, 16, 0, 0, 0, 10, 0, 0, 1 << 20)
    with pytest.raises(abi.AAError):  # negative radius
        abi.aa_candidates_peaks2d_device(p.handle, 5000, 16, 1 << 12, 1 << 12, 10, -1, 4,
                                         1 << 12, 1 << 12, 1 << 12, 1 << 20)
