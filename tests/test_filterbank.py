"""SIGPROC filterbank reader (host part of the file input): header fields,
block reads and error handling, against files written from the format's
definition by tests/filterbank_writer.py."""
import struct

import numpy as np
import pytest

from filterbank_writer import fil_string, header_bytes, write_fil
from paper_1912_07704_gb300 import abi
from paper_1912_07704_gb300.api import Plan, read_filterbank

FIELDS = {"telescope_id": 7, "machine_id": 11, "source_name": "SYNTH J0000+00", "data_type": 1,
          "fch1": 1508.0, "foff": -0.0732421875, "nchans": 203, "nbits": 8, "tstart": 60000.5,
          "tsamp": 64e-6, "nifs": 1, "src_raj": 123456.7, "signed": 0}


def test_header_fields_and_sizes(tmp_path):
    rng = np.random.default_rng(1)
    data = rng.integers(0, 256, size=(1001, 203), dtype=np.uint8)
    p = tmp_path / "a.fil"
    hlen = write_fil(p, FIELDS, data)
    h = abi.aa_fil_read_header(str(p))
    assert (h.nchans, h.nbits, h.nifs, h.data_type, h.telescope_id, h.machine_id) == (203, 8, 1, 1, 7, 11)
    assert h.fch1_mhz == 1508.0 and h.foff_mhz == -0.0732421875 and h.tsamp_s == 64e-6
    assert h.tstart_mjd == 60000.5 and h.source_name == b"SYNTH J0000+00"
    assert h.header_bytes == hlen and h.nsamples == 1001


def test_block_reads(tmp_path):
    rng = np.random.default_rng(2)
    data = rng.integers(0, 256, size=(777, 64), dtype=np.uint8)
    p = tmp_path / "b.fil"
    write_fil(p, dict(FIELDS, nchans=64), data)
    h, whole = read_filterbank(str(p))
    assert np.array_equal(whole.numpy(), data)
    for t0, n in ((0, 1), (5, 100), (700, 77), (777, 0)):
        _, part = read_filterbank(str(p), t0, n)
        assert np.array_equal(part.numpy(), data[t0:t0 + n])
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        read_filterbank(str(p), 700, 78)


def test_hand_built_header_bytes(tmp_path):
    """A minimal header spelled out byte by byte."""
    raw = (struct.pack("<i", 12) + b"HEADER_START" + struct.pack("<i", 6) + b"nchans" +
           struct.pack("<i", 4) + struct.pack("<i", 5) + b"nbits" + struct.pack("<i", 8) +
           struct.pack("<i", 4) + b"fch1" + struct.pack("<d", 1400.0) +
           struct.pack("<i", 4) + b"foff" + struct.pack("<d", -1.0) +
           struct.pack("<i", 5) + b"tsamp" + struct.pack("<d", 1e-3) +
           struct.pack("<i", 10) + b"HEADER_END")
    p = tmp_path / "c.fil"
    p.write_bytes(raw + bytes(range(4 * 3)))  # 3 samples of 4 channels
    h = abi.aa_fil_read_header(str(p))
    assert (h.nchans, h.nbits, h.fch1_mhz, h.foff_mhz, h.tsamp_s) == (4, 8, 1400.0, -1.0, 1e-3)
    assert h.header_bytes == len(raw) and h.nsamples == 3
    assert h.telescope_id == -1 and h.source_name == b""
    _, d = read_filterbank(str(p))
    assert d.numpy().tolist() == [[0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11]]


@pytest.mark.parametrize("case", ["no_start", "unknown", "nbits4", "nifs2", "truncated", "missing"])
def test_malformed_headers(tmp_path, case):
    p = tmp_path / "bad.fil"
    fields = dict(FIELDS)
    if case == "no_start":
        raw = header_bytes(fields)[len(fil_string("HEADER_START")):]
    elif case == "unknown":
        raw = fil_string("HEADER_START") + fil_string("frobnicate") + struct.pack("<i", 1) + fil_string("HEADER_END")
    elif case == "nbits4":
        raw = header_bytes(dict(fields, nbits=4))
    elif case == "nifs2":
        raw = header_bytes(dict(fields, nifs=2))
    elif case == "truncated":
        raw = header_bytes(fields)[:-20]
    else:  # missing tsamp
        fields.pop("tsamp")
        raw = header_bytes(fields)
    p.write_bytes(raw)
    with pytest.raises(abi.AAError, match="AA_ERR_CONFIG"):
        abi.aa_fil_read_header(str(p))


def test_missing_file_and_plan_from_header(tmp_path):
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        abi.aa_fil_read_header(str(tmp_path / "nope.fil"))
    p = tmp_path / "d.fil"
    write_fil(p, dict(FIELDS, nchans=256, fch1=1500.0, foff=-1.171875),
              np.zeros((10, 256), np.uint8))
    h = abi.aa_fil_read_header(str(p))
    plan = Plan.from_filterbank(h, [(0.0, 1.0, 256, 1)])
    assert plan.nchans == 256 and plan.fch1 == 1500.0 and plan.foff == -1.171875
