"""Writes SIGPROC filterbank files for the tests, from the format's
definition: keyword strings as int32 length + bytes, int32 / float64 / string
values, HEADER_START ... HEADER_END, then time-major 8-bit samples."""
import struct

INT_KEYS = {"telescope_id", "machine_id", "data_type", "barycentric", "pulsarcentric", "nbits",
            "nsamples", "nchans", "nifs", "nbeams", "ibeam"}
DOUBLE_KEYS = {"fch1", "foff", "tstart", "tsamp", "src_raj", "src_dej", "az_start", "za_start",
               "refdm", "period"}
STRING_KEYS = {"source_name", "rawdatafile"}


def fil_string(s: str) -> bytes:
    b = s.encode()
    return struct.pack("<i", len(b)) + b


def header_bytes(fields: dict) -> bytes:
    out = fil_string("HEADER_START")
    for k, v in fields.items():
        out += fil_string(k)
        if k in INT_KEYS:
            out += struct.pack("<i", int(v))
        elif k in DOUBLE_KEYS:
            out += struct.pack("<d", float(v))
        elif k in STRING_KEYS:
            out += fil_string(str(v))
        elif k == "signed":
            out += struct.pack("<b", int(v))
        else:
            raise KeyError(k)
    return out + fil_string("HEADER_END")


def write_fil(path, fields: dict, data_tm) -> int:
    """data_tm: uint8 array [nsamp][nchans].  Returns the header length."""
    h = header_bytes(fields)
    with open(path, "wb") as f:
        f.write(h)
        f.write(data_tm.tobytes())
    return len(h)
