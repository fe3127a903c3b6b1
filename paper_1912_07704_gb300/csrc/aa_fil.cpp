// SIGPROC filterbank input (arXiv:1912.07704 Sec. 4: the front-end can direct
// the library to a file on disk).  Host code: header parsing and block reads
// into caller-owned memory; the device corner turn is in aa_corner.cu.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aa_internal.h"

using namespace aa;

namespace {

enum class Kind { Int, Double, String, Byte, Marker };

// Keywords of the header and the type of their value.
Kind keyword_kind(const std::string& k, bool& known) {
    static const char* ints[] = {"telescope_id", "machine_id", "data_type", "barycentric",
                                 "pulsarcentric", "nbits", "nsamples", "nchans", "nifs",
                                 "nbeams", "ibeam", "npuls", "nbins"};
    static const char* doubles[] = {"fch1", "foff", "tstart", "tsamp", "src_raj", "src_dej",
                                    "az_start", "za_start", "refdm", "period"};
    static const char* strings[] = {"source_name", "rawdatafile"};
    known = true;
    for (const char* s : ints)
        if (k == s) return Kind::Int;
    for (const char* s : doubles)
        if (k == s) return Kind::Double;
    for (const char* s : strings)
        if (k == s) return Kind::String;
    if (k == "signed") return Kind::Byte;
    if (k == "HEADER_START" || k == "HEADER_END") return Kind::Marker;
    known = false;
    return Kind::Marker;
}

struct Cursor {
    const std::vector<unsigned char>& b;
    size_t pos = 0;
    bool take(void* dst, size_t n) {
        if (pos + n > b.size()) return false;
        std::memcpy(dst, b.data() + pos, n);
        pos += n;
        return true;
    }
    // int32 length + bytes (lengths outside 1..255 are not a header string)
    bool string(std::string& out) {
        int32_t n = 0;
        if (!take(&n, 4) || n < 1 || n > 255 || pos + (size_t)n > b.size()) return false;
        out.assign(reinterpret_cast<const char*>(b.data() + pos), (size_t)n);
        pos += (size_t)n;
        return true;
    }
};

int64_t file_size(FILE* f) {
    if (fseeko(f, 0, SEEK_END) != 0) return -1;
    const int64_t n = (int64_t)ftello(f);
    fseeko(f, 0, SEEK_SET);
    return n;
}

}  // namespace

extern "C" aa_status aa_fil_read_header(const char* path, aa_fil_header* out) {
    clear_error();
    if (!path || !out) { set_error("path/out is NULL"); return AA_ERR_ARG; }
    FILE* f = std::fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return AA_ERR_ARG; }
    const int64_t size = file_size(f);
    std::vector<unsigned char> buf((size_t)std::min<int64_t>(std::max<int64_t>(size, 0), 1 << 16));
    const size_t got = std::fread(buf.data(), 1, buf.size(), f);
    std::fclose(f);
    buf.resize(got);

    aa_fil_header h{};
    h.telescope_id = -1;
    h.machine_id = -1;
    bool have_nchans = false, have_nbits = false, have_fch1 = false, have_foff = false,
         have_tsamp = false, ended = false;
    h.nifs = 1;
    Cursor c{buf};
    std::string key;
    if (!c.string(key) || key != "HEADER_START") {
        set_error("%s: no HEADER_START", path);
        return AA_ERR_CONFIG;
    }
    while (!ended) {
        if (!c.string(key)) { set_error("%s: header ends without HEADER_END", path); return AA_ERR_CONFIG; }
        bool known = false;
        const Kind kind = keyword_kind(key, known);
        if (!known) { set_error("%s: unknown header keyword '%s'", path, key.c_str()); return AA_ERR_CONFIG; }
        int32_t iv = 0;
        double dv = 0;
        std::string sv;
        unsigned char bv = 0;
        bool ok = true;
        switch (kind) {
            case Kind::Int: ok = c.take(&iv, 4); break;
            case Kind::Double: ok = c.take(&dv, 8); break;
            case Kind::String: ok = c.string(sv); break;
            case Kind::Byte: ok = c.take(&bv, 1); break;
            case Kind::Marker:
                if (key == "HEADER_END") ended = true;
                else { set_error("%s: nested HEADER_START", path); return AA_ERR_CONFIG; }
                break;
        }
        if (!ok) { set_error("%s: truncated value of '%s'", path, key.c_str()); return AA_ERR_CONFIG; }
        if (key == "nchans") { h.nchans = iv; have_nchans = true; }
        else if (key == "nbits") { h.nbits = iv; have_nbits = true; }
        else if (key == "nifs") h.nifs = iv;
        else if (key == "data_type") h.data_type = iv;
        else if (key == "telescope_id") h.telescope_id = iv;
        else if (key == "machine_id") h.machine_id = iv;
        else if (key == "fch1") { h.fch1_mhz = dv; have_fch1 = true; }
        else if (key == "foff") { h.foff_mhz = dv; have_foff = true; }
        else if (key == "tsamp") { h.tsamp_s = dv; have_tsamp = true; }
        else if (key == "tstart") h.tstart_mjd = dv;
        else if (key == "source_name") std::snprintf(h.source_name, sizeof h.source_name, "%s", sv.c_str());
    }
    if (!have_nchans || !have_nbits || !have_fch1 || !have_foff || !have_tsamp) {
        set_error("%s: header lacks nchans, nbits, fch1, foff or tsamp", path);
        return AA_ERR_CONFIG;
    }
    if (h.nbits != 8 || h.nifs != 1 || h.nchans < 1) {
        set_error("%s: only 8-bit, single-IF data are read (nbits %d, nifs %d, nchans %d)", path,
                  h.nbits, h.nifs, h.nchans);
        return AA_ERR_CONFIG;
    }
    h.header_bytes = (int64_t)c.pos;
    h.nsamples = size > h.header_bytes ? (size - h.header_bytes) / h.nchans : 0;
    *out = h;
    return AA_OK;
}

extern "C" aa_status aa_fil_read_block(const char* path, const aa_fil_header* h, int64_t t0,
                                       int64_t nsamp, uint8_t* host_tm) {
    clear_error();
    if (!path || !h) { set_error("path/header is NULL"); return AA_ERR_ARG; }
    if (h->nchans < 1 || t0 < 0 || nsamp < 0 || t0 + nsamp > h->nsamples) {
        set_error("samples [%lld, %lld) outside the file's %lld", (long long)t0,
                  (long long)(t0 + nsamp), (long long)h->nsamples);
        return AA_ERR_ARG;
    }
    if (nsamp == 0) return AA_OK;  // the buffer may be NULL then
    if (!host_tm) { set_error("buffer is NULL"); return AA_ERR_ARG; }
    FILE* f = std::fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return AA_ERR_ARG; }
    const int64_t off = h->header_bytes + t0 * (int64_t)h->nchans;
    const size_t want = (size_t)(nsamp * (int64_t)h->nchans);
    size_t got = 0;
    if (fseeko(f, (off_t)off, SEEK_SET) == 0) got = std::fread(host_tm, 1, want, f);
    std::fclose(f);
    if (got != want) {
        set_error("%s: read %zu of %zu bytes at offset %lld", path, got, want, (long long)off);
        return AA_ERR_CONFIG;
    }
    return AA_OK;
}
