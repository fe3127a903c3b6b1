"""File input on the GPU: the corner turn (time-major block -> channel-major
rows) against numpy's transpose, and a SIGPROC file of the 256-channel
workload read, corner-turned and dedispersed equal to the channel-major
original dedispersed directly."""
import numpy as np
import pytest
import torch

from filterbank_writer import write_fil
from paper_1912_07704_gb300 import abi, synth
from paper_1912_07704_gb300.api import Plan, candidates_from_device, corner_turn, read_filterbank

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nsamp,nchans,stride_pad,pitch_pad",
                         [(1000, 203, 0, 0), (4096, 1024, 0, 0), (777, 64, 13, 37),
                          (64, 64, 0, 0), (1, 1, 0, 15), (65, 4097, 3, 1)])
def test_corner_turn_equals_transpose(nsamp, nchans, stride_pad, pitch_pad):
    rng = np.random.default_rng(nsamp + nchans)
    full = rng.integers(0, 256, size=(nsamp, nchans + stride_pad), dtype=np.uint8)
    tm = torch.from_numpy(full).cuda()[:, :nchans]  # row stride nchans + stride_pad
    pitch = nsamp + pitch_pad
    out = torch.full((nchans, pitch), 0xAB, dtype=torch.uint8, device="cuda")
    abi.aa_corner_turn_device(tm.data_ptr(), nsamp, nchans, tm.stride(0), out.data_ptr(), pitch,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got[:, :nsamp], full[:, :nchans].T)
    assert np.all(got[:, nsamp:] == 0xAB)  # the pitch padding is not written


def test_corner_turn_argument_checks():
    x = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        abi.aa_corner_turn_device(x.data_ptr(), 4, 4, 3, x.data_ptr(), 4, s)  # stride < nchans
    with pytest.raises(abi.AAError, match="AA_ERR_ARG"):
        abi.aa_corner_turn_device(x.data_ptr(), 4, 4, 4, x.data_ptr(), 3, s)  # pitch < nsamp


def test_file_to_dedispersion(tmp_path, oracle):
    w = synth.PLAIN_256
    x = synth.make_filterbank(
        w, synth.pulses_single(),
        lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)).numpy()
    path = tmp_path / "plain256.fil"
    write_fil(path, {"nchans": w.nchans, "nbits": 8, "fch1": w.fch1, "foff": w.foff,
                     "tsamp": w.tsamp, "source_name": "synthetic"}, np.ascontiguousarray(x.T))
    h, tm_host = read_filterbank(str(path))
    assert h.nsamples == w.nsamp
    plan = Plan.from_filterbank(h, w.ranges)
    cm = corner_turn(tm_host.cuda(non_blocking=True))
    from_file = plan.dedisperse_device(cm, h.nsamples)
    d, nsamp = plan.device_input(x)
    direct = plan.dedisperse_device(d, nsamp)
    torch.cuda.synchronize()
    for a, b in zip(plan.range_views(from_file, nsamp), plan.range_views(direct, nsamp)):
        assert torch.equal(a, b)
    c1, n1, _ = plan.sps_search_device(from_file, nsamp, w.max_width, w.threshold, 1 << 16)
    c2, n2, _ = plan.sps_search_device(direct, nsamp, w.max_width, w.threshold, 1 << 16)
    torch.cuda.synchronize()
    a1 = candidates_from_device(c1, n1, 1 << 16)
    assert len(a1) > 0 and np.array_equal(a1, candidates_from_device(c2, n2, 1 << 16))
