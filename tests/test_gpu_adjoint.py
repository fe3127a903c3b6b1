"""Differentiable form on the GPU (through the C ABI) against the FP64
oracle: forward parity, <A x, g> = <x, A^T g> in FP32, adjoint parity, the
MSE-loss gradients against FP64 central finite differences (256 channels,
4096 samples), the chunk-recomputed gradient against the materialised one,
the autograd bindings, and sampled rows at 1024 channels / 65536 samples."""
import numpy as np
import pytest
import torch

from paper_1912_07704_gb300 import synth
from paper_1912_07704_gb300.api import Plan
from paper_1912_07704_gb300.autograd import Dedisperse, DedispersionMSE

pytestmark = pytest.mark.gpu


def setup_case(oracle, w, pulse_dm):
    plan = Plan.from_workload(w)
    lay = plan.layout(w.nsamp)[0]
    d1 = lambda dm: oracle.shifts(w.nchans, w.fch1, w.foff, w.tsamp, dm, 1)
    pulse = [synth.Pulse(pulse_dm, w.nsamp // 4, 16, 1.0)]
    x = synth.float_filterbank(w, pulse, d1, device="cuda")
    wt = synth.channel_weights(w.nchans, w.data_seed + 100, device="cuda")
    xt = synth.float_filterbank(w, pulse, d1, device="cpu", noise=False).double().numpy()
    tmpl_rows = oracle.forward_f64(xt, np.ones(w.nchans), plan.shifts(0), lay.length)
    tmpl = torch.zeros(plan.query(w.nsamp).dd_elems, dtype=torch.float32, device="cuda")
    plan.range_views(tmpl, w.nsamp)[0].copy_(torch.from_numpy(tmpl_rows).float())
    return plan, lay, x, wt, tmpl, tmpl_rows


@pytest.fixture(scope="module")
def small(oracle):
    return setup_case(oracle, synth.ADJ_256, 96.0)


def test_forward_parity(oracle, small):
    plan, lay, x, w, tmpl, _ = small
    y = plan.f32_forward(x, w)
    torch.cuda.synchronize()
    ref = oracle.forward_f64(x.double().cpu().numpy(), w.double().cpu().numpy(), plan.shifts(0),
                             lay.length)
    got = plan.range_views(y, x.shape[1])[0].double().cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * max(scale, 1.0)


def test_dot_product_identity_fp32(small):
    plan, lay, x, w, tmpl, _ = small
    g = torch.zeros_like(tmpl)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    plan.range_views(g, x.shape[1])[0].copy_(
        torch.randn((lay.ndm, lay.length), generator=gen, device="cuda"))
    y = plan.f32_forward(x, w)
    gx, gw = plan.f32_adjoint(x, w, g)
    torch.cuda.synchronize()
    yv = plan.range_views(y, x.shape[1])[0].double()
    gv = plan.range_views(g, x.shape[1])[0].double()
    lhs = float((yv * gv).sum())
    rhs_x = float((x.double() * gx.double()).sum())
    rhs_w = float((w.double() * gw.double()).sum())
    assert abs(lhs - rhs_x) <= 1e-5 * abs(lhs)
    assert abs(lhs - rhs_w) <= 1e-5 * abs(lhs)


def test_adjoint_parity(oracle, small):
    plan, lay, x, w, tmpl, _ = small
    rng = np.random.default_rng(6)
    gy = rng.standard_normal((lay.ndm, lay.length))
    g = torch.zeros_like(tmpl)
    plan.range_views(g, x.shape[1])[0].copy_(torch.from_numpy(gy).float())
    gx, gw = plan.f32_adjoint(x, w, g)
    torch.cuda.synchronize()
    ogx, ogw = oracle.adjoint_f64(x.double().cpu().numpy(), w.double().cpu().numpy(),
                                  plan.shifts(0), gy)
    assert np.abs(gx.double().cpu().numpy() - ogx).max() <= 1e-5 * np.abs(ogx).max()
    assert np.abs(gw.double().cpu().numpy() - ogw).max() <= 1e-5 * np.abs(ogw).max()


def test_mse_gradients_vs_fp64_finite_differences(oracle, small):
    plan, lay, x, w, tmpl, tmpl_rows = small
    loss, gx, gw = plan.f32_mse(x, w, tmpl, grad=True)
    torch.cuda.synchronize()
    xh, wh = x.double().cpu().numpy(), w.double().cpu().numpy()
    sh = plan.shifts(0)
    L0 = oracle.mse_f64(xh, wh, sh, lay.length, tmpl_rows)
    assert abs(float(loss) - L0) <= 1e-5 * abs(L0)
    h = 1e-2  # the loss is quadratic in x and in w: central differences are exact
    for c in (0, 100, 255):
        wp, wm = wh.copy(), wh.copy()
        wp[c] += h
        wm[c] -= h
        fd = (oracle.mse_f64(xh, wp, sh, lay.length, tmpl_rows)
              - oracle.mse_f64(xh, wm, sh, lay.length, tmpl_rows)) / (2 * h)
        assert abs(float(gw[c]) - fd) <= 1e-4 * max(abs(fd), 1e-6), (c, float(gw[c]), fd)
    gxh = gx.double().cpu().numpy()
    for (c, t) in ((3, 1500), (128, 2500), (255, 3000)):
        xp, xm = xh.copy(), xh.copy()
        xp[c, t] += h
        xm[c, t] -= h
        fd = (oracle.mse_f64(xp, wh, sh, lay.length, tmpl_rows)
              - oracle.mse_f64(xm, wh, sh, lay.length, tmpl_rows)) / (2 * h)
        assert abs(gxh[c, t] - fd) <= 1e-4 * max(abs(fd), 1e-8), (c, t, gxh[c, t], fd)


def test_chunked_recomputation_equals_materialised_adjoint(small):
    plan, lay, x, w, tmpl, _ = small
    loss, gx, gw = plan.f32_mse(x, w, tmpl, grad=True)
    y = plan.f32_forward(x, w)
    n = lay.ndm * lay.length
    gy = torch.zeros_like(y)
    yv, tv = plan.range_views(y, x.shape[1])[0], plan.range_views(tmpl, x.shape[1])[0]
    plan.range_views(gy, x.shape[1])[0].copy_(2.0 * (yv - tv) / n)
    gx2, gw2 = plan.f32_adjoint(x, w, gy)
    torch.cuda.synchronize()
    assert torch.allclose(gx, gx2, rtol=1e-4, atol=1e-9 * float(gx2.abs().max()))
    assert torch.allclose(gw, gw2, rtol=1e-4, atol=1e-6 * float(gw2.abs().max()))


def test_autograd_functions(small):
    plan, lay, x, w, tmpl, _ = small
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    y = Dedisperse.apply(xr, wr, plan)
    yv = plan.range_views(y, x.shape[1])[0]
    tv = plan.range_views(tmpl, x.shape[1])[0]
    loss_a = ((yv - tv) ** 2).mean()
    loss_a.backward()
    xb = x.clone().requires_grad_(True)
    wb = w.clone().requires_grad_(True)
    loss_b = DedispersionMSE.apply(xb, wb, tmpl, plan)
    loss_b.backward()
    torch.cuda.synchronize()
    assert abs(float(loss_a.detach()) - float(loss_b.detach())) <= 1e-5 * abs(float(loss_b.detach()))
    assert torch.allclose(xr.grad, xb.grad, rtol=1e-3, atol=1e-6 * float(xb.grad.abs().max()))
    assert torch.allclose(wr.grad, wb.grad, rtol=1e-3, atol=1e-6 * float(wb.grad.abs().max()))


def test_full_size_sampled_rows(oracle):
    plan, lay, x, w, tmpl, tmpl_rows = setup_case(oracle, synth.ADJ_1024, 400.0)
    y = plan.f32_forward(x, w)
    loss, gx, gw = plan.f32_mse(x, w, tmpl, grad=True)
    torch.cuda.synchronize()
    rows = [0, 511, 800, 1023]
    xh, wh = x.double().cpu().numpy(), w.double().cpu().numpy()
    ref = oracle.forward_f64(xh, wh, plan.shifts(0)[rows], lay.length)
    got = plan.range_views(y, x.shape[1])[0][rows].double().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # the gradient wrt the weights: <gw, w> = 2/N <y - T, y> (Euler, y linear in w)
    yv = plan.range_views(y, x.shape[1])[0].double()
    tv = plan.range_views(tmpl, x.shape[1])[0].double()
    n = lay.ndm * lay.length
    euler = float((2.0 / n) * ((yv - tv) * yv).sum())
    assert abs(float((gw.double() * w.double()).sum()) - euler) <= 1e-4 * abs(euler)
    assert abs(float(loss) - float(((yv - tv) ** 2).mean())) <= 1e-5 * float(loss)
