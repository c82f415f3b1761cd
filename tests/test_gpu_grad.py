"""The differentiable form on the GPU against the FP64 oracle: soft-min loss,
adjoint of f (template and frames), FP64 central finite differences, and the
Adam template refinement (parity unpinned beyond its first gradient).

Tolerances: the soft-min is 1-Lipschitz in the cost (sup norm), so the
loss inherits the cost surface's bound: within 1e-4 relative with the
denominator floored at 1e-2 * max f of the frame (absolute 1e-6 * max f);
the
gradient must be within 1e-3 relative of FP64 central differences (the
target), pointwise where |g| >= 1e-2 * max|g| and absolutely (1e-5 * max|g|)
below that, and within 1e-3 normwise of the oracle's analytic gradient.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import Plan, build, synth
from paper_1506_06039_gb300.binding import TEMPLATE_F32, XCORR_DIRECT_BF16X3, XCORR_FFT_FP32
from paper_1506_06039_gb300.autograd import MocoSoftMin, refine_template, softmin_plan

pytestmark = pytest.mark.gpu

TAU = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def stack(m, n, T, w, seed, shift=None):
    st = synth.make_stack_np(m, n, T, max(6, m * n // 700), shift if shift is not None else min(w - 2, 8),
                             seed=seed, template="clean")
    rng = np.random.default_rng(seed)
    tmpl = st.frames.astype(np.float64).mean(0) + rng.normal(0, 50, (m, n))
    return st.frames, tmpl.astype(np.float32)


def gpu_loss_grad(frames, tmpl, w, grad_frames=False, xcorr=None, group_frames=0):
    fr = torch.from_numpy(frames).cuda()
    tb = torch.from_numpy(tmpl).cuda()
    if xcorr is None:
        plan = softmin_plan(fr, tb, w, group_frames=group_frames)
    else:
        m, n = tmpl.shape
        plan = Plan(dict(m=m, n=n, w=w, levels=0, template_dtype=TEMPLATE_F32, xcorr=xcorr,
                         group_frames=group_frames), tb)
    try:
        cost = plan.cost_surface(fr)
        loss, weights = plan.softmin(cost, TAU)
        out = plan.cost_backward(fr, weights, grad_frames=grad_frames)
        torch.cuda.synchronize()
    finally:
        plan.close()
    if grad_frames:
        gt, gf = out
        return cost.cpu().numpy(), loss.cpu().numpy(), gt.cpu().numpy(), gf.cpu().numpy()
    return cost.cpu().numpy(), loss.cpu().numpy(), out.cpu().numpy(), None


def check_loss(loss, lf, frames, tmpl, w):
    fmax = np.array([oracle.cost_f64(fr.astype(np.float64), tmpl.astype(np.float64), w).max() for fr in frames])
    err = np.abs(loss - lf) / np.maximum(np.abs(lf), 1e-2 * fmax)
    assert err.max() <= 1e-4, err


def oracle_tau(frames, tmpl, w):
    return oracle.softmin_tau(frames.astype(np.float64), tmpl.astype(np.float64), w, TAU)


def test_softmin_loss_and_gradients_match_oracle():
    frames, tmpl = stack(64, 72, 6, 8, seed=21)
    cost, loss, gt, gf = gpu_loss_grad(frames, tmpl, 8, grad_frames=True)
    tau = oracle_tau(frames, tmpl, 8)
    L, lf, gb, ga = oracle.softmin_loss(frames.astype(np.float64), tmpl.astype(np.float64), 8, tau,
                                        grad_template=True, grad_frames=True)
    check_loss(loss, lf, frames, tmpl, 8)
    assert np.abs(gt - gb).max() <= 1e-3 * np.abs(gb).max()
    assert np.abs(gf - ga).max() <= 1e-3 * np.abs(ga).max()


@pytest.mark.parametrize("route", ["fft", "direct"])
def test_template_adjoint_routes_ragged_groups(route):
    # The correlation part of dL/db through the FFTs (FFT form) and through
    # the tiled direct contraction (direct form), on a ragged frame size that
    # spans several column blocks and FFT tiles, with frame groups of 4 (three
    # groups, the last one short).
    m, n, w, T = 90, 88, 7, 10
    frames, tmpl = stack(m, n, T, w, seed=33)
    xc = XCORR_FFT_FP32 if route == "fft" else XCORR_DIRECT_BF16X3
    _, loss, gt, _ = gpu_loss_grad(frames, tmpl, w, xcorr=xc, group_frames=4)
    tau = oracle_tau(frames, tmpl, w)
    _, lf, gb, _ = oracle.softmin_loss(frames.astype(np.float64), tmpl.astype(np.float64), w, tau,
                                       grad_template=True)
    check_loss(loss, lf, frames, tmpl, w)
    assert np.abs(gt - gb).max() <= 1e-3 * np.abs(gb).max()


@pytest.mark.parametrize("route", ["fft", "direct"])
def test_fused_softmin_grad_equals_separate_calls(route):
    # moco_softmin_grad (one pass: the row spectra serve search and adjoint on
    # FFT-form plans; the three calls in turn otherwise) against
    # moco_cost_surface + moco_softmin + moco_cost_backward, over three frame
    # groups with a short last one.
    m, n, w, T = 64, 72, 6, 11
    frames, tmpl = stack(m, n, T, w, seed=71)
    fr = torch.from_numpy(frames).cuda()
    xc = XCORR_FFT_FP32 if route == "fft" else XCORR_DIRECT_BF16X3
    plan = Plan(dict(m=m, n=n, w=w, levels=0, template_dtype=TEMPLATE_F32, xcorr=xc, group_frames=4),
                torch.from_numpy(tmpl).cuda())
    try:
        loss, grad, cost, weights = plan.softmin_grad(fr, TAU, grad_scale=0.5)
        c2 = plan.cost_surface(fr)
        l2, w2 = plan.softmin(c2, TAU)
        g2 = plan.cost_backward(fr, w2, grad_scale=0.5)
        torch.cuda.synchronize()
    finally:
        plan.close()
    assert torch.equal(cost, c2) and torch.equal(loss, l2) and torch.equal(weights, w2)
    g, g2 = grad.cpu().numpy(), g2.cpu().numpy()
    assert np.abs(g - g2).max() <= 1e-5 * np.abs(g2).max()  # FP32 atomics: order of the sums only
    tau = oracle_tau(frames, tmpl, w)
    _, lf, gb, _ = oracle.softmin_loss(frames.astype(np.float64), tmpl.astype(np.float64), w, tau, grad_template=True)
    check_loss(loss.cpu().numpy(), lf, frames, tmpl, w)
    assert np.abs(g - 0.5 * gb).max() <= 1e-3 * np.abs(0.5 * gb).max()


def test_gradient_central_differences_64_pixels():
    # 64 seeded pixels, FP64 central differences of the oracle loss (tau held
    # at the oracle's median rule), step 1e-2 (the loss is smooth in b).
    frames, tmpl = stack(48, 48, 4, 6, seed=5)
    _, _, gt, _ = gpu_loss_grad(frames, tmpl, 6)
    fr64, tb64 = frames.astype(np.float64), tmpl.astype(np.float64)
    tau = oracle_tau(frames, tmpl, 6)
    rng = np.random.default_rng(0)
    pix = rng.choice(48 * 48, 64, replace=False)
    eps = 1e-2
    gmax = np.abs(gt).max()
    for p in pix:
        i, j = divmod(int(p), 48)
        bp, bm = tb64.copy(), tb64.copy()
        bp[i, j] += eps
        bm[i, j] -= eps
        fd = (oracle.softmin_loss(fr64, bp, 6, tau)[0] - oracle.softmin_loss(fr64, bm, 6, tau)[0]) / (2 * eps)
        assert abs(gt[i, j] - fd) <= 1e-3 * max(abs(fd), 1e-2 * gmax), (i, j, gt[i, j], fd)


def test_refine256_gradient_full_size():
    # The refinement workload's frame size and window (256x256, w = 16) on two
    # frames: analytic FP64 gradient and central differences on 64 pixels.
    wl = synth.WORKLOADS["refine256"]
    frames, tmpl = stack(wl.m, wl.n, 2, wl.w, seed=wl.seed, shift=wl.shift_max)
    _, loss, gt, _ = gpu_loss_grad(frames, tmpl, wl.w)
    fr64, tb64 = frames.astype(np.float64), tmpl.astype(np.float64)
    tau = oracle_tau(frames, tmpl, wl.w)
    L, lf, gb, _ = oracle.softmin_loss(fr64, tb64, wl.w, tau, grad_template=True)
    check_loss(loss, lf, frames, tmpl, wl.w)
    assert np.abs(gt - gb).max() <= 1e-3 * np.abs(gb).max()
    rng = np.random.default_rng(1)
    gmax = np.abs(gb).max()
    for p in rng.choice(wl.m * wl.n, 64, replace=False):
        i, j = divmod(int(p), wl.n)
        bp, bm = tb64.copy(), tb64.copy()
        bp[i, j] += 1e-2
        bm[i, j] -= 1e-2
        fd = (oracle.softmin_loss(fr64, bp, wl.w, tau)[0] - oracle.softmin_loss(fr64, bm, wl.w, tau)[0]) / 2e-2
        assert abs(gt[i, j] - fd) <= 1e-3 * max(abs(fd), 1e-2 * gmax), (i, j, gt[i, j], fd)


def test_autograd_function_and_refinement():
    frames, tmpl = stack(64, 64, 24, 8, seed=9)
    fr = torch.from_numpy(frames).cuda()
    t0 = torch.from_numpy(tmpl).cuda()
    plan = softmin_plan(fr, t0, 8)
    try:
        t = t0.clone().requires_grad_(True)
        loss = MocoSoftMin.apply(t, fr, plan, TAU, 0)
        (3.0 * loss).backward()
        tau = oracle_tau(frames, tmpl, 8)
        L, _, gb, _ = oracle.softmin_loss(frames.astype(np.float64), tmpl.astype(np.float64), 8, tau,
                                          grad_template=True)
        assert float(loss.detach()) == pytest.approx(L, rel=1e-4)
        g = t.grad.cpu().numpy()
        assert np.abs(g - 3.0 * gb).max() <= 1e-3 * np.abs(3.0 * gb).max()
    finally:
        plan.close()
    refined, losses = refine_template(fr, t0, 8, steps=20, lr=1.0)
    assert losses[-1] < losses[0]
    assert torch.isfinite(refined).all()
