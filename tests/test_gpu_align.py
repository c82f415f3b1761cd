"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import Plan, build, synth

from parity import COST_RTOL, check_align, cost_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_align(frames, tmpl, w, levels=-1, **shape_kw):
    m, n = tmpl.shape
    with Plan(dict(m=m, n=n, w=w, levels=levels, **shape_kw), dev(tmpl)) as plan:
        shifts, best, margin = plan.align(dev(frames), best_cost=True, margin=True)
        torch.cuda.synchronize()
        return shifts.cpu().numpy(), best.cpu().numpy(), margin.cpu().numpy(), plan.info()


def test_tiny128_workload_matches_oracle():
    wl = synth.WORKLOADS["tiny128"]
    st = synth.make_stack_np(wl.m, wl.n, wl.T, wl.nblobs, wl.shift_max, wl.seed, template=wl.template)
    shifts, best, margin, info = run_align(st.frames, st.template, wl.w)
    assert info["levels"] == 0 and info["fft_rows"] >= 128 + wl.w - 1
    ref, exempt = check_align(st.frames, st.template, wl.w, -1, shifts, best)
    assert exempt == 0
    # the planted shifts are recovered on this clean-template stack
    assert np.array_equal(shifts, st.shifts)


def test_tiny128_cost_surface_within_tolerance():
    wl = synth.WORKLOADS["tiny128"]
    st = synth.make_stack_np(wl.m, wl.n, 16, wl.nblobs, wl.shift_max, wl.seed, template=wl.template)
    with Plan(dict(m=wl.m, n=wl.n, w=wl.w), dev(st.template)) as plan:
        cost = plan.cost_surface(dev(st.frames)).cpu().numpy()
    ref = oracle.cost_surface(st.frames, st.template, wl.w)
    assert cost_rel_err(cost, ref) <= COST_RTOL


@pytest.mark.parametrize("m,n,w,levels", [
    (72, 56, 7, 0),      # ragged, non-square, no level
    (40, 48, 1, 0),      # a single shift
    (33, 64, 17, 0),     # widest window: 2w - 1 == m
    (300, 264, 9, -1),   # one 2x2 level (max > 256), ragged searched grid 150 x 132
    (301, 272, 6, 1),    # odd m with a level: the last row is dropped
])
def test_ragged_shapes_match_oracle(m, n, w, levels):
    st = synth.make_stack_np(m, n, 7, max(4, m * n // 1500), min(w - 1, 5) * (2 if levels else 1),
                             seed=m * 1000 + n, template="clean")
    shifts, best, _, _ = run_align(st.frames, st.template, w, levels)
    check_align(st.frames, st.template, w, levels, shifts, best)
    with Plan(dict(m=m, n=n, w=w, levels=levels), dev(st.template)) as plan:
        cost = plan.cost_surface(dev(st.frames[:3])).cpu().numpy()
    assert cost_rel_err(cost, oracle.cost_surface(st.frames[:3], st.template, w, levels=levels)) <= COST_RTOL


@pytest.mark.parametrize("s0,t0", [(7, -5), (-13, 3), (1, 1), (0, -9)])
def test_planted_odd_shift_full_resolution_exact(s0, t0):
    # Noiseless frame = template moved by (s0, t0): f is exactly 0 there and the
    # jitter at full resolution must land on it.
    m = n = 320
    st = synth.make_stack_np(m, n, 1, 60, 0, seed=31 + s0, template="clean", noise=False)
    b = st.template
    a = np.full((m, n), 100, np.uint16)
    a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
        b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    shifts, best, _, _ = run_align(a[None], b, 12)
    assert tuple(shifts[0]) == (s0, t0)
    check_align(a[None], b, 12, -1, shifts, best)


def test_jitter_every_column_offset():
    # Planted noiseless full-resolution shifts whose doubled coarse optimum
    # covers every offset of the jitter's 8-column load blocks (t0 mod 8),
    # both signs, and shifts at the window edge.
    m = n = 288
    st = synth.make_stack_np(m, n, 1, 50, 0, seed=404, template="clean", noise=False)
    b = st.template
    planted = [(s, t) for s in (-17, -4, 0, 9) for t in range(-17, 18, 3)]
    frames = np.full((len(planted), m, n), 100, np.uint16)
    for f, (s0, t0) in enumerate(planted):
        frames[f, max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
            b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    shifts, best, _, _ = run_align(frames, b, 10)
    assert [tuple(x) for x in shifts] == planted
    check_align(frames, b, 10, -1, shifts, best)


def brute_ssd(a, b, s, t):
    """Exact sum over D of (a[i+s][j+t] - b[i][j])^2 by direct int64 evaluation."""
    m, n = b.shape
    i0, i1, j0, j1 = max(0, -s), min(m, m - s), max(0, -t), min(n, n - t)
    d = a[i0 + s:i1 + s, j0 + t:j1 + t].astype(np.int64) - b[i0:i1, j0:j1].astype(np.int64)
    return int((d * d).sum()), (i1 - i0) * (j1 - j0)


@pytest.mark.parametrize("m,n,w", [(264, 264, 40), (330, 296, 9)])
def test_full_range_values_final_cost_exact(m, n, w):
    # Values over the whole 16-bit range (both byte halves of every product
    # busy), planted shifts out to the window's edge (whole row bands of the
    # frame outside the overlap), a saturated and an all-zero frame. The
    # full-resolution cost at the returned shift must be S / Area with S the
    # exact integer sum, to the last bit.
    rng = np.random.default_rng(m * 7 + n + w)
    b = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    e = 2 * (w - 1) - 1
    planted = [(-e, e), (e, -e), (5, -7), (0, 1), (-e, 0), (e - 2, e)]
    frames = []
    for s0, t0 in planted:
        a = rng.integers(0, 65536, (m, n)).astype(np.int64)
        a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
            b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
        a += rng.integers(-3000, 3001, (m, n))
        frames.append(np.clip(a, 0, 65535).astype(np.uint16))
    frames += [np.full((m, n), 65535, np.uint16), np.zeros((m, n), np.uint16)]
    frames = np.stack(frames)
    with Plan(dict(m=m, n=n, w=w, levels=1), dev(b)) as plan:
        shifts, best, _, final = plan.align(dev(frames), best_cost=True, final_cost=True)
        torch.cuda.synchronize()
        shifts, best, final = shifts.cpu().numpy(), best.cpu().numpy(), final.cpu().numpy()
    check_align(frames, b, w, 1, shifts, best)
    assert [tuple(x) for x in shifts[:len(planted)]] == planted
    for f in range(frames.shape[0]):
        S, A = brute_ssd(frames[f], b, int(shifts[f, 0]), int(shifts[f, 1]))
        assert final[f] == S / A, (f, final[f], S, A)


def test_final_cost_equals_oracle_without_level():
    st = synth.make_stack_np(96, 80, 5, 30, 4, seed=77, template="clean")
    with Plan(dict(m=96, n=80, w=6, levels=0), dev(st.template)) as plan:
        shifts, best, _, final = plan.align(dev(st.frames), best_cost=True, final_cost=True)
        torch.cuda.synchronize()
    assert np.array_equal(final.cpu().numpy(), best.cpu().numpy())


def test_identity_and_constant_frames():
    rng = np.random.default_rng(3)
    b = rng.integers(0, 3000, (64, 64)).astype(np.uint16)
    frames = np.stack([b, np.full_like(b, 500), np.full_like(b, int(b.mean().round()))])
    shifts, best, margin, _ = run_align(frames, b, 9)
    # f = 0 at (0, 0) up to the FP32 cross term: within 1e-6 * max f
    ref = oracle.cost_surface(frames[:1], b, 9)
    assert tuple(shifts[0]) == (0, 0) and abs(best[0]) <= 1e-6 * ref.max()
    check_align(frames, b, 9, -1, shifts, best)
    c = np.full((64, 64), 700, np.uint16)
    shifts, best, margin, _ = run_align(np.stack([c, c]), c, 5)
    assert np.all(shifts == 0) and np.all(best == 0.0)


def test_empty_and_single_frame():
    st = synth.make_stack_np(64, 64, 1, 10, 3, seed=5, template="clean")
    with Plan(dict(m=64, n=64, w=6), dev(st.template)) as plan:
        out = plan.align(dev(st.frames[:0]))
        assert out.shape == (0, 2)
        one = plan.align(dev(st.frames[:1])).cpu().numpy()
    check_align(st.frames[:1], st.template, 6, -1, one)


def test_group_boundaries_do_not_change_results():
    st = synth.make_stack_np(96, 96, 23, 20, 6, seed=77, template="clean")
    a, _, _, _ = run_align(st.frames, st.template, 8, group_frames=5)
    b, _, _, _ = run_align(st.frames, st.template, 8, group_frames=0)
    assert np.array_equal(a, b)
    check_align(st.frames, st.template, 8, -1, a)


@pytest.mark.parametrize("group_frames", [0, 96])
def test_large_calls_match_separate_calls(group_frames):
    # 1100 frames with a level in one call (one group, or 12 groups of 96 with
    # a short last one) against calls of 100 frames: identical shifts, best
    # and final costs; the oracle checks a sample.
    T, m, n, w = 1100, 64, 72, 6
    st = synth.make_stack_np(m, n, T, 12, 8, seed=1234, template="clean")
    with Plan(dict(m=m, n=n, w=w, levels=1, group_frames=group_frames), dev(st.template)) as plan:
        a, ab, _, af = plan.align(dev(st.frames), best_cost=True, final_cost=True)
        parts = [plan.align(dev(st.frames[k:k + 100]), best_cost=True, final_cost=True) for k in range(0, T, 100)]
        torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), np.concatenate([p[0].cpu().numpy() for p in parts]))
    assert np.array_equal(ab.cpu().numpy(), np.concatenate([p[1].cpu().numpy() for p in parts]))
    assert np.array_equal(af.cpu().numpy(), np.concatenate([p[3].cpu().numpy() for p in parts]))
    sample = np.random.default_rng(5).choice(T, 40, replace=False)
    check_align(st.frames[sample], st.template, w, 1, a.cpu().numpy()[sample], ab.cpu().numpy()[sample])


def test_align_host_matches_device_path():
    st = synth.make_stack_np(264, 264, 11, 40, 6, seed=8, template="clean")
    with Plan(dict(m=264, n=264, w=8, group_frames=4), dev(st.template)) as plan:
        d = plan.align(dev(st.frames)).cpu().numpy()
        h = plan.align_host(torch.from_numpy(st.frames).pin_memory()).numpy()
    assert np.array_equal(d, h)
    check_align(st.frames, st.template, 8, -1, d)


def test_set_template_equals_fresh_plan():
    s1 = synth.make_stack_np(80, 80, 6, 15, 5, seed=1, template="clean")
    s2 = synth.make_stack_np(80, 80, 6, 15, 5, seed=2, template="clean")
    with Plan(dict(m=80, n=80, w=7), dev(s1.template)) as plan:
        plan.set_template(dev(s2.template))
        a = plan.cost_surface(dev(s2.frames)).cpu().numpy()
    with Plan(dict(m=80, n=80, w=7), dev(s2.template)) as plan:
        b = plan.cost_surface(dev(s2.frames)).cpu().numpy()
    assert np.array_equal(a, b)


def test_several_shapes_and_stacks_in_one_call():
    from paper_1506_06039_gb300 import moco_align_stack
    sa = synth.make_stack_np(64, 64, 5, 10, 4, seed=11, template="clean")
    sb = synth.make_stack_np(272, 264, 4, 40, 6, seed=12, template="clean")
    plan = Plan([dict(m=64, n=64, w=6), dict(m=272, n=264, w=5)], [dev(sa.template), dev(sb.template)])
    try:
        outa = torch.empty((5, 2), dtype=torch.int32, device="cuda")
        outb = torch.empty((4, 2), dtype=torch.int32, device="cuda")
        moco_align_stack(plan.handle, [dict(shape_idx=0, frames=dev(sa.frames), shifts=outa),
                                       dict(shape_idx=1, frames=dev(sb.frames), shifts=outb)])
        torch.cuda.synchronize()
    finally:
        plan.close()
    check_align(sa.frames, sa.template, 6, -1, outa.cpu().numpy())
    check_align(sb.frames, sb.template, 5, -1, outb.cpu().numpy())


def test_std512_clean_template_recovers_planted_shifts():
    # Same frame recipe with the clean (unshifted, noise-free) template: the
    # planted shifts are the answer on (almost) every frame.
    wl = synth.WORKLOADS["std512"]
    st = synth.make_stack_torch(wl.m, wl.n, 300, wl.nblobs, wl.shift_max, wl.seed, template="clean")
    with Plan(dict(m=wl.m, n=wl.n, w=wl.w), st.template) as plan:
        shifts = plan.align(st.frames).cpu().numpy()
    assert (shifts == st.shifts).all(axis=1).mean() > 0.99
    sample = np.random.default_rng(1).choice(300, 8, replace=False)
    check_align(st.frames.cpu().numpy()[sample], st.template.cpu().numpy(), wl.w, -1, shifts[sample])


def test_largest_fft_length_wide_window():
    # 520 x 520 without a level and w = 57: searched grid + window = 576, the
    # longest transform, and 113^2 shifts (the combine keeps 113^2 costs in
    # shared memory beside the 576-point transform buffer).
    m = n = 520
    w = 57
    st = synth.make_stack_np(m, n, 2, 300, 40, seed=5200, template="clean")
    shifts, best, margin, info = run_align(st.frames, st.template, w, levels=0)
    assert info["fft_rows"] == 576 and info["fft_cols"] == 576
    check_align(st.frames, st.template, w, 0, shifts, best)
    with Plan(dict(m=m, n=n, w=w, levels=0), dev(st.template)) as plan:
        cost = plan.cost_surface(dev(st.frames[:1])).cpu().numpy()
    assert cost_rel_err(cost, oracle.cost_surface(st.frames[:1], st.template, w, levels=0)) <= COST_RTOL
