"""The correction step on the GPU (moco_apply_shifts, through the C ABI)
against the oracle: corrected frames and the corrected mean image must be
identical (uint16 values; the mean is one FP64 division of exact integers
on both sides)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import MocoError, Plan, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(plan, frames, shifts, fill, corrected=True, mean=True):
    c, mu = plan.apply_shifts(dev(frames), dev(shifts.astype(np.int32)), fill=fill, corrected=corrected, mean=mean)
    torch.cuda.synchronize()
    return (c.cpu().numpy() if c is not None else None), (mu.cpu().numpy() if mu is not None else None)


@pytest.mark.parametrize("m,n", [(70, 136), (64, 64), (33, 8)])
def test_random_shifts_match_oracle(m, n):
    rng = np.random.default_rng(m * n)
    T = 37
    frames = rng.integers(0, 65536, (T, m, n)).astype(np.uint16)
    # every column offset mod 8, both signs, zero, and shifts past the frame
    shifts = np.stack([rng.integers(-m // 2, m // 2 + 1, T), rng.integers(-n, n + 1, T)], 1)
    shifts[:16, 1] = np.arange(-8, 8)
    shifts[16] = (m, 0)
    shifts[17] = (0, -n - 5)
    shifts[18] = (-(m + 100), n + 100)
    shifts[19] = (0, 0)
    tmpl = frames[0]
    with Plan(dict(m=m, n=n, w=2, levels=0), dev(tmpl)) as plan:
        for fill in (0, 517):
            c, mu = run(plan, frames, shifts, fill)
            rc, rmu = oracle.apply_shifts(frames, shifts, fill=fill)
            assert np.array_equal(c, rc)
            assert np.array_equal(mu, rmu)
        c_only, none = run(plan, frames, shifts, 3, mean=False)
        assert none is None and np.array_equal(c_only, oracle.apply_shifts(frames, shifts, fill=3)[0])
        none, mu_only = run(plan, frames, shifts, 3, corrected=False)
        assert none is None and np.array_equal(mu_only, oracle.apply_shifts(frames, shifts, fill=3)[1])


def test_align_then_apply_recovers_template_region():
    # noiseless clean frames: after alignment, the corrected frames equal the
    # rounded template wherever their source is inside the frame
    m = n = 128
    st = synth.make_stack_np(m, n, 12, 40, 6, seed=21, template="clean", noise=False)
    b = st.template
    frames = np.full((12, m, n), 100, np.uint16)
    for f, (s0, t0) in enumerate(st.shifts):
        frames[f, max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
            b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    with Plan(dict(m=m, n=n, w=8), dev(b)) as plan:
        shifts = plan.align(dev(frames)).cpu().numpy()
        c, mu = run(plan, frames, shifts, 0)
    assert np.array_equal(shifts, st.shifts)
    rc, rmu = oracle.apply_shifts(frames, shifts, fill=0)
    assert np.array_equal(c, rc) and np.array_equal(mu, rmu)
    for f, (s0, t0) in enumerate(shifts):
        inside = np.zeros((m, n), bool)
        inside[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)] = True
        assert np.array_equal(c[f][inside], b[inside])


def test_full_size_workload_after_alignment():
    # the benchmark's configuration: 2000 frames of 512x512, the shifts the
    # search returns, the mean over every frame compared in full, corrected
    # frames on a seeded sample
    wl = synth.WORKLOADS["std512"]
    st = synth.make_stack_torch(wl.m, wl.n, wl.T, wl.nblobs, wl.shift_max, seed=wl.seed, template=wl.template)
    with Plan(dict(m=wl.m, n=wl.n, w=wl.w), st.template) as plan:
        shifts = plan.align(st.frames)
        c, mu = plan.apply_shifts(st.frames, shifts, fill=100)
        torch.cuda.synchronize()
    frames_h = st.frames.cpu().numpy()
    shifts_h = shifts.cpu().numpy()
    _, rmu = oracle.apply_shifts(frames_h, shifts_h, fill=100, corrected=False)
    assert np.array_equal(mu.cpu().numpy(), rmu)
    pick = np.random.default_rng(5).choice(wl.T, 6, replace=False)
    rc, _ = oracle.apply_shifts(frames_h[pick], shifts_h[pick], fill=100, mean=False)
    assert np.array_equal(np.stack([c[int(k)].cpu().numpy() for k in pick]), rc)


def test_empty_stack_and_errors():
    m, n = 32, 64
    tmpl = np.zeros((m, n), np.uint16)
    with Plan(dict(m=m, n=n, w=2, levels=0), dev(tmpl)) as plan:
        c, mu = run(plan, np.zeros((0, m, n), np.uint16), np.zeros((0, 2), np.int32), 77)
        assert c.shape == (0, m, n) and np.all(mu == 77.0)
        frames = torch.zeros((3, m, n), dtype=torch.uint16, device="cuda")
        shifts = torch.zeros((3, 2), dtype=torch.int32, device="cuda")
        flat = torch.zeros(3 * m * n + 8, dtype=torch.uint16, device="cuda")
        with pytest.raises(MocoError):  # misaligned frames
            plan.apply_shifts(flat[1:1 + 3 * m * n].view(3, m, n), shifts)
        with pytest.raises(MocoError):  # misaligned output
            c = torch.zeros(3 * m * n + 8, dtype=torch.uint16, device="cuda")
            from paper_1506_06039_gb300 import moco_apply_shifts
            moco_apply_shifts(plan.handle, 0, frames, shifts, 0, c[1:1 + 3 * m * n].view(3, m, n), None)
