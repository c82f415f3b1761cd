"""More than one level on the GPU (levels 2..4: the search on level L, one
3x3 refinement per finer level) against the oracle's general pyramid."""
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


def planted(b, s0, t0, fill=100):
    m, n = b.shape
    a = np.full((m, n), fill, np.uint16)
    a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
        b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    return a


def run(frames, b, w, L):
    m, n = b.shape
    with Plan(dict(m=m, n=n, w=w, levels=L), dev(b)) as plan:
        assert plan.info()["levels"] == L
        shifts, best, _, final = plan.align(dev(frames), best_cost=True, final_cost=True)
        torch.cuda.synchronize()
        return shifts.cpu().numpy(), best.cpu().numpy(), final.cpu().numpy()


@pytest.mark.parametrize("L", [2, 3])
def test_planted_noiseless_shifts(L):
    m = n = 256
    st = synth.make_stack_np(m, n, 1, 60, 0, seed=170 + L, template="clean", noise=False)
    b = st.template
    shifts = [(7, -5), (-11, 9), (3, 3), (-1, 10), (2 ** L * 3, -(2 ** L) * 2), (0, 0)]
    frames = np.stack([planted(b, s, t) for s, t in shifts])
    got, best, final = run(frames, b, 6, L)
    assert [tuple(x) for x in got] == shifts
    assert np.all(final == 0.0)
    ref = oracle.align(frames, b, 6, levels=L)
    assert np.array_equal(got, ref["shifts"])


@pytest.mark.parametrize("L,w", [(2, 16), (3, 8), (4, 5)])
def test_noisy_stack_matches_oracle(L, w):
    m = n = 512
    st = synth.make_stack_np(m, n, 24, 400, min(40, (w - 1) * 2 ** L), seed=190 + L, template="clean")
    got, best, final = run(st.frames, st.template, w, L)
    ref, exempt = check_align(st.frames, st.template, w, L, got, best)
    same = np.all(got == ref["shifts"], axis=1)
    # exact full-resolution sums on both sides: bit-identical where the shift agrees
    assert np.array_equal(final[same], ref["ffinal"][same])
    assert same.mean() >= 0.9


def test_ragged_sizes_and_cost_surface():
    m, n, L, w = 300, 264, 2, 6
    st = synth.make_stack_np(m, n, 9, 80, 10, seed=301, template="clean")
    got, best, final = run(st.frames, st.template, w, L)
    check_align(st.frames, st.template, w, L, got, best)
    with Plan(dict(m=m, n=n, w=w, levels=L), dev(st.template)) as plan:
        cost = plan.cost_surface(dev(st.frames[:4])).cpu().numpy()
    assert cost_rel_err(cost, oracle.cost_surface(st.frames[:4], st.template, w, levels=L)) <= COST_RTOL


def test_largest_frames_three_levels():
    # 4096 x 4096 frames (the largest the plan takes) through three levels:
    # the search on the 512 x 512 level-3 grid (576-point transforms), exact
    # 3x3 refinements on levels 2 and 1, the jitter at full resolution.
    m = n = 4096
    st = synth.make_stack_np(m, n, 2, 2000, 60, seed=4096, template="clean")
    got, best, final = run(st.frames, st.template, 12, 3)
    ref, _ = check_align(st.frames, st.template, 12, 3, got, best)
    same = np.all(got == ref["shifts"], axis=1)
    assert same.all()
    assert np.array_equal(final, ref["ffinal"])
