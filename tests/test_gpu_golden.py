"""The CUDA path against the golden fixtures (tests/golden): the worked
example's cost surface and argmin, and the planted stack's shifts and costs
(no level and one level)."""
import numpy as np
import pytest
import torch

from paper_1506_06039_gb300 import Plan, build

from parity import COST_RTOL, cost_rel_err
from test_golden import load_planted, load_worked, planted_stack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_worked_example_on_the_gpu():
    a, b, w, rows = load_worked()
    with Plan(dict(m=b.shape[0], n=b.shape[1], w=w, levels=0), dev(b)) as plan:
        cost = plan.cost_surface(dev(a[None])).cpu().numpy()[0]
        shifts = plan.align(dev(a[None])).cpu().numpy()
        torch.cuda.synchronize()
    ref = np.empty_like(cost)
    for s, t, S, A in rows:
        ref[s + w - 1, t + w - 1] = S / A
    assert cost_rel_err(cost[None], ref[None]) <= COST_RTOL
    assert tuple(shifts[0]) == (0, 1)  # the fixture's unique zero


@pytest.mark.parametrize("levels", [0, 1])
def test_planted_fixture_on_the_gpu(levels):
    st = planted_stack()
    rec = load_planted()[levels]
    want = np.array([(s, t) for _, s, t, _, _ in rec])
    fbest = np.array([fb for *_, fb, _ in rec])
    ffinal = np.array([ff for *_, ff in rec])
    with Plan(dict(m=64, n=72, w=6, levels=levels), dev(st.template)) as plan:
        shifts, best, _, final = plan.align(dev(st.frames), best_cost=True, final_cost=True)
        torch.cuda.synchronize()
    assert np.array_equal(shifts.cpu().numpy(), want)
    assert np.max(np.abs(best.cpu().numpy() - fbest) / fbest) <= COST_RTOL
    if levels:
        assert np.array_equal(final.cpu().numpy(), ffinal)  # exact int64 jitter sums on both sides
