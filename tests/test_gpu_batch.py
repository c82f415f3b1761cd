"""The batching form: stacks of uneven frame size, length and window, each
with its own template, aligned in one moco_align_stack call, also replayed
from a captured CUDA graph; checked against the oracle on sampled frames."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import Plan, build, moco_align_stack, synth

from parity import check_align

pytestmark = pytest.mark.gpu

# (size, frames, w): every size and window of the mixed workload, with the
# oracle kept affordable (1024^2 only at small w).
SPECS = [(256, 37, 8), (512, 53, 16), (1024, 21, 8), (256, 29, 32), (512, 45, 64), (1024, 17, 16),
         (512, 31, 32), (256, 40, 64)]


@pytest.fixture(scope="module")
def batch():
    build.build()
    stacks = []
    for k, (size, T, w) in enumerate(SPECS):
        down = 2 if size > 256 else 1
        w = min(w, (size // down + 1) // 2)
        st = synth.make_stack_torch(size, size, T, max(1, int(400 * (size / 512) ** 2)),
                                    min(8, (w - 1) * down), seed=synth.SEED_BASE + 3 + 1000 * k, template="clean")
        stacks.append((st, w))
    shapes = [dict(m=st.frames.shape[1], n=st.frames.shape[2], w=w) for st, w in stacks]
    plan = Plan(shapes, [st.template for st, _ in stacks])
    yield plan, stacks
    plan.close()


def run(plan, stacks):
    outs = [torch.empty((st.frames.shape[0], 2), dtype=torch.int32, device="cuda") for st, _ in stacks]
    moco_align_stack(plan.handle, [dict(shape_idx=k, frames=st.frames, shifts=outs[k])
                                   for k, (st, _) in enumerate(stacks)])
    return outs


def test_mixed_batch_one_call_matches_oracle(batch):
    plan, stacks = batch
    outs = run(plan, stacks)
    torch.cuda.synchronize()
    plan.status()
    rng = np.random.default_rng(0)
    for k, (st, w) in enumerate(stacks):
        got = outs[k].cpu().numpy()
        # clean templates: planted shifts are the answer on (almost) every frame
        assert (got == st.shifts).all(axis=1).mean() >= 0.9, k
        pick = rng.choice(st.frames.shape[0], 2, replace=False)
        check_align(st.frames.cpu().numpy()[pick], st.template.cpu().numpy(), w, -1, got[pick])


def test_mixed_batch_from_captured_graph(batch):
    plan, stacks = batch
    eager = [o.cpu().numpy() for o in run(plan, stacks)]  # also sets kernel attributes before capture
    torch.cuda.synchronize()
    outs = [torch.full((st.frames.shape[0], 2), -7, dtype=torch.int32, device="cuda") for st, _ in stacks]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            moco_align_stack(plan.handle, [dict(shape_idx=k, frames=st.frames, shifts=outs[k])
                                           for k, (st, _) in enumerate(stacks)], stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for o in outs:
            o.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        for k in range(len(stacks)):
            assert np.array_equal(outs[k].cpu().numpy(), eager[k]), k
