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


def all_outputs(plan, items):
    """One moco_align_stack call over `items` [(shape_idx, frames)] with every
    output requested; returns numpy (shifts, best, margin, final) per item."""
    outs = []
    for k, fr in items:
        T = fr.shape[0]
        outs.append(dict(shape_idx=k, frames=fr, shifts=torch.empty((T, 2), dtype=torch.int32, device="cuda"),
                         best_cost=torch.empty(T, dtype=torch.float64, device="cuda"),
                         margin=torch.empty(T, dtype=torch.float32, device="cuda"),
                         final_cost=torch.empty(T, dtype=torch.float64, device="cuda")))
    moco_align_stack(plan.handle, outs)
    torch.cuda.synchronize()
    return [tuple(o[key].cpu().numpy() for key in ("shifts", "best_cost", "margin", "final_cost")) for o in outs]


def test_several_stacks_equal_one_stack_at_a_time(batch):
    # Several stacks with a level take the persistent several-stack refinement
    # (their optima parked in the shift buffers); alone, each takes the
    # one-stack path. Every output must be identical.
    plan, stacks = batch
    together = all_outputs(plan, [(k, st.frames) for k, (st, _) in enumerate(stacks)])
    for k, (st, _) in enumerate(stacks):
        alone = all_outputs(plan, [(k, st.frames)])[0]
        for a, b in zip(together[k], alone):
            assert np.array_equal(a, b), k


def test_several_stacks_beyond_one_refinement_launch():
    # 33000 frames of 16 x 16 with one level (more than the 32768 frames one
    # refinement launch holds) next to a 272 x 264 stack: the refinement is
    # split over launches; results equal the one-stack path and the oracle.
    build.build()
    big = synth.make_stack_np(16, 16, 33000, 2, 2, seed=91, template="clean")
    small = synth.make_stack_np(272, 264, 9, 40, 6, seed=92, template="clean")
    plan = Plan([dict(m=16, n=16, w=2, levels=1), dict(m=272, n=264, w=5)],
                [torch.from_numpy(big.template).cuda(), torch.from_numpy(small.template).cuda()])
    try:
        fb, fs = torch.from_numpy(big.frames).cuda(), torch.from_numpy(small.frames).cuda()
        together = all_outputs(plan, [(0, fb), (1, fs)])
        alone = [all_outputs(plan, [(0, fb)])[0], all_outputs(plan, [(1, fs)])[0]]
        plan.status()
    finally:
        plan.close()
    for t, a in zip(together, alone):
        for x, y in zip(t, a):
            assert np.array_equal(x, y)
    pick = np.random.default_rng(3).choice(33000, 64, replace=False)
    pick = np.concatenate([pick, [32767, 32768, 32999]])  # around the launch boundary
    check_align(big.frames[pick], big.template, 2, 1, together[0][0][pick])
    check_align(small.frames, small.template, 5, -1, together[1][0])
