"""moco_jitter_noalloc (the refinement step with static scratch, for callers
that cannot allocate device memory) against moco_align_stack, through the C
ABI, on two calls in a row. Collected last so that a stop at the first
failure has run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1506_06039_gb300 import Plan, binding, build, synth

pytestmark = pytest.mark.gpu


def host_argmin(cost, w):
    """Searched-grid optimum per frame with the library's tie-break
    (smallest f, then |s|+|t|, then s, then t) on the FP64 costs."""
    T = cost.shape[0]
    s, t = np.meshgrid(np.arange(-(w - 1), w), np.arange(-(w - 1), w), indexing="ij")
    out = np.empty((T, 2), np.int32)
    for f in range(T):
        order = np.lexsort((t.ravel(), s.ravel(), (np.abs(s) + np.abs(t)).ravel(), cost[f].ravel()))
        k = order[0]
        out[f] = (s.ravel()[k], t.ravel()[k])
    return out


def test_noalloc_jitter_matches_align_stack_twice():
    build.build()
    m, n, w, T = 320, 272, 10, 11
    st = synth.make_stack_np(m, n, T, 60, 12, seed=2718, template="clean")
    frames = torch.from_numpy(st.frames).cuda()
    tmpl = torch.from_numpy(st.template).cuda()
    with Plan(dict(m=m, n=n, w=w), tmpl) as plan:
        ref = plan.align(frames).cpu().numpy()
        cost = plan.cost_surface(frames).cpu().numpy()
    coarse = torch.from_numpy(host_argmin(cost, w)).cuda()
    lib = binding.lib()
    for _ in range(2):
        out = torch.full((T, 2), -12345, dtype=torch.int32, device="cuda")
        st_ = lib.moco_jitter_noalloc(ctypes.c_void_p(frames.data_ptr()), T, m, n, ctypes.c_void_p(tmpl.data_ptr()),
                                      ctypes.c_void_p(coarse.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st_ == binding.MOCO_OK, lib.moco_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_more_frames_than_its_scratch():
    build.build()
    lib = binding.lib()
    st_ = lib.moco_jitter_noalloc(ctypes.c_void_p(16), 8193, 64, 64, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None)
    assert st_ == binding.MOCO_ERR_INVALID_ARG
    assert b"8192" in lib.moco_last_error()
