"""moco_jitter_noalloc, the refinement step for callers that cannot allocate
device memory (its scratch is a fixed static array), through the C ABI on two
calls in a row: against moco_align_stack's own refinement and against the
oracle's upsampling step, on a batch large enough for the kernel's full
32-row bands, with coarse optima whose candidates reach the frame's last rows
and columns, and with caller-given coarse shifts that leave no overlap (which
must come back as INT32_MIN). Collected last so that a stop at the first
failure has run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import Plan, binding, build, synth

pytestmark = pytest.mark.gpu

INT32_MIN = np.iinfo(np.int32).min


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


def raw_call(frames, tmpl, coarse, out):
    T, m, n = frames.shape
    return binding.lib().moco_jitter_noalloc(ctypes.c_void_p(frames.data_ptr()), T, m, n,
                                             ctypes.c_void_p(tmpl.data_ptr()), ctypes.c_void_p(coarse.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def two_calls(frames, tmpl, coarse):
    """The raw C entry point, then the Python wrapper: both results."""
    T = frames.shape[0]
    outs = []
    out = torch.full((T, 2), -12345, dtype=torch.int32, device="cuda")
    st_ = raw_call(frames, tmpl, coarse, out)
    assert st_ == binding.MOCO_OK, binding.lib().moco_last_error()
    torch.cuda.synchronize()
    outs.append(out.cpu().numpy())
    out2 = torch.full((T, 2), -12345, dtype=torch.int32, device="cuda")
    binding.moco_jitter_noalloc(frames, tmpl, coarse, out2)
    torch.cuda.synchronize()
    outs.append(out2.cpu().numpy())
    return outs


def test_noalloc_jitter_matches_align_stack_and_oracle_twice():
    build.build()
    # 11 warp items per frame (34 column groups x 10 bands of 32 rows) x 240 frames = 2640
    # warps, at least two waves of eight per SM of 152: the launcher keeps full 32-row bands
    m, n, w, T = 320, 272, 10, 240
    st = synth.make_stack_np(m, n, T, 60, 12, seed=2718, template="clean")
    frames = torch.from_numpy(st.frames).cuda()
    tmpl = torch.from_numpy(st.template).cuda()
    with Plan(dict(m=m, n=n, w=w), tmpl) as plan:
        ref = plan.align(frames).cpu().numpy()
        cost = plan.cost_surface(frames).cpu().numpy()
    coarse_h = host_argmin(cost, w)
    coarse = torch.from_numpy(coarse_h).cuda()
    want, _ = oracle.refine(st.frames, st.template, coarse_h)
    for got in two_calls(frames, tmpl, coarse):
        assert np.array_equal(got, ref)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("T", [7, 160])
def test_noalloc_jitter_frame_edges_and_rejected_coarse(T):
    # Coarse optima up to the largest allowed, |2 sc| + 1 = m - 1 and
    # |2 tc| + 1 = n - 1: the candidates' overlaps shrink to the frame's last
    # one to three rows and columns. Frames with random content and frames
    # that hold the template moved to the extreme shift. Some frames get a
    # coarse shift one past the limit: INT32_MIN comes back for exactly those.
    build.build()
    m, n = 320, 272
    hs, ht = (m - 2) // 2, (n - 2) // 2
    rng = np.random.default_rng(31 + T)
    b = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    frames = rng.integers(0, 65536, (T, m, n)).astype(np.uint16)
    edges = [(hs, ht), (-hs, -ht), (hs, -ht), (-hs, ht), (hs, 0), (0, -ht), (hs - 1, ht - 1)]
    coarse = np.stack([rng.integers(-hs, hs + 1, T), rng.integers(-ht, ht + 1, T)], 1).astype(np.int32)
    for f in range(T):
        coarse[f] = edges[f % len(edges)] if f % 3 == 0 or T < 10 else coarse[f]
    for f in range(0, T, 5):  # the template itself at the extreme odd shift (exact zero there)
        s0, t0 = 2 * int(coarse[f, 0]) + (1 if coarse[f, 0] > 0 else -1), 2 * int(coarse[f, 1]) + (1 if coarse[f, 1] >= 0 else -1)
        if abs(s0) < m and abs(t0) < n:
            a = frames[f]
            a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
                b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    bad = np.arange(T) % 4 == 3
    coarse[bad & (np.arange(T) % 8 == 3), 0] = hs + 1      # |2 sc| + 1 = m + 1
    coarse[bad & (np.arange(T) % 8 == 7), 1] = -(ht + 1)   # |2 tc| + 1 = n + 1
    want, _ = oracle.refine(frames, b, coarse)
    assert np.all(want[bad] == INT32_MIN) and not np.any(want[~bad] == INT32_MIN)
    fr = torch.from_numpy(frames).cuda()
    for got in two_calls(fr, torch.from_numpy(b).cuda(), torch.from_numpy(coarse).cuda()):
        assert np.array_equal(got, want), np.nonzero(np.any(got != want, axis=1))[0][:8]


def test_noalloc_rejects_more_frames_than_its_scratch():
    build.build()
    lib = binding.lib()
    st_ = lib.moco_jitter_noalloc(ctypes.c_void_p(16), 8193, 64, 64, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None)
    assert st_ == binding.MOCO_ERR_INVALID_ARG
    assert b"8192" in lib.moco_last_error()


def test_noalloc_wrapper_checks_shapes():
    build.build()
    fr = torch.zeros((3, 16, 16), dtype=torch.uint16, device="cuda")
    tm = torch.zeros((16, 8), dtype=torch.uint16, device="cuda")
    c = torch.zeros((3, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        binding.moco_jitter_noalloc(fr, tm, c, c.clone())
    with pytest.raises(ValueError):
        binding.moco_jitter_noalloc(fr, torch.zeros((16, 16), dtype=torch.uint16, device="cuda"), c[:2], c.clone())
