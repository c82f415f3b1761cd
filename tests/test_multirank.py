"""The benchmark's multi-rank logic (one process per GPU, weak scaling, no
collective on the data path, time = the slowest rank) on two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_value(world, 2000, 7, ms / 1e3)
        q.put((rank, ms, value, bench.rank_seed(15060603901, rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    # every rank sees the slowest rank's time and the same whole-job value
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 2000 * 7 / 0.015)
    # each rank draws its own stack
    assert res[0][3] != res[1][3]


def test_single_rank_passthrough():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 2000, 10, 2.0) == 10000.0


# ---- data-parallel template refinement: the all-reduce of the gradient ------

def _refine_problem():
    import numpy as np
    from paper_1506_06039_gb300 import synth
    st = synth.make_stack_np(24, 32, 6, 5, 2, seed=44, template="clean")
    rng = np.random.default_rng(3)
    tmpl = st.frames.astype(np.float64).mean(0) + rng.normal(0, 20, (24, 32))
    return st.frames, tmpl.astype(np.float32), 4


def _oracle_step(frames, w):
    """Loss and template gradient of these frames (FP64 oracle, tau = 0.05 x
    median at the current template, held constant)."""
    import numpy as np
    import torch
    import oracle

    def step(t):
        tb = t.detach().double().numpy()
        tau = oracle.softmin_tau(frames, tb, w, 0.05)
        L, _, gb, _ = oracle.softmin_loss(frames.astype(np.float64), tb, w, tau, grad_template=True)
        return torch.tensor(L, dtype=torch.float64), torch.from_numpy(gb)
    return step


def _refine_worker(rank, world, port, q):
    import torch
    from paper_1506_06039_gb300.autograd import adam_refine
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames, tmpl, w = _refine_problem()
        t, losses = adam_refine(torch.from_numpy(tmpl), _oracle_step(frames[rank::world], w), steps=3, lr=2.0,
                                group=dist.group.WORLD)
        q.put((rank, t.numpy(), losses))
    finally:
        dist.destroy_process_group()


def test_two_rank_refinement_equals_one_process_over_all_frames():
    import numpy as np
    import torch
    from paper_1506_06039_gb300.autograd import adam_refine
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_refine_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=5) for _ in range(world)), key=lambda r: r[0])
    frames, tmpl, w = _refine_problem()
    t1, l1 = adam_refine(torch.from_numpy(tmpl), _oracle_step(frames, w), steps=3, lr=2.0)
    # every rank holds the same template: the one-process refinement over all frames
    assert np.array_equal(res[0][1], res[1][1])
    np.testing.assert_allclose(res[0][1], t1.numpy(), rtol=0, atol=1e-4)
    np.testing.assert_allclose(res[0][2], l1, rtol=1e-8)  # float32 gradients summed in another order
    assert not np.array_equal(t1.numpy(), tmpl)  # the template moved


# ---- one stack sharded over ranks: contiguous frame ranges, gathered shifts --

def test_frame_ranges_tile_the_stack():
    from paper_1506_06039_gb300.shard import frame_range
    for T in (0, 1, 7, 2000, 2001):
        for world in (1, 2, 3, 8):
            ranges = [frame_range(T, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == T
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1


def _shard_problem():
    from paper_1506_06039_gb300 import synth
    # 11 frames over two ranks (6 + 5): a ragged split; one 2x2 level and the jitter
    return synth.make_stack_np(272, 264, 11, 40, 10, seed=606, template="clean"), 6


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch
    import oracle
    from paper_1506_06039_gb300.shard import align_sharded, broadcast_template
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st, w = _shard_problem()
        # only rank 0 holds the template at first; the broadcast gives it to the other
        tmpl = torch.from_numpy(st.template.astype(np.uint16)) if rank == 0 else torch.zeros(st.template.shape,
                                                                                               dtype=torch.uint16)
        broadcast_template(tmpl)
        # counts above 32767 keep their bytes through the byte view
        high = torch.tensor([40000, 65535, 1, 32768], dtype=torch.uint16) if rank == 0 else \
            torch.zeros(4, dtype=torch.uint16)
        broadcast_template(high)
        assert high.to(torch.int32).tolist() == [40000, 65535, 1, 32768]
        seen = []

        def align_fn(fr):
            seen.append(fr.shape[0])
            r = oracle.align(fr, tmpl.numpy(), w)
            return torch.from_numpy(r["shifts"])

        shifts = align_sharded(st.frames, align_fn)
        q.put((rank, shifts.numpy(), seen))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_stack_equals_one_process():
    import numpy as np
    import oracle
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=5) for _ in range(world)), key=lambda r: r[0])
    st, w = _shard_problem()
    ref = oracle.align(st.frames, st.template, w)
    assert res[0][2] == [6] and res[1][2] == [5]  # each rank searched its own range only
    for r in res:
        assert np.array_equal(r[1], ref["shifts"])
