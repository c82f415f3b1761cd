"""On the GPU: the measured arithmetic peaks (moco_alu_peak) fall within the
part's unit-count bounds, and one stack aligned through the sharding helpers
(a one-rank NCCL group: frame range, template broadcast, gathered shifts)
equals the plan's own alignment."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_1506_06039_gb300 import PEAK_DP2A, PEAK_FP32_FMA, Plan, build, moco_alu_peak, synth

pytestmark = pytest.mark.gpu


def test_alu_peaks_within_unit_count_bounds():
    build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32 = moco_alu_peak(PEAK_FP32_FMA)
    dp2a = moco_alu_peak(PEAK_DP2A)
    # upper bounds: 128 FP32 lanes x 2 flop and 64 dp2a lanes per SM at 2.2 GHz;
    # lower bounds: a quarter of those at 1 GHz (a measurement that is not the pipe)
    assert sms * 128 * 2 * 1.0e9 / 4 < fp32 < sms * 128 * 2 * 2.2e9
    assert sms * 64 * 1.0e9 / 4 < dp2a < sms * 64 * 2.2e9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_alignment_one_nccl_rank_equals_plan():
    import torch.distributed as dist
    from paper_1506_06039_gb300.shard import align_sharded, broadcast_template
    build.build()
    st = synth.make_stack_np(272, 264, 13, 40, 6, seed=77, template="clean")
    frames = torch.from_numpy(st.frames).cuda()
    tmpl = torch.from_numpy(st.template).cuda()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        t = tmpl.clone()
        broadcast_template(t)
        with Plan(dict(m=272, n=264, w=5), t) as plan:
            got = align_sharded(frames, lambda fr: plan.align(fr))
            want = plan.align(frames)
            torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())
