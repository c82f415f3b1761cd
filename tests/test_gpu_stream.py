"""The closed-loop single-frame mode (moco_stream_*): frame by frame from
host memory, the same shifts as the batched path and as the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import FrameStream, Plan, build, synth

from parity import check_align

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("m,n,w,levels", [(264, 264, 8, -1), (128, 96, 6, 0)])
def test_stream_matches_batched_and_oracle(m, n, w, levels):
    st = synth.make_stack_np(m, n, 12, 60, 6, seed=m + n, template="clean")
    with Plan(dict(m=m, n=n, w=w, levels=levels), torch.from_numpy(st.template).cuda()) as plan:
        batched = plan.align(torch.from_numpy(st.frames).cuda()).cpu().numpy()
        got = np.empty_like(batched)
        with FrameStream(plan) as fs:
            for f in range(st.frames.shape[0]):
                fs.frame.copy_(torch.from_numpy(st.frames[f]))
                got[f] = fs.align()
            # the handle replays the same graph: a second pass gives the same
            for f in range(3):
                fs.frame.copy_(torch.from_numpy(st.frames[f]))
                assert tuple(fs.align()) == tuple(got[f])
    assert np.array_equal(got, batched)
    check_align(st.frames, st.template, w, levels, got)
