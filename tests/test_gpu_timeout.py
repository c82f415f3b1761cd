"""The timeout path of the bounded device-side waits, made to run out on the
GPU without a fault: a wait on an mbarrier that nobody completes gives up
after about a second, the plan reports MOCO_ERR_TIMEOUT once, and the plan
and context stay usable (an alignment afterwards equals the one before)."""
import time

import pytest
import torch

from paper_1506_06039_gb300 import MocoError, Plan, build, synth
from paper_1506_06039_gb300.binding import MOCO_ERR_TIMEOUT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_wait_that_runs_out_reports_timeout_and_leaves_the_plan_usable():
    st = synth.make_stack_torch(128, 128, 8, 60, 6, synth.SEED_BASE + 71, template="clean")
    with Plan(dict(m=128, n=128, w=8), st.template) as plan:
        before = plan.align(st.frames).cpu()
        plan.status()  # nothing pending
        t0 = time.perf_counter()
        plan.selftest_wait()
        with pytest.raises(MocoError) as e:
            plan.status()
        waited = time.perf_counter() - t0
        assert e.value.status == MOCO_ERR_TIMEOUT
        assert 0.2 < waited < 30.0  # the wait gave up on its own clock limit
        plan.status()  # reported once, then cleared
        after = plan.align(st.frames).cpu()
        torch.cuda.synchronize()
    assert torch.equal(before, after)
