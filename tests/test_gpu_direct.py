"""The direct tensor-core form of the cross term (BF16 hi+lo x3, FP32
accumulation in tensor memory) against the FP64 oracle, on the same rules as
the FFT form (tests/parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_06039_gb300 import XCORR_AUTO, XCORR_DIRECT_BF16X3, XCORR_FFT_FP32, Plan, build, synth

from parity import COST_RTOL, check_align, cost_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def direct_plan(m, n, w, tmpl, levels=-1, **kw):
    return Plan(dict(m=m, n=n, w=w, levels=levels, xcorr=XCORR_DIRECT_BF16X3, **kw), tmpl)


def test_direct_small_cost_surface_and_shifts():
    st = synth.make_stack_np(64, 64, 5, 12, 3, seed=3, template="clean")
    with direct_plan(64, 64, 4, dev(st.template), levels=0) as plan:
        assert plan.info()["xcorr"] == XCORR_DIRECT_BF16X3
        cost = plan.cost_surface(dev(st.frames)).cpu().numpy()
        shifts, best, _ = plan.align(dev(st.frames), best_cost=True)
        torch.cuda.synchronize()
        plan.status()
    ref = oracle.cost_surface(st.frames, st.template, 4, levels=0)
    assert cost_rel_err(cost, ref) <= COST_RTOL
    check_align(st.frames, st.template, 4, 0, shifts.cpu().numpy(), best.cpu().numpy())


@pytest.mark.parametrize("m,n,w,levels", [(128, 128, 10, 0), (72, 200, 7, 0), (300, 264, 9, -1), (96, 64, 17, 0)])
def test_direct_shapes_match_oracle(m, n, w, levels):
    st = synth.make_stack_np(m, n, 9, max(4, m * n // 1500), min(w - 1, 5) * (2 if levels else 1),
                             seed=m + n, template="clean")
    with direct_plan(m, n, w, dev(st.template), levels=levels) as plan:
        cost = plan.cost_surface(dev(st.frames[:4])).cpu().numpy()
        shifts, best, _ = plan.align(dev(st.frames), best_cost=True)
        torch.cuda.synchronize()
        plan.status()
    assert cost_rel_err(cost, oracle.cost_surface(st.frames[:4], st.template, w, levels=levels)) <= COST_RTOL
    check_align(st.frames, st.template, w, levels, shifts.cpu().numpy(), best.cpu().numpy())


def test_direct_more_than_one_m_tile():
    st = synth.make_stack_np(64, 64, 300, 12, 4, seed=17, template="clean")
    with direct_plan(64, 64, 6, dev(st.template), levels=0) as plan:
        shifts = plan.align(dev(st.frames)).cpu().numpy()
        plan.status()
    check_align(st.frames, st.template, 6, 0, shifts)


def test_auto_form_agrees_with_both():
    st = synth.make_stack_np(128, 128, 12, 30, 6, seed=5, template="clean")
    res = {}
    for form in (XCORR_FFT_FP32, XCORR_DIRECT_BF16X3, XCORR_AUTO):
        with Plan(dict(m=128, n=128, w=8, xcorr=form), dev(st.template)) as plan:
            res[form] = plan.align(dev(st.frames)).cpu().numpy()
            if form == XCORR_AUTO:
                assert plan.info()["xcorr"] in (XCORR_FFT_FP32, XCORR_DIRECT_BF16X3)
    ref, _ = check_align(st.frames, st.template, 8, -1, res[XCORR_FFT_FP32])
    for form in (XCORR_DIRECT_BF16X3, XCORR_AUTO):
        check_align(st.frames, st.template, 8, -1, res[form], ref=ref)
