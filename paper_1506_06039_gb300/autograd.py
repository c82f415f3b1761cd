"""torch.autograd wrapper of the differentiable form (not in the paper).

MocoSoftMin computes, for a float template b and uint16 frames a_f,
    L = sum_f -tau_f log sum_{s,t} exp(-f_st(a_f, b) / tau_f),
    tau_f = tau_scale * median_{s,t} f_st (held constant),
with f Section 2's cost: moco_set_template, then moco_softmin_grad (cost
surface, soft-min and template adjoint in one pass) when the template
requires a gradient, else moco_cost_surface and moco_softmin. Only the
per-frame losses are summed here (a reduction of T numbers).
"""
from __future__ import annotations

import torch

from .binding import TEMPLATE_F32, Plan


class MocoSoftMin(torch.autograd.Function):
    """The summed soft-min loss. When the template requires a gradient, the
    forward pass computes it too (moco_softmin_grad: the frames' row spectra
    serve the search and the adjoint) and backward scales it by the incoming
    gradient (the loss is a scalar, its gradient linear in that factor);
    otherwise only the loss is computed."""

    @staticmethod
    def forward(ctx, template, frames, plan, tau_scale=0.05, shape_idx=0):
        plan.set_template(template.detach().contiguous(), shape_idx)
        if ctx.needs_input_grad[0]:
            loss, grad_t, _, _ = plan.softmin_grad(frames, tau_scale, shape_idx=shape_idx)
            ctx.save_for_backward(grad_t)
        else:
            cost = plan.cost_surface(frames, shape_idx)
            loss, _ = plan.softmin(cost, tau_scale, shape_idx)
        return loss.sum()

    @staticmethod
    def backward(ctx, grad_out):
        (grad_t,) = ctx.saved_tensors
        return grad_t * grad_out.to(grad_t.dtype), None, None, None, None


def softmin_plan(frames, template, w, group_frames=0):
    """A plan for the differentiable form: float template, no downsampling."""
    m, n = template.shape
    return Plan(dict(m=m, n=n, w=w, levels=0, template_dtype=TEMPLATE_F32, group_frames=group_frames),
                template.detach().float().contiguous())


def adam_refine(template0, step, steps=50, lr=1.0, group=None):
    """Adam on a float template. step(t) returns (loss, gradient) of this
    process's frames at template t. With a torch.distributed process group
    (one rank per GPU, each holding its own frames) the gradient and the loss
    are summed over the ranks before every update, so every rank applies the
    same update to the same template: the data-parallel form of the
    refinement, whose only exchange is this all-reduce of m x n floats.
    Returns (template, losses)."""
    tmpl = template0.detach().clone().float().requires_grad_(True)
    opt = torch.optim.Adam([tmpl], lr=lr)
    losses = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        loss, grad = step(tmpl)
        grad = grad.detach().to(tmpl.dtype).clone()
        loss = loss.detach().reshape(1).double().clone()
        if group is not None:
            import torch.distributed as dist
            dist.all_reduce(grad, group=group)
            dist.all_reduce(loss, group=group)
        tmpl.grad = grad
        opt.step()
        losses.append(float(loss))
    return tmpl.detach(), losses


def refine_template(frames, template0, w, steps=50, lr=1.0, tau_scale=0.05, plan=None, group=None):
    """Gradient-based template refinement with Adam (see adam_refine; group:
    an optional process group over which the frames are sharded). Returns
    (template, losses)."""
    own = plan is None
    if own:
        plan = softmin_plan(frames, template0, w)

    def step(t):
        loss = MocoSoftMin.apply(t, frames, plan, tau_scale, 0)
        (g,) = torch.autograd.grad(loss, t)
        return loss, g

    try:
        return adam_refine(template0, step, steps=steps, lr=lr, group=group)
    finally:
        if own:
            plan.close()
