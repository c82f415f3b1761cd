"""One stack over several GPUs: frames are independent given the template
(Section 2 aligns each frame against the one template on its own), so a stack
splits into contiguous frame ranges, one per rank. The template is broadcast
from one rank, every rank aligns its range with its own plan, and the shifts
(8 bytes per frame) are gathered so that every rank holds the whole stack's.
The only exchanges are that broadcast and that gather; nothing crosses ranks
while frames are searched.

Works with any torch.distributed backend (NCCL between GPUs; gloo on the CPU
for the tests); the per-rank alignment is a callable, normally
``lambda fr: plan.align(fr)`` with a Plan on the rank's own device.
"""
from __future__ import annotations


def frame_range(T: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous range [lo, hi) of rank `rank`'s frames: T split as evenly as
    possible, the first T % world ranks taking one frame more."""
    if world < 1 or not 0 <= rank < world or T < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and T >= 0")
    base, extra = divmod(T, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def broadcast_template(template, group=None, src: int = 0):
    """Every rank's `template` (same shape and dtype) becomes rank src's, in place.
    A 16-bit template travels as its bytes (a uint8 view): NCCL has no unsigned
    16-bit type and gloo no 16-bit integer type at all."""
    import torch
    import torch.distributed as dist
    wire = template.view(torch.uint8) if template.dtype in (torch.uint16, torch.int16) else template
    dist.broadcast(wire, src=src, group=group)
    return template


def gather_shifts(local_shifts, T: int, group=None):
    """Concatenation over ranks, in rank order, of each rank's (hi - lo, 2)
    int32 shifts: the (T, 2) shifts of the whole stack on every rank. Ranges
    differ by at most one frame, so each is padded to the longest first."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    longest = frame_range(T, world, 0)[1]
    pad = torch.zeros((longest, 2), dtype=local_shifts.dtype, device=local_shifts.device)
    pad[:local_shifts.shape[0]] = local_shifts
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = []
    for r in range(world):
        lo, hi = frame_range(T, world, r)
        out.append(parts[r][:hi - lo])
    return torch.cat(out, 0)


def align_sharded(frames, align_fn, group=None):
    """Shifts (T, 2) of the whole stack `frames` (T, m, n), computed by this
    rank for its own range only (align_fn(frames[lo:hi]) -> (hi - lo, 2) int32)
    and gathered from the others. `frames` may be a view the rank only reads
    within its range (for example a memory map or a device copy of its part
    placed at its offset)."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    T = frames.shape[0]
    lo, hi = frame_range(T, world, rank)
    local = align_fn(frames[lo:hi])
    if tuple(local.shape) != (hi - lo, 2):
        raise ValueError("align_fn returned shape %s for %d frames" % (tuple(local.shape), hi - lo))
    return gather_shifts(local, T, group)
