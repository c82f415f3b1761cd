"""Comparison rules between the CUDA path and the oracle (shared by GPU tests).

Tolerances, derived from the arithmetic: the cross term is FP32 (FFT) or
BF16 hi+lo with FP32 accumulation; energies are exact int64; the combine is
FP32 from the exact energies carried as FP32 pairs (an error-free sum of the
two energies, then one rounding in the difference with 2h and one in the
division by the area: about 1.2e-7 relative to f itself, whatever the
cancellation). An FP32 FFT correlation has an absolute error of order
u * log2(N) * ||a|| * ||b|| (u = 2^-24), so the error of f is of order
1e-6 * max f whatever f itself is. The cost surface must therefore agree
with the oracle's FP64 value within 1e-4 relative wherever f >= 1e-2 * max f
(max over that frame's window), and within the absolute 1e-6 * max f below
that (a relative error with the denominator floored at 1e-2 * max f). The
argmin must equal the oracle's on every frame whose oracle margin
(f2 - f1) / f1 exceeds 1e-5; below that margin (near-ties, which an FP32
cross term cannot resolve) the CUDA optimum's cost must still be within the
cost tolerance of the oracle's best. Full-resolution jitter sums are exact
int64 on both sides, so when the searched-grid optimum agrees the final
shift must be identical.
"""
import numpy as np

import oracle

COST_RTOL = 1e-4
COST_FLOOR = 1e-2
MARGIN = 1e-5


def cost_rel_err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = COST_FLOOR * ref.reshape(ref.shape[0], -1).max(axis=1)
    floor = floor.reshape((-1,) + (1,) * (ref.ndim - 1))
    return float((np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)).max())


def check_align(frames, template, w, levels, shifts_gpu, best_gpu=None, ref=None, nthreads=0):
    """Returns (oracle result, number of frames exempt by margin)."""
    if ref is None:
        ref = oracle.align(frames, template, w, levels=levels, nthreads=nthreads)
    shifts_gpu = np.asarray(shifts_gpu)
    decided = ref["margin"] > MARGIN
    bad = np.nonzero(decided & np.any(shifts_gpu != ref["shifts"], axis=1))[0]
    assert bad.size == 0, "frames %s: gpu %s vs oracle %s (margins %s)" % (
        bad[:8], shifts_gpu[bad[:8]].tolist(), ref["shifts"][bad[:8]].tolist(), ref["margin"][bad[:8]])
    if best_gpu is not None:
        best_gpu = np.asarray(best_gpu, np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            err = np.abs(best_gpu - ref["fbest"]) / np.abs(ref["fbest"])
        over = np.nonzero(~(err <= COST_RTOL))[0]
        if over.size:
            # near-zero optima: the floor is 1e-6 * the largest f of that frame
            fmax = oracle.cost_surface(np.asarray(frames)[over], template, w, levels=levels).reshape(over.size, -1).max(1)
            err2 = np.abs(best_gpu[over] - ref["fbest"][over]) / np.maximum(np.abs(ref["fbest"][over]),
                                                                             COST_FLOOR * fmax)
            assert err2.max() <= COST_RTOL, "best cost rel err %g (frames %s)" % (err2.max(), over[:8])
    return ref, int((~decided).sum())


def fbest_rel_err(best_gpu, ref):
    """Un-floored relative error of the optimum's cost, |f_gpu - f_ref| / f_ref
    (frames whose oracle optimum is exactly 0 are left out): the number the
    floored bar does not show."""
    best_gpu = np.asarray(best_gpu, np.float64)
    f = np.asarray(ref["fbest"], np.float64)
    keep = f > 0
    if not keep.any():
        return 0.0
    return float((np.abs(best_gpu[keep] - f[keep]) / f[keep]).max())


def check_margin(margin_gpu, best_gpu, ref, fmax):
    """The CUDA margin (f2 - f1) / f1 against the oracle's. Each of f1, f2 may
    be off by COST_RTOL * max(f, COST_FLOOR * fmax) (the cost bar), so with
    d_k that bound over f_k the margin may differ by (1 + margin) (d1 + d2) /
    (1 - d1). Frames with f1 = 0 compare only as 'infinite or not'."""
    mg = np.asarray(margin_gpu, np.float64)
    mr = np.asarray(ref["margin"], np.float64)
    f1 = np.asarray(ref["fbest"], np.float64)
    fmax = np.asarray(fmax, np.float64)
    f2 = f1 * (1.0 + mr)
    floor = COST_FLOOR * fmax
    with np.errstate(divide="ignore", invalid="ignore"):
        d1 = COST_RTOL * np.maximum(f1, floor) / f1
        d2 = COST_RTOL * np.maximum(f2, floor) / f2
        bound = (1.0 + mr) * (d1 + d2) / np.maximum(1.0 - d1, 1e-12)
    finite = np.isfinite(mr) & (f1 > 0) & (d1 < 0.5)
    bad = np.nonzero(finite & ~(np.abs(mg - mr) <= bound))[0]
    assert bad.size == 0, "margin: frames %s gpu %s oracle %s bound %s" % (
        bad[:8], mg[bad[:8]], mr[bad[:8]], bound[bad[:8]])
    return float(np.max(np.abs(mg - mr)[finite] / np.maximum(mr[finite], 1e-30))) if finite.any() else 0.0
