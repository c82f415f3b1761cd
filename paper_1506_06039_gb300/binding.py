"""Python binding of include/moco.h (argument marshalling only).

Every function here has the C entry point's name and calls it through
ctypes with torch tensors' device pointers and the current CUDA stream;
all arithmetic runs in the CUDA library. The library must have been built
(paper_1506_06039_gb300.build.build()); if it is missing, lib() raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MOCO_OK = 0
MOCO_ERR_INVALID_ARG = 1
MOCO_ERR_UNSUPPORTED = 2
MOCO_ERR_OOM = 3
MOCO_ERR_CUDA = 4
MOCO_ERR_TIMEOUT = 5

XCORR_AUTO = 0
XCORR_FFT_FP32 = 1
XCORR_DIRECT_BF16X3 = 2

TEMPLATE_U16 = 0
TEMPLATE_F32 = 1

# Every entry point include/moco.h declares (checked by the CPU tests).
EXPORTS = (
    "moco_plan", "moco_set_template", "moco_align_stack", "moco_cost_surface", "moco_softmin",
    "moco_cost_backward", "moco_align_host", "moco_plan_query", "moco_plan_destroy",
    "moco_status_string", "moco_last_error", "moco_profile_enable", "moco_profile_read", "moco_plan_status",
    "moco_jitter_noalloc", "moco_apply_shifts", "moco_stream_create", "moco_stream_align", "moco_stream_destroy",
    "moco_softmin_grad", "moco_selftest_wait", "moco_alu_peak",
)

PEAK_FP32_FMA = 0
PEAK_DP2A = 1


class MocoShape(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("w", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("template_dtype", ctypes.c_int32),
                ("xcorr", ctypes.c_int32), ("group_frames", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MocoShapeInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("mc", ctypes.c_int32), ("nc", ctypes.c_int32),
                ("fft_rows", ctypes.c_int32), ("fft_cols", ctypes.c_int32),
                ("xcorr", ctypes.c_int32), ("group_frames", ctypes.c_int32),
                ("offset", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


class MocoStack(ctypes.Structure):
    _fields_ = [("shape_idx", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("frames_dev", ctypes.c_void_p), ("T", ctypes.c_int64),
                ("shifts_dev", ctypes.c_void_p), ("best_cost_dev", ctypes.c_void_p),
                ("margin_dev", ctypes.c_void_p), ("final_cost_dev", ctypes.c_void_p)]


class MocoKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class MocoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libmoco.so (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("libmoco.so is missing (%s): build it with "
                                   "paper_1506_06039_gb300.build.build()" % path)
            L = ctypes.CDLL(path)
            P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.moco_plan.argtypes = [ctypes.POINTER(MocoShape), i32, ctypes.POINTER(P), P, ctypes.POINTER(P)]
            L.moco_set_template.argtypes = [P, i32, P, P]
            L.moco_align_stack.argtypes = [P, ctypes.POINTER(MocoStack), i32, P]
            L.moco_cost_surface.argtypes = [P, i32, P, i64, P, P]
            L.moco_softmin.argtypes = [P, i32, P, i64, dbl, P, P, P]
            L.moco_cost_backward.argtypes = [P, i32, P, i64, P, ctypes.c_float, P, P, P]
            L.moco_softmin_grad.argtypes = [P, i32, P, i64, dbl, ctypes.c_float, P, P, P, P, P]
            L.moco_align_host.argtypes = [P, i32, P, i64, P, P]
            L.moco_plan_query.argtypes = [P, i32, ctypes.POINTER(MocoShapeInfo)]
            L.moco_plan_destroy.argtypes = [P]
            L.moco_status_string.argtypes = [i32]
            L.moco_status_string.restype = ctypes.c_char_p
            L.moco_last_error.argtypes = []
            L.moco_last_error.restype = ctypes.c_char_p
            L.moco_profile_enable.argtypes = [P, i32]
            L.moco_plan_status.argtypes = [P]
            L.moco_selftest_wait.argtypes = [P, i32, P]
            L.moco_jitter_noalloc.argtypes = [P, i64, i32, i32, P, P, P, P]
            L.moco_alu_peak.argtypes = [i32, P, ctypes.POINTER(dbl), P]
            L.moco_apply_shifts.argtypes = [P, i32, P, i64, P, ctypes.c_uint16, P, P, P]
            L.moco_stream_create.argtypes = [P, i32, P, P, ctypes.POINTER(P)]
            L.moco_stream_align.argtypes = [P, P]
            L.moco_stream_destroy.argtypes = [P]
            L.moco_profile_read.argtypes = [P, ctypes.POINTER(MocoKernelStat), i32, ctypes.POINTER(i32), i32]
            for name in EXPORTS:
                if name not in ("moco_status_string", "moco_last_error"):
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


def _status_name(status: int) -> str:
    try:
        return lib().moco_status_string(status).decode()
    except Exception:  # pragma: no cover
        return "status %d" % status


def _check(status: int):
    if status != MOCO_OK:
        raise MocoError(status, lib().moco_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, name, device=True):
    import torch
    if t is None:
        raise ValueError("%s is required" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if device and not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


# ---- the C entry points, one to one ---------------------------------------

def moco_plan(shapes, templates, stream=None) -> ctypes.c_void_p:
    """shapes: list of dicts with m, n, w and optional levels (-1),
    template_dtype (0 = U16, 1 = F32), xcorr (0 = auto), group_frames (0).
    templates: list of CUDA tensors (uint16 or float32, [m, n])."""
    import torch
    arr = (MocoShape * len(shapes))()
    for k, s in enumerate(shapes):
        arr[k] = MocoShape(int(s["m"]), int(s["n"]), int(s["w"]), int(s.get("levels", -1)),
                           int(s.get("template_dtype", TEMPLATE_U16)), int(s.get("xcorr", XCORR_AUTO)),
                           int(s.get("group_frames", 0)), 0)
        dt = torch.float32 if arr[k].template_dtype == TEMPLATE_F32 else torch.uint16
        _need(templates[k], dt, "template %d" % k)
    tp = (ctypes.c_void_p * len(templates))(*[t.data_ptr() for t in templates])
    out = ctypes.c_void_p()
    _check(lib().moco_plan(arr, len(shapes), tp, _stream(stream), ctypes.byref(out)))
    return out


def moco_set_template(plan, shape_idx, template, stream=None):
    _check(lib().moco_set_template(plan, shape_idx, _ptr(template), _stream(stream)))


def moco_align_stack(plan, stacks, stream=None):
    """stacks: list of dicts {shape_idx, frames, shifts, best_cost=None, margin=None, final_cost=None}."""
    import torch
    arr = (MocoStack * len(stacks))()
    for k, s in enumerate(stacks):
        fr = _need(s["frames"], torch.uint16, "frames")
        sh = _need(s["shifts"], torch.int32, "shifts")
        bc = s.get("best_cost")
        mg = s.get("margin")
        fc = s.get("final_cost")
        if bc is not None:
            _need(bc, torch.float64, "best_cost")
        if mg is not None:
            _need(mg, torch.float32, "margin")
        if fc is not None:
            _need(fc, torch.float64, "final_cost")
        T = fr.shape[0] if fr.dim() == 3 else 1
        arr[k] = MocoStack(int(s.get("shape_idx", 0)), 0, fr.data_ptr(), T, sh.data_ptr(),
                           bc.data_ptr() if bc is not None else None,
                           mg.data_ptr() if mg is not None else None,
                           fc.data_ptr() if fc is not None else None)
    _check(lib().moco_align_stack(plan, arr, len(stacks), _stream(stream)))


def moco_cost_surface(plan, shape_idx, frames, cost, stream=None):
    import torch
    _need(frames, torch.uint16, "frames")
    _need(cost, torch.float64, "cost")
    T = frames.shape[0] if frames.dim() == 3 else 1
    _check(lib().moco_cost_surface(plan, shape_idx, _ptr(frames), T, _ptr(cost), _stream(stream)))


def moco_apply_shifts(plan, shape_idx, frames, shifts, fill=0, corrected=None, mean=None, stream=None):
    """Corrected frames (uint16, like frames) and/or the corrected mean image
    (float64 [m, n]) into the given tensors (either may be None)."""
    import torch
    _need(frames, torch.uint16, "frames")
    _need(shifts, torch.int32, "shifts")
    if corrected is not None:
        _need(corrected, torch.uint16, "corrected")
    if mean is not None:
        _need(mean, torch.float64, "mean")
    T = frames.shape[0] if frames.dim() == 3 else 1
    _check(lib().moco_apply_shifts(plan, shape_idx, _ptr(frames), T, _ptr(shifts), int(fill),
                                   corrected.data_ptr() if corrected is not None else None,
                                   mean.data_ptr() if mean is not None else None, _stream(stream)))


class FrameStream:
    """The closed-loop single-frame mode: write a frame into .frame (pinned
    host, uint16 [m, n]), call align(), read .shift (pinned host, int32 [2])."""

    def __init__(self, plan, shape_idx=0):
        import torch
        m, n = int(plan.shapes[shape_idx]["m"]), int(plan.shapes[shape_idx]["n"])
        self.frame = torch.zeros((m, n), dtype=torch.uint16).pin_memory()
        self.shift = torch.zeros(2, dtype=torch.int32).pin_memory()
        self._plan = plan  # the plan must outlive the handle
        h = ctypes.c_void_p()
        _check(lib().moco_stream_create(plan.handle, shape_idx, self.frame.data_ptr(), self.shift.data_ptr(),
                                        ctypes.byref(h)))
        self.handle = h

    def align(self, stream=None):
        _check(lib().moco_stream_align(self.handle, _stream(stream)))
        return int(self.shift[0]), int(self.shift[1])

    def close(self):
        if self.handle:
            _check(lib().moco_stream_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def moco_softmin(plan, shape_idx, cost, tau_scale, loss, weights, stream=None):
    import torch
    _need(cost, torch.float64, "cost")
    _need(loss, torch.float64, "loss")
    _need(weights, torch.float32, "weights")
    _check(lib().moco_softmin(plan, shape_idx, _ptr(cost), cost.shape[0], float(tau_scale), _ptr(loss),
                              _ptr(weights), _stream(stream)))


def moco_cost_backward(plan, shape_idx, frames, grad_cost, grad_template, grad_frames=None, grad_scale=1.0,
                       stream=None):
    import torch
    _need(frames, torch.uint16, "frames")
    _need(grad_cost, torch.float32, "grad_cost")
    _need(grad_template, torch.float32, "grad_template")
    if grad_frames is not None:
        _need(grad_frames, torch.float32, "grad_frames")
    T = frames.shape[0] if frames.dim() == 3 else 1
    _check(lib().moco_cost_backward(plan, shape_idx, _ptr(frames), T, _ptr(grad_cost), float(grad_scale),
                                    _ptr(grad_template), _ptr(grad_frames), _stream(stream)))


def moco_softmin_grad(plan, shape_idx, frames, tau_scale, cost, loss, weights, grad_template, grad_scale=1.0,
                      stream=None):
    import torch
    _need(frames, torch.uint16, "frames")
    _need(cost, torch.float64, "cost")
    _need(loss, torch.float64, "loss")
    _need(weights, torch.float32, "weights")
    _need(grad_template, torch.float32, "grad_template")
    T = frames.shape[0] if frames.dim() == 3 else 1
    _check(lib().moco_softmin_grad(plan, shape_idx, _ptr(frames), T, float(tau_scale), float(grad_scale),
                                   _ptr(cost), _ptr(loss), _ptr(weights), _ptr(grad_template), _stream(stream)))


def moco_align_host(plan, shape_idx, frames_host, shifts_host, stream=None):
    import torch
    _need(frames_host, torch.uint16, "frames_host", device=False)
    _need(shifts_host, torch.int32, "shifts_host", device=False)
    if frames_host.is_cuda or shifts_host.is_cuda:
        raise ValueError("moco_align_host takes host tensors")
    T = frames_host.shape[0] if frames_host.dim() == 3 else 1
    _check(lib().moco_align_host(plan, shape_idx, _ptr(frames_host), T, _ptr(shifts_host), _stream(stream)))


def moco_plan_query(plan, shape_idx) -> dict:
    info = MocoShapeInfo()
    _check(lib().moco_plan_query(plan, shape_idx, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in MocoShapeInfo._fields_}


def moco_plan_destroy(plan):
    _check(lib().moco_plan_destroy(plan))


def moco_jitter_noalloc(frames, template, coarse, shifts, stream=None):
    """3x3 full-resolution refinement of given 2x2-grid optima; allocates nothing.
    frames (T, m, n) uint16, template (m, n) uint16, coarse and shifts (T, 2)
    int32, all on one CUDA device; runs on that device."""
    import torch
    _need(frames, torch.uint16, "frames")
    _need(template, torch.uint16, "template")
    _need(coarse, torch.int32, "coarse")
    _need(shifts, torch.int32, "shifts")
    if frames.dim() != 3:
        raise ValueError("frames must be (T, m, n)")
    T, m, n = frames.shape
    if tuple(template.shape) != (m, n):
        raise ValueError("template must be (%d, %d), got %s" % (m, n, tuple(template.shape)))
    if tuple(coarse.shape) != (T, 2) or tuple(shifts.shape) != (T, 2):
        raise ValueError("coarse and shifts must be (%d, 2)" % T)
    if len({t.device for t in (frames, template, coarse, shifts)}) != 1:
        raise ValueError("frames, template, coarse and shifts must be on one device")
    with torch.cuda.device(frames.device):
        _check(lib().moco_jitter_noalloc(_ptr(frames), T, m, n, _ptr(template), _ptr(coarse), _ptr(shifts),
                                         _stream(stream)))


def moco_alu_peak(kind: int, device=None) -> float:
    """Measured FP32 FMA (flop/s) or dp2a (instructions/s) rate of the current
    (or given) CUDA device; synchronises."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        sink = torch.zeros(1, dtype=torch.int32, device=dev)
        rate = ctypes.c_double(0.0)
        _check(lib().moco_alu_peak(int(kind), _ptr(sink), ctypes.byref(rate), _stream(None)))
    return float(rate.value)


def moco_plan_status(plan):
    _check(lib().moco_plan_status(plan))


def moco_selftest_wait(plan, shape_idx: int = 0, stream=None):
    _check(lib().moco_selftest_wait(plan, shape_idx, _stream(stream)))


def moco_profile_enable(plan, max_launches: int):
    _check(lib().moco_profile_enable(plan, int(max_launches)))


def moco_profile_read(plan, reset: bool = True) -> dict:
    """{kernel name: (launches, total_ms)} since the last reset."""
    cap = 16
    arr = (MocoKernelStat * cap)()
    cnt = ctypes.c_int32()
    _check(lib().moco_profile_read(plan, arr, cap, ctypes.byref(cnt), int(reset)))
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms))
            for k in range(min(cnt.value, cap))}


def moco_status_string(status: int) -> str:
    return lib().moco_status_string(status).decode()


# ---- a small object wrapper ---------------------------------------------

class Plan:
    """Owns a moco plan for one or more shapes.

        plan = Plan([dict(m=512, n=512, w=32)], [template_u16_cuda])
        shifts = plan.align(frames_u16_cuda)           # (T, 2) int32
    """

    def __init__(self, shapes, templates, stream=None):
        if isinstance(shapes, dict):
            shapes = [shapes]
        if not isinstance(templates, (list, tuple)):
            templates = [templates]
        self.shapes = [dict(s) for s in shapes]
        self.handle = moco_plan(self.shapes, list(templates), stream)

    def info(self, shape_idx=0) -> dict:
        return moco_plan_query(self.handle, shape_idx)

    def W(self, shape_idx=0) -> int:
        return 2 * int(self.shapes[shape_idx]["w"]) - 1

    def align(self, frames, shape_idx=0, best_cost=False, margin=False, final_cost=False, stream=None):
        """shifts; or (shifts, best_cost, margin) when either is asked for;
        with final_cost, (shifts, best_cost, margin, final_cost)."""
        import torch
        T = frames.shape[0]
        dev = frames.device
        shifts = torch.empty((T, 2), dtype=torch.int32, device=dev)
        bc = torch.empty(T, dtype=torch.float64, device=dev) if best_cost else None
        mg = torch.empty(T, dtype=torch.float32, device=dev) if margin else None
        fc = torch.empty(T, dtype=torch.float64, device=dev) if final_cost else None
        moco_align_stack(self.handle, [dict(shape_idx=shape_idx, frames=frames, shifts=shifts,
                                            best_cost=bc, margin=mg, final_cost=fc)], stream)
        if final_cost:
            return shifts, bc, mg, fc
        if best_cost or margin:
            return shifts, bc, mg
        return shifts

    def apply_shifts(self, frames, shifts, fill=0, corrected=True, mean=True, shape_idx=0, stream=None):
        """(corrected frames or None, corrected mean image float64 or None)."""
        import torch
        m, n = int(self.shapes[shape_idx]["m"]), int(self.shapes[shape_idx]["n"])
        out = torch.empty_like(frames) if corrected else None
        mu = torch.empty((m, n), dtype=torch.float64, device=frames.device) if mean else None
        moco_apply_shifts(self.handle, shape_idx, frames, shifts, fill, out, mu, stream)
        return out, mu

    def cost_surface(self, frames, shape_idx=0, stream=None):
        import torch
        W = self.W(shape_idx)
        cost = torch.empty((frames.shape[0], W, W), dtype=torch.float64, device=frames.device)
        moco_cost_surface(self.handle, shape_idx, frames, cost, stream)
        return cost

    def softmin(self, cost, tau_scale, shape_idx=0, stream=None):
        """(loss[T] float64, weights[T, W, W] float32) of a cost surface."""
        import torch
        loss = torch.empty(cost.shape[0], dtype=torch.float64, device=cost.device)
        weights = torch.empty(cost.shape, dtype=torch.float32, device=cost.device)
        moco_softmin(self.handle, shape_idx, cost, tau_scale, loss, weights, stream)
        return loss, weights

    def cost_backward(self, frames, grad_cost, grad_template=None, grad_frames=False, grad_scale=1.0,
                      shape_idx=0, stream=None):
        import torch
        m, n = int(self.shapes[shape_idx]["m"]), int(self.shapes[shape_idx]["n"])
        if grad_template is None:
            grad_template = torch.zeros((m, n), dtype=torch.float32, device=frames.device)
        gf = torch.empty(frames.shape, dtype=torch.float32, device=frames.device) if grad_frames else None
        moco_cost_backward(self.handle, shape_idx, frames, grad_cost, grad_template, gf, grad_scale, stream)
        return (grad_template, gf) if grad_frames else grad_template

    def softmin_grad(self, frames, tau_scale, grad_template=None, grad_scale=1.0, shape_idx=0, stream=None):
        """(loss[T] float64, grad_template[m, n] float32 (accumulated), cost, weights): the
        soft-min loss of every frame and the gradient of their sum with respect to the
        template, in one pass over the frames."""
        import torch
        W = self.W(shape_idx)
        m, n = int(self.shapes[shape_idx]["m"]), int(self.shapes[shape_idx]["n"])
        T = frames.shape[0]
        cost = torch.empty((T, W, W), dtype=torch.float64, device=frames.device)
        loss = torch.empty(T, dtype=torch.float64, device=frames.device)
        weights = torch.empty((T, W, W), dtype=torch.float32, device=frames.device)
        if grad_template is None:
            grad_template = torch.zeros((m, n), dtype=torch.float32, device=frames.device)
        moco_softmin_grad(self.handle, shape_idx, frames, tau_scale, cost, loss, weights, grad_template, grad_scale,
                          stream)
        return loss, grad_template, cost, weights

    def set_template(self, template, shape_idx=0, stream=None):
        moco_set_template(self.handle, shape_idx, template, stream)

    def align_host(self, frames_host, shape_idx=0, shifts_host=None, stream=None):
        import torch
        if shifts_host is None:
            shifts_host = torch.empty((frames_host.shape[0], 2), dtype=torch.int32).pin_memory()
        moco_align_host(self.handle, shape_idx, frames_host, shifts_host, stream)
        return shifts_host

    def status(self):
        """Raises MocoError (MOCO_ERR_TIMEOUT) if a device-side wait gave up."""
        moco_plan_status(self.handle)

    def selftest_wait(self, shape_idx: int = 0, stream=None):
        """Launches the timeout path's check (a bounded wait that gives up
        after about a second); the next status() raises MOCO_ERR_TIMEOUT."""
        moco_selftest_wait(self.handle, shape_idx, stream)

    def profile(self, max_launches: int):
        moco_profile_enable(self.handle, max_launches)

    def profile_read(self, reset: bool = True) -> dict:
        return moco_profile_read(self.handle, reset)

    def close(self):
        if self.handle:
            moco_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
