"""Benchmark: frames/s aligned on the standard workload (2000 frames of
512x512 uint16, one 2x2 box level to 256x256, window w = 32, exhaustive
search then the 3x3 jitter at full resolution), synthetic calcium-like data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl moco|reference]

One step = one full alignment of the whole stack (every kernel of the path)
with the frames already resident in device memory; the stack (1 GiB) is
larger than L2, so no flush is needed between steps. Prints one JSON line.
Under torchrun each rank aligns its own stack (weak scaling, no collective on
the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s aligned (256², w=32, full search+upsample), plain vs chosen form"
UNIT = "frames/s"
FP32_LANES_PER_SM = 128
INT_MAD_LANES_PER_SM = 64  # 32-bit integer multiply-add (and dp2a) pipe
NUM_SMS = 152
SM_MAX_MHZ = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="moco", choices=["moco", "reference"])
    p.add_argument("--workload", default="std512")
    p.add_argument("--frames", type=int, default=0, help="override the workload's frame count (profiling runs)")
    p.add_argument("--form", default="auto", choices=["auto", "fft", "direct"])
    p.add_argument("--group", type=int, default=0, help="frames per internal batch (0 = plan's choice)")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-correction", action="store_true", help="skip the correction-step measurement")
    p.add_argument("--correction-steps", type=int, default=50)
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(seed, rank):
    """Weak scaling: every rank aligns its own stack, drawn from its own seed."""
    return seed + 1000 * rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's number (the job's time); x itself with one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, frames_per_rank, steps, seconds):
    """Whole-job frames/s: the frames all ranks aligned over the slowest rank's time."""
    return world * frames_per_rank * steps / seconds


def workload_config(wl, form):
    level = wl.m > 256 or wl.n > 256  # the paper's rule: one 2x2 level above 256x256
    desc = ("%s: %d frames of %dx%d uint16, 2x2 box to %dx%d, w=%d on the searched grid, 3x3 jitter at full "
            "resolution" % (wl.name, wl.T, wl.m, wl.n, wl.m // 2, wl.n // 2, wl.w)) if level else \
        ("%s: %d frames of %dx%d uint16, no level, w=%d" % (wl.name, wl.T, wl.m, wl.n, wl.w))
    return {
        "workload": desc,
        "frames": wl.T, "m": wl.m, "n": wl.n, "w": wl.w, "blobs": wl.nblobs,
        "shift_range": wl.shift_max,
        "template": "rounded mean of the first 100 frames" if wl.template == "mean100" else "clean (rounded X0)",
        "form": form,
        "l2": "inputs (%.0f MiB of frames) larger than L2; no flush" % (wl.T * wl.m * wl.n * 2 / 2 ** 20),
    }


# ---- clocks during the timed region ------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "moco_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6],
                                 swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in rows):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---- algorithmic work per kernel launch ----------------------------------------

def fft_flops(N):
    return 5.0 * N * math.log2(N)


def kernel_work(info, wl, frames):
    """Per-kernel algorithmic work for `frames` frames: (bytes, flops, exact
    integer multiply-adds)."""
    m, n, w = wl.m, wl.n, wl.w
    mc, nc, Nr, Nc = info["mc"], info["nc"], info["fft_rows"], info["fft_cols"]
    W = 2 * w - 1
    ncv = Nc // 2 + 1
    per = {
        # direct form: three BF16 products (hi.hi, hi.lo, lo.hi) of the W^2-shift contraction
        "k_direct": (2 * mc * nc * 2, 3 * 2.0 * W * W * mc * nc, 0.0),
        "k_frame_rows": (2 * m * n + 8 * ncv * mc, (mc / 2) * fft_flops(Nc), 0.0),
        "k_energy": (8 * (mc + nc) + 8 * W * W, 0.0, 0.0),
        "k_cols": (8 * ncv * mc + 8 * W * ncv, ncv * (2 * fft_flops(Nr) + 6 * Nr), 0.0),
        # h's row spectra in, the energies' edge sums and corner blocks in, the costs out
        "k_rows_inv": (8 * W * ncv + 8 * (mc + nc) + 16 * (w - 1) ** 2 + 8 * W * W,
                       math.ceil(W / 2) * fft_flops(Nc), 0.0),
        # nine exact squared differences per full-resolution pixel
        "k_jitter": (2 * m * n, 0.0, 9.0 * m * n),
    }
    return {k: (b * frames, f * frames, i * frames) for k, (b, f, i) in per.items()}


# DRAM bytes (read + write) per frame of the current kernels, from one ncu
# capture of 512 frames of the std512 workload in the FFT form
# (dram__bytes_read.sum + dram__bytes_write.sum of the first timed step's
# launches), scaled to a launch by its frame count; other workloads and
# forms report no traffic.
TRAFFIC_WORKLOAD = ("std512", "fft_fp32")
TRAFFIC_PER_FRAME = {"k_frame_rows": (270.745600e6 + 126.752256e6) / 512,
                     "k_cols": (152.447488e6 + 20.004864e6) / 512,
                     "k_rows_inv": (45.940224e6 + 0.0e6) / 512,
                     "k_jitter": (261.729792e6 + 3.866624e6) / 512}


# The bound of each kernel in the method's roofline (the frame pass and the
# upsampling step read every full-resolution pixel: HBM; the transforms: FP32
# ALU; the direct form's contraction: tensor cores). `frac` is taken against
# that bound; the fractions against the other peaks are reported beside it.
KERNEL_BOUND = {"k_frame_rows": "hbm", "k_jitter": "hbm", "k_cols": "fp32", "k_rows_inv": "fp32",
                "k_direct": "tensor", "k_energy": "hbm"}


def measured_alu_peaks():
    """FP32 FMA (TFLOP/s) and dp2a (T instructions/s) rates measured on this
    device by the library's own loop kernels (moco_alu_peak), or the unit-count
    figures at the maximum clock when that call fails."""
    from paper_1506_06039_gb300 import PEAK_DP2A, PEAK_FP32_FMA, moco_alu_peak
    out = {}
    for key, kind, derived in (("fp32", PEAK_FP32_FMA, NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6),
                               ("int", PEAK_DP2A, NUM_SMS * INT_MAD_LANES_PER_SM * SM_MAX_MHZ * 1e6)):
        try:
            out[key] = (moco_alu_peak(kind) / 1e12, "measured (moco_alu_peak: 16 independent chains per thread, "
                                                   "one resident wave on every SM, best of 3 x ~20 ms)")
        except Exception as exc:  # pragma: no cover - reported, not hidden
            out[key] = (derived / 1e12, "derived from unit counts at %d MHz (moco_alu_peak failed: %s)"
                        % (SM_MAX_MHZ, exc))
    return out


def roofline(profile, info, wl, frames_per_step, steps, peaks, alu):
    """Dominant kernel (largest share of device time) against its bound."""
    total = sum(ms for _, ms in profile.values()) or 1.0
    name = max(profile, key=lambda k: profile[k][1])
    launches, ms = profile[name]
    work = kernel_work(info, wl, frames_per_step * steps)
    byts, flops, imads = work.get(name, (0.0, 0.0, 0.0))
    dur_s = ms / 1e3
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp32_peak, fp32_src = alu["fp32"]
    imad_peak, imad_src = alu["int"]
    tensor = name == "k_direct"  # its flops run on the tensor cores (BF16), the others' on FP32 lanes
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
    fracs = {"hbm": (byts / dur_s / 1e9) / hbm if byts else 0.0,
             "fp32": (flops / dur_s / 1e12) / fp32_peak if flops and not tensor else 0.0,
             "tensor": (flops / dur_s / 1e12) / bf16_peak if flops and tensor else 0.0,
             "int": (imads / dur_s / 1e12) / imad_peak if imads else 0.0}
    bound = KERNEL_BOUND.get(name, "hbm")
    if bound == "tensor":
        rf = {"bound": "tensor", "achieved": flops / dur_s / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
              "frac": fracs["tensor"],
              "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured; kernel timed inside a long step)"}
    elif bound == "fp32":
        rf = {"bound": "alu", "achieved": flops / dur_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
              "frac": fracs["fp32"], "peak_source": "FP32 FMA, " + fp32_src}
    else:
        rf = {"bound": "hbm", "achieved": byts / dur_s / 1e9, "peak": hbm, "unit": "GB/s", "frac": fracs["hbm"],
              "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    per_launch_frames = frames_per_step * steps / launches
    from paper_1506_06039_gb300 import XCORR_DIRECT_BF16X3, XCORR_FFT_FP32
    form = {XCORR_FFT_FP32: "fft_fp32", XCORR_DIRECT_BF16X3: "direct_bf16x3"}.get(info.get("xcorr"))
    traffic = TRAFFIC_PER_FRAME.get(name) if (wl.name, form) == TRAFFIC_WORKLOAD else None
    rf.update({"kernel": name, "launches": launches, "avg_launch_ms": ms / launches,
               "share": ms / total,
               "traffic": traffic * per_launch_frames if traffic else None,
               "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum on 512 frames, scaled to "
                                  "%d frames per launch" % per_launch_frames) if traffic else None,
               "algorithmic_per_launch": {"bytes": byts / launches, "flops": flops / launches,
                                          "int_mads": imads / launches},
               "fractions": fracs,
               "peaks": {"hbm_gbs": hbm, "fp32_tflops": fp32_peak, "dp2a_tops": imad_peak, "bf16_tflops": bf16_peak,
                         "fp32_source": fp32_src, "dp2a_source": imad_src}})
    return rf


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ---- CPU baseline: the oracle as it stands --------------------------------------

def cpu_baseline(frames_host, template_host, w, seconds):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    chunk = cores
    while True:
        sel = frames_host[done % len(frames_host):done % len(frames_host) + chunk]
        oracle.align(sel, template_host, w, nthreads=cores)
        done += len(sel)
        el = time.perf_counter() - t0
        if el >= seconds or done >= len(frames_host):
            break
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d frames of the same workload (%.1f s, OpenMP over frames)" % (done, el)}


def accuracy_sample(plan, frames_dev, template_host, w, shifts_dev, sample=16, seed=0):
    """Part of the CPU-baseline leg: the oracle's FP64 results on a seeded
    sample of the timed frames against the CUDA path's. The CUDA costs come
    from one moco_cost_surface call over the whole stack (the timed launch
    configuration), the optimum's cost and the margin from one untimed
    moco_align_stack call with those outputs; the shifts are the timed run's.
    Cost error: pointwise, relative, denominator floored at 1e-2 x the frame's
    largest f; also without the floor at the optimum and normwise."""
    import numpy as np
    import torch
    import oracle
    T = frames_dev.shape[0]
    idx = np.sort(np.random.default_rng(seed).choice(T, min(sample, T), replace=False))
    sel = torch.from_numpy(idx).to(frames_dev.device)
    shifts2, best, margin = plan.align(frames_dev, best_cost=True, margin=True)
    cost = plan.cost_surface(frames_dev)
    cost_s = cost[sel].cpu().numpy()
    del cost
    torch.cuda.synchronize()
    deterministic = bool(torch.equal(shifts2, shifts_dev))
    fr = frames_dev.view(torch.int16)[sel].view(torch.uint16).cpu().numpy()  # (no uint16 gather kernel)
    shifts = shifts_dev[sel].cpu().numpy()
    best, margin = best[sel].cpu().numpy(), margin[sel].cpu().numpy()
    ref_cost = oracle.cost_surface(fr, template_host, w)
    ref = oracle.align(fr, template_host, w)
    k = len(idx)
    fmax = ref_cost.reshape(k, -1).max(1)
    d = np.abs(cost_s - ref_cost).reshape(k, -1)
    floored = d / np.maximum(np.abs(ref_cost).reshape(k, -1), 1e-2 * fmax[:, None])
    f1 = ref["fbest"]
    pos = f1 > 0
    at_best = float((np.abs(best[pos] - f1[pos]) / f1[pos]).max()) if pos.any() else 0.0
    fin = np.isfinite(ref["margin"]) & pos
    mg_err = float((np.abs(margin[fin] - ref["margin"][fin]) / np.maximum(ref["margin"][fin], 1e-30)).max()) \
        if fin.any() else 0.0
    decided = ref["margin"] > 1e-5
    agree = np.all(shifts == ref["shifts"], axis=1)
    return {"sample": "%d frames (seeded) of the %d timed frames; oracle: exact int64 brute force, FP64" % (k, T),
            "max_cost_rel_err_floored": float(floored.max()),
            "max_cost_err_normwise": float((d.max(1) / fmax).max()),
            "max_rel_err_at_fbest": at_best,
            "max_margin_rel_err": mg_err,
            "argmin_agree": int(agree.sum()), "argmin_agree_decided": int((agree & decided).sum()),
            "exempt": int((~decided).sum()), "frames": k,
            "min_fbest_over_fmax": float((f1 / fmax).min()),
            "deterministic_rerun": deterministic,
            "bars": {"cost_rel": 1e-4, "floor": "1e-2 x max f", "argmin_margin": 1e-5}}


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1506_06039_gb300 import synth
    oracle.build()
    wl = synth.WORKLOADS[args.workload]
    cores = os.cpu_count() or 1
    sample = max(cores, 8)
    st = synth.make_stack_np(wl.m, wl.n, sample, wl.nblobs, wl.shift_max, wl.seed, template="mean100")
    for _ in range(args.warmup):
        oracle.align(st.frames[:cores], st.template, wl.w, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.align(st.frames, st.template, wl.w, nthreads=cores)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    cfg = workload_config(wl, "oracle (exact int64 brute force)")
    cfg["sample_frames_per_step"] = sample
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "%d frames of the workload per step (host-generated, same recipe), OpenMP over frames" % sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---- the CUDA path ------------------------------------------------------------

def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "mixed":
        return run_mixed(args, world, rank, local)
    if args.workload == "refine256":
        return run_grad(args, world, rank, local)
    if args.workload == "pyramid":
        return run_pyramid(args, world, rank, local)
    if args.workload == "latency":
        return run_latency(args, world, rank, local)

    import numpy as np
    import torch
    from paper_1506_06039_gb300 import Plan, XCORR_AUTO, XCORR_DIRECT_BF16X3, XCORR_FFT_FP32, build, synth

    build.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    wl = synth.WORKLOADS[args.workload]
    if args.frames:
        import dataclasses
        wl = dataclasses.replace(wl, T=args.frames)
    st = synth.make_stack_torch(wl.m, wl.n, wl.T, wl.nblobs, wl.shift_max, rank_seed(wl.seed, rank),
                                template=wl.template)
    form = {"auto": XCORR_AUTO, "fft": XCORR_FFT_FP32, "direct": XCORR_DIRECT_BF16X3}[args.form]
    plan = Plan(dict(m=wl.m, n=wl.n, w=wl.w, xcorr=form, group_frames=args.group), st.template)
    info = plan.info()
    form_name = {XCORR_FFT_FP32: "fft_fp32", XCORR_DIRECT_BF16X3: "direct_bf16x3"}[info["xcorr"]]
    shifts = torch.empty((wl.T, 2), dtype=torch.int32, device="cuda")

    def step():
        plan_align(plan, st.frames, shifts)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    groups = math.ceil(wl.T / info["group_frames"])
    plan.profile(max_launches=args.steps * groups * 6 + 64)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
    profile = plan.profile_read(reset=True)
    plan.profile(0)
    value = job_value(world, wl.T, args.steps, ms / 1e3)
    launches = sum(l for l, _ in profile.values())
    peaks = load_peaks()
    alu = measured_alu_peaks()
    rf = roofline(profile, info, wl, wl.T, args.steps, peaks, alu)


    e2e = None
    if not args.no_e2e:
        host = torch.empty(st.frames.shape, dtype=torch.uint16).pin_memory()
        host.copy_(st.frames.cpu())
        out_h = torch.empty((wl.T, 2), dtype=torch.int32).pin_memory()
        plan.align_host(host, shifts_host=out_h)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.align_host(host, shifts_host=out_h)
        el = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
        h2d = int(wl.T * wl.m * wl.n * 2)
        # The host link's own rate: one plain pinned copy of the same bytes,
        # timed with CUDA events (the e2e ceiling when compute is hidden).
        dev = torch.empty_like(host, device="cuda")
        link_ms = []
        for _ in range(3):
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record()
            dev.copy_(host, non_blocking=True)
            l1.record()
            torch.cuda.synchronize()
            link_ms.append(l0.elapsed_time(l1))
        del dev
        link_gbs = h2d / (min(link_ms) / 1e3) / 1e9
        e2e_gbs = h2d * args.e2e_steps / el / 1e9
        e2e = {"value": job_value(world, wl.T, args.e2e_steps, el), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(wl.T * 8),
               "steps": args.e2e_steps, "api": "moco_align_host (pinned host buffers)",
               "h2d_link_gbs": link_gbs, "link_frac": e2e_gbs / link_gbs}

    correction = None
    if not args.no_correction:
        correction = measure_correction(plan, st.frames, shifts, wl, args.correction_steps, peaks, pg)

    cpu = accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        idx = np.random.default_rng(0).choice(wl.T, min(256, wl.T), replace=False)
        cpu = cpu_baseline(st.frames.cpu().numpy()[idx], st.template.cpu().numpy(), wl.w, args.cpu_seconds)
        accuracy = accuracy_sample(plan, st.frames, st.template.cpu().numpy(), wl.w, shifts)
    if rank == 0:
        tot_ms = sum(t for _, t in profile.values()) or 1.0
        cfg = workload_config(wl, form_name)
        cfg["group_frames"] = info["group_frames"]
        cfg["fft"] = [info["fft_rows"], info["fft_cols"]]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic", "config": cfg,
               "plain_form": {"form": "fft_fp32", "value": value if form_name == "fft_fp32" else None},
               "roofline": rf, "cpu_baseline": cpu, "accuracy": accuracy, "e2e": e2e, "gpu_launches": launches,
               "clocks": clocks, "correction": correction,
               "kernels": {k: {"launches": l, "ms": t, "share": t / tot_ms} for k, (l, t) in profile.items()}}
        print(json.dumps(out), flush=True)
    plan.close()
    if pg:
        pg.destroy_process_group()


def measure_correction(plan, frames, shifts, wl, steps, peaks, pg):
    """The correction step on the aligned stack (corrected frames + mean
    image), timed alone with CUDA events on the launching stream."""
    import torch
    from paper_1506_06039_gb300 import moco_apply_shifts
    corrected = torch.empty_like(frames)
    mean = torch.empty((wl.m, wl.n), dtype=torch.float64, device=frames.device)
    stream = torch.cuda.current_stream()

    def step():
        moco_apply_shifts(plan.handle, 0, frames, shifts, 100, corrected, mean, stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda") / steps
    world = pg.get_world_size() if pg else 1
    byts = 4.0 * wl.m * wl.n * wl.T  # read each frame once, write its corrected copy
    hbm = peaks.get("hbm_gbs", 6800.0)
    del corrected
    return {"metric": "frames/s corrected (corrected stack + corrected mean image)",
            "value": wl.T * world / (ms / 1e3), "unit": "frames/s", "ms_per_step": ms, "steps": steps,
            "roofline": {"bound": "hbm", "kernel": "k_apply", "achieved": byts / (ms / 1e3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": byts / (ms / 1e3) / 1e9 / hbm, "traffic": None,
                         "algorithmic_per_launch": {"bytes": byts},
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
            "api": "moco_apply_shifts (device buffers; fill 100)"}


def run_mixed(args, world, rank, local):
    """The batching form: 32 stacks of uneven size, length and window, each
    with its own template, aligned by one call replayed from a CUDA graph."""
    import numpy as np
    import torch
    from paper_1506_06039_gb300 import Plan, build, moco_align_stack, synth

    build.build()
    torch.cuda.set_device(local)
    specs = synth.mixed_batch_specs(nstacks=32)
    if args.frames:
        for s_ in specs:
            s_["T"] = min(s_["T"], args.frames)
    stacks = []
    for s_ in specs:
        st = synth.make_stack_torch(s_["m"], s_["n"], s_["T"], s_["nblobs"], s_["shift_max"],
                                    rank_seed(s_["seed"], rank), template="clean", chunk=64)
        stacks.append((st, s_["w"]))
    plan = Plan([dict(m=s_["m"], n=s_["n"], w=s_["w"]) for s_ in specs], [st.template for st, _ in stacks])
    outs = [torch.empty((st.frames.shape[0], 2), dtype=torch.int32, device="cuda") for st, _ in stacks]
    items = [dict(shape_idx=k, frames=st.frames, shifts=outs[k]) for k, (st, _) in enumerate(stacks)]
    moco_align_stack(plan.handle, items)
    torch.cuda.synchronize()
    # Per-kernel device times from profiled eager calls (untimed), summed over
    # the stacks; the timed steps are replays of one captured call.
    prof_steps = max(1, min(3, args.steps))
    plan.profile(max_launches=prof_steps * 1024)
    for _ in range(prof_steps):
        moco_align_stack(plan.handle, items)
    torch.cuda.synchronize()
    profile = plan.profile_read(reset=True)
    plan.profile(0)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            moco_align_stack(plan.handle, items, stream=cs)
    torch.cuda.current_stream().wait_stream(cs)
    for _ in range(max(3, args.warmup)):
        g.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        g.replay()
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    frames = sum(st.frames.shape[0] for st, _ in stacks)
    forms = [plan.info(k)["xcorr"] for k in range(len(specs))]
    rf, kernels = mixed_roofline(profile, plan, specs, stacks, prof_steps, load_peaks(), measured_alu_peaks())
    if rank == 0:
        out = {"metric": METRIC + " [batching form: 32 uneven stacks]", "value": world * frames * args.steps / (ms / 1e3),
               "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
               "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "fp32", "data": "synthetic",
               "config": {"workload": "mixed: 32 stacks, sizes {256,512,1024}^2, 100-3000 frames, w in {8,16,32,64}",
                          "frames": frames, "bytes": int(sum(st.frames.numel() * 2 for st, _ in stacks)),
                          "forms": {"fft_fp32": forms.count(1), "direct_bf16x3": forms.count(2)},
                          "form_by_stack": ["%dx%d w=%d: %s" % (s_["m"], s_["n"], s_["w"],
                                                                 "direct" if f_ == 2 else "fft")
                                            for s_, f_ in zip(specs, forms)],
                          "graph": "one captured moco_align_stack call"},
               "clocks": clocks, "roofline": rf, "kernels": kernels,
               "gpu_launches": sum(l for l, _ in profile.values()) // prof_steps}
        print(json.dumps(out), flush=True)
    plan.close()


def mixed_roofline(profile, plan, specs, stacks, steps, peaks, alu):
    """Per-kernel algorithmic work summed over the stacks (each with its own
    shape, window and FFT lengths) against the profiled device time; the
    dominant kernel against its bound."""
    import types
    tot = {}
    for k, (s_, (st, _)) in enumerate(zip(specs, stacks)):
        wl = types.SimpleNamespace(m=s_["m"], n=s_["n"], w=s_["w"], name="mixed")
        for name, (b, f, i) in kernel_work(plan.info(k), wl, st.frames.shape[0] * steps).items():
            acc = tot.setdefault(name, [0.0, 0.0, 0.0])
            acc[0] += b
            acc[1] += f
            acc[2] += i
    total_ms = sum(ms for _, ms in profile.values()) or 1.0
    hbm = peaks.get("hbm_gbs", 6800.0)
    kernels = {}
    for name, (launches, ms) in profile.items():
        b, f, i = tot.get(name, (0.0, 0.0, 0.0))
        sec = ms / 1e3
        kernels[name] = {"launches_per_step": launches / steps, "ms_per_step": ms / steps, "share": ms / total_ms,
                         "hbm_frac": b / sec / 1e9 / hbm if b else None,
                         "fp32_frac": f / sec / 1e12 / alu["fp32"][0] if f and name != "k_direct" else None,
                         "tensor_frac": (f / sec / 1e12 / peaks.get("bf16_tflops_sustained", 1700.0)
                                         if f and name == "k_direct" else None),
                         "int_frac": i / sec / 1e12 / alu["int"][0] if i else None}
    name = max(profile, key=lambda k: profile[k][1])
    bound = KERNEL_BOUND.get(name, "hbm")
    key = {"hbm": "hbm_frac", "fp32": "fp32_frac", "tensor": "tensor_frac"}[bound]
    rf = {"kernel": name, "bound": "alu" if bound == "fp32" else bound, "frac": kernels[name][key],
          "share": kernels[name]["share"], "traffic": None,
          "peak": {"hbm": hbm, "fp32": alu["fp32"][0], "tensor": peaks.get("bf16_tflops_sustained")}[bound],
          "unit": {"hbm": "GB/s", "fp32": "TFLOP/s", "tensor": "TFLOP/s"}[bound],
          "note": "work summed over the 32 stacks' shapes; kernel times from profiled eager calls"}
    return rf, kernels


def run_grad(args, world, rank, local):
    """The differentiable form: per step, the soft-min loss of every frame and
    its gradient with respect to a float template (set template, cost
    surface, soft-min, adjoint), all through the C ABI."""
    import torch
    from paper_1506_06039_gb300 import build, moco_set_template, moco_softmin_grad, synth
    from paper_1506_06039_gb300.autograd import softmin_plan

    build.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    wl = synth.WORKLOADS["refine256"]
    T = args.frames or wl.T
    st = synth.make_stack_torch(wl.m, wl.n, T, wl.nblobs, wl.shift_max, rank_seed(wl.seed, rank), template="clean")
    gen = torch.Generator(device="cuda").manual_seed(wl.seed)
    tmpl = st.frames.float().mean(0) + 50.0 * torch.randn((wl.m, wl.n), generator=gen, device="cuda")
    plan = softmin_plan(st.frames, tmpl, wl.w)
    W = 2 * wl.w - 1
    cost = torch.empty((T, W, W), dtype=torch.float64, device="cuda")
    loss = torch.empty(T, dtype=torch.float64, device="cuda")
    weights = torch.empty((T, W, W), dtype=torch.float32, device="cuda")
    grad = torch.zeros((wl.m, wl.n), dtype=torch.float32, device="cuda")
    def step():
        # one refinement step's device work: template in, per-frame loss and dL/db out
        stream = torch.cuda.current_stream()
        moco_set_template(plan.handle, 0, tmpl, stream)
        moco_softmin_grad(plan.handle, 0, st.frames, 0.05, cost, loss, weights, grad, 1.0, stream)
        if pg:
            # data-parallel refinement: the template gradient summed over the ranks' frames
            pg.all_reduce(grad)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # Per-kernel times from profiled eager steps (untimed) ...
    plan.profile(max_launches=args.steps * 64 + 64)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    profile = plan.profile_read(reset=True)
    plan.profile(0)
    # ... and the timed steps as replays of one captured step (the library's
    # calls allocate and synchronise nothing, so the step captures as a whole;
    # with several ranks the all-reduce stays eager).
    graph = None
    if not pg:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        if graph is not None:
            graph.replay()
        else:
            step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
    if rank == 0:
        tot = sum(t for _, t in profile.values()) or 1.0
        out = {"metric": "frames/s, soft-min loss and template gradient (differentiable form)",
               "value": job_value(world, T, args.steps, ms / 1e3), "unit": UNIT, "n_gpus": world,
               "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
               "config": {"workload": "refine256: %d frames of 256x256, w=16 (31^2 shifts), float template "
                                      "(mean frame + N(0, 50^2)), tau = 0.05 x median" % T, "frames": T,
                          "timed": ("replays of one captured step (moco_set_template + moco_softmin_grad); "
                                    "kernel times from as many profiled eager steps") if graph is not None
                          else "eager steps"},
               "gpu_launches": sum(l for l, _ in profile.values()), "clocks": clocks,
               "kernels": {k: {"launches": l, "ms": t, "share": t / tot} for k, (l, t) in profile.items()}}
        if world > 1:
            out["config"]["parallelism"] = "dp%d: frames sharded, template gradient all-reduced every step" % world
        print(json.dumps(out), flush=True)
    plan.close()
    if pg:
        pg.destroy_process_group()


def run_pyramid(args, world, rank, local):
    """Downsampling ablation: a large-motion stack (shifts up to +-120 px at
    512^2, clean template) aligned with L = 1 .. 4 levels, the window on
    level L just covering the motion; throughput and agreement with the
    planted shifts per L, and parity with the oracle on a frame sample."""
    import numpy as np
    import torch
    import oracle
    from paper_1506_06039_gb300 import Plan, XCORR_FFT_FP32, build, synth

    build.build()
    torch.cuda.set_device(local)
    m = n = 512
    T = args.frames or 1000
    motion = 120
    out_rows = {}
    for structure, sig, nblobs in (("blobs 3-6 px", (3.0, 6.0), 400), ("fine: blobs 0.7-1.5 px", (0.7, 1.5), 3000)):
        st = synth.make_stack_torch(m, n, T, nblobs, motion, rank_seed(synth.SEED_BASE + 7, rank), template="clean",
                                    sigma_range=sig)
        out_rows[structure] = ablate(st, m, n, T, motion, args.steps)
        del st
    if rank == 0:
        print(json.dumps({"metric": "downsampling ablation: frames/s and planted-shift agreement per level count",
                          "config": {"workload": "%d frames of 512x512, shifts up to +-%d px, clean template, "
                                                 "Poisson noise" % (T, motion), "steps": args.steps},
                          "structures": out_rows}), flush=True)


def ablate(st, m, n, T, motion, steps):
    import numpy as np
    import torch
    import oracle
    from paper_1506_06039_gb300 import Plan, XCORR_FFT_FP32
    planted = torch.as_tensor(np.asarray(st.shifts), device="cuda")
    rows = []
    sample = np.random.default_rng(0).choice(T, 16, replace=False)
    frames_h = np.stack([st.frames[int(k)].cpu().numpy() for k in sample])
    tmpl_h = st.template.cpu().numpy()
    for L in (1, 2, 3, 4):
        w = -(-motion // 2 ** L) + 2  # 2w - 1 covers +-motion / 2^L on level L
        plan = Plan(dict(m=m, n=n, w=w, levels=L, xcorr=XCORR_FFT_FP32), st.template)
        shifts = torch.empty((T, 2), dtype=torch.int32, device="cuda")
        for _ in range(3):
            plan_align(plan, st.frames, shifts)
        torch.cuda.synchronize()
        plan.profile(max_launches=steps * 16 + 64)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            plan_align(plan, st.frames, shifts)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        prof = plan.profile_read(reset=True)
        plan.profile(0)
        err = (shifts.long() - planted.long()).abs().max(dim=1).values
        ref = oracle.align(frames_h, tmpl_h, w, levels=L)
        rows.append({"levels": L, "w": w, "searched_grid": [m >> L, n >> L], "frames_per_s": T / (ms / 1e3),
                     "ms_per_step": ms, "planted_exact": float((err == 0).float().mean()),
                     "planted_within_1px": float((err <= 1).float().mean()),
                     "max_error_px": int(err.max()),
                     "oracle_agreement_on_sample": float(np.mean(np.all(
                         shifts.cpu().numpy()[sample] == ref["shifts"], axis=1))),
                     "kernels_ms": {k: t / steps for k, (_, t) in prof.items()}})
        plan.close()
    return rows


def run_latency(args, world, rank, local):
    """Closed-loop single-frame latency through the library's frame stream
    (moco_stream_*): each frame of the std512 stack is written to the pinned
    host frame, aligned (one graph replay: copy in, search, jitter, copy the
    shift out) and its shift read before the next frame; per-frame wall-clock
    latency percentiles."""
    import numpy as np
    import torch
    from paper_1506_06039_gb300 import FrameStream, Plan, build, synth

    build.build()
    torch.cuda.set_device(local)
    wl = synth.WORKLOADS["std512"]
    T = args.frames or 512
    st = synth.make_stack_torch(wl.m, wl.n, T, wl.nblobs, wl.shift_max, rank_seed(wl.seed, rank),
                                template=wl.template)
    host = st.frames.cpu().numpy()
    plan = Plan(dict(m=wl.m, n=wl.n, w=wl.w), st.template)
    fs = FrameStream(plan)
    fview = fs.frame.numpy()
    stream = torch.cuda.Stream()
    lat, lat_align = [], []
    out = np.empty((T, 2), np.int32)
    for rep in range(2):  # the first pass warms up
        for f in range(T):
            t0 = time.perf_counter()
            fview[...] = host[f]
            t1 = time.perf_counter()
            out[f] = fs.align(stream)
            t2 = time.perf_counter()
            if rep:
                lat.append(t2 - t0)
                lat_align.append(t2 - t1)
    fs.close()
    # device time per kernel for one frame (eager, library event pairs)
    one = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    plan.profile(max_launches=20 * 16)
    for _ in range(20):
        plan_align(plan, st.frames[:1], one)
    torch.cuda.synchronize()
    prof = plan.profile_read(reset=True)
    plan.profile(0)
    ref = torch.empty((T, 2), dtype=torch.int32, device="cuda")
    plan_align(plan, st.frames, ref)
    torch.cuda.synchronize()
    agree = float(np.mean(np.all(out == ref.cpu().numpy(), axis=1)))
    lat_us = np.array(lat) * 1e6
    plan.close()
    if rank == 0:
        print(json.dumps({"metric": "single-frame latency, closed loop (host frame in, shift out)",
                          "unit": "us", "p50": float(np.percentile(lat_us, 50)),
                          "p90": float(np.percentile(lat_us, 90)), "p99": float(np.percentile(lat_us, 99)),
                          "max": float(lat_us.max()), "frames": T,
                          "align_only_p50": float(np.percentile(np.array(lat_align) * 1e6, 50)),
                          "align_only_p99": float(np.percentile(np.array(lat_align) * 1e6, 99)),
                          "one_frame_kernel_us": {k: 1e3 * t / 20 for k, (_, t) in prof.items()},
                          "frames_per_s_closed_loop": T / (lat_us.sum() / 1e6),
                          "agreement_with_batched_path": agree,
                          "config": {"workload": "std512 frames (512x512 -> 256x256, w=32, 3x3 jitter), one at a time",
                                     "h2d_bytes_per_frame": wl.m * wl.n * 2, "d2h_bytes_per_frame": 8,
                                     "api": "moco_stream_create / moco_stream_align (one captured graph per handle)",
                                     "timed": "host copy of the frame into the pinned buffer + moco_stream_align"}}),
              flush=True)


def plan_align(plan, frames, shifts):
    from paper_1506_06039_gb300 import moco_align_stack
    moco_align_stack(plan.handle, [dict(shape_idx=0, frames=frames, shifts=shifts)])


if __name__ == "__main__":
    main()
