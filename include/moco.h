/*
 * moco GB300 engine: the C ABI.
 *
 * The operation is the translation search of "moco: Fast Motion Correction
 * for Calcium Imaging" (Dubbs, Guevara, Peterka, Yuste; arXiv 1506.06039),
 * Section 2: for every frame a of a stack and a template b, pick the integer
 * shift (s, t), max(|s|, |t|) < w, that minimises
 *
 *     f_{s,t} = 1/Area(D_{s,t}) * sum_{(i,j) in D_{s,t}} (a[i+s][j+t] - b[i][j])^2,
 *     D_{s,t} = {(i,j): 0 <= i < m, 0 <= j < n, 0 <= i+s < m, 0 <= j+t < n}
 *
 * (written 0-based). Images larger than 256x256 are searched once on a 2x2
 * box-downsampled grid (Sections 2 and 3), then the doubled optimum is
 * refined by the 3x3 local search at full resolution (Section 2's
 * upsampling step). A frame whose content moved by +(s0, t0) relative to the
 * template, frame[i][j] = b[i-s0][j-t0], returns (s0, t0).
 *
 * Conventions shared by every entry point:
 *  - Images are row-major, 0-based. Frames are uint16 [T][m][n], contiguous,
 *    16-byte aligned, n a multiple of 8.
 *  - Pointers named *_dev are caller-owned device memory on the plan's
 *    device; *_host are caller-owned host memory (pinned for overlap).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Every call below except moco_plan, moco_set_template,
 *    moco_align_host and moco_plan_destroy is asynchronous on that stream,
 *    allocates nothing and never synchronises.
 *  - A plan is not thread-safe: its workspace is shared by all calls, so
 *    calls on one plan must be ordered on one stream (or otherwise
 *    serialised). Different plans are independent.
 *  - Errors are reported by the return value only; nothing is thrown across
 *    the ABI. Invalid arguments are rejected before any launch.
 *  - Shift (s, t) cost surfaces are laid out [T][2w-1][2w-1], entry
 *    (s+w-1, t+w-1), in FP64, in box-mean units on the searched grid (the
 *    exact 4-sum cost divided by 16 when one 2x2 level is used).
 *  - Ties (the paper does not say): smallest f, then smallest |s|+|t|, then
 *    smallest s, then smallest t.
 */
#ifndef MOCO_H_
#define MOCO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOCO_OK = 0,
    MOCO_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad alignment, bad index */
    MOCO_ERR_UNSUPPORTED = 2, /* a shape this build cannot run (reported by moco_plan) */
    MOCO_ERR_OOM = 3,         /* device allocation failed in moco_plan */
    MOCO_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    MOCO_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} moco_status;

/* How the cross term h_{s,t} = sum_D a[i+s][j+t] b[i][j] is computed. */
typedef enum {
    MOCO_XCORR_AUTO = 0,          /* measured by the plan's autotuner */
    MOCO_XCORR_FFT_FP32 = 1,      /* zero-padded 2-D FFTs in FP32 (Section 2) */
    MOCO_XCORR_DIRECT_BF16X3 = 2  /* direct contraction on tensor cores, BF16 hi+lo */
} moco_xcorr;

typedef enum {
    MOCO_TEMPLATE_U16 = 0, /* uint16 template: exact integer energies */
    MOCO_TEMPLATE_F32 = 1  /* float template (differentiable form; levels must be 0) */
} moco_template_dtype;

/* One image shape a plan serves. */
typedef struct {
    int32_t m, n;           /* full-resolution rows and columns (n % 8 == 0, n <= 4096) */
    int32_t w;              /* window on the searched grid: max(|s|,|t|) < w, 2w-1 <= min(mc, nc) */
    int32_t levels;         /* -1: the paper's rule (1 if m > 256 or n > 256, else 0); or 0 .. 4:
                               the search runs on level L (2^L x 2^L box sums), then each
                               finer level refines the doubled optimum by a 3x3 search with
                               exact sums (Section 2, "multiplied by two multiple times");
                               L >= 2 uses the FFT form only */
    int32_t template_dtype; /* moco_template_dtype */
    int32_t xcorr;          /* moco_xcorr */
    int32_t group_frames;   /* frames per internal batch (workspace size); 0 = chosen by the plan */
    int32_t reserved;       /* must be 0 */
} moco_shape;

/* What the plan resolved for one shape (moco_plan_query). */
typedef struct {
    int32_t levels, mc, nc;  /* levels used and the searched-grid size */
    int32_t fft_rows;        /* FFT length along image rows (>= mc + w - 1) */
    int32_t fft_cols;        /* FFT length along image columns (>= nc + w - 1) */
    int32_t xcorr;           /* the form in use (never AUTO) */
    int32_t group_frames;    /* frames per internal batch */
    int32_t offset;          /* integer offset c subtracted from frame and template */
    int64_t workspace_bytes; /* device bytes of this shape's tables plus the plan's shared batch scratch */
} moco_shape_info;

typedef struct moco_plan_s* moco_plan_t;

/* One stack for moco_align_stack. */
typedef struct {
    int32_t shape_idx;      /* index into the plan's shapes */
    int32_t reserved;       /* must be 0 */
    const uint16_t* frames_dev; /* [T][m][n] */
    int64_t T;              /* number of frames (0 is allowed: nothing is launched) */
    int32_t* shifts_dev;    /* out [T][2]: final (s, t) per frame */
    double* best_cost_dev;  /* out, nullable [T]: f at the searched-grid optimum (box-mean units) */
    float* margin_dev;      /* out, nullable [T]: (f2 - f1) / f1 on the searched grid; f2 = next smallest f */
    double* final_cost_dev; /* out, nullable [T]: f at the final shift. With a level: S / Area(D) at full
                               resolution from the exact integer sum S, in FP64 (the upsampling step of
                               Section 2); without: equal to best_cost */
} moco_stack;

/* Creates a plan for `nshapes` shapes (Section 2's problem statement: the
 * template b and the user's window w per shape). templates_dev[k] points to
 * shape k's template, uint16 or float [m][n] per template_dtype; it is copied
 * into the plan. Allocates all workspace, prepares the template (offset,
 * energies, spectrum) on `stream`, resolves MOCO_XCORR_AUTO by timing both
 * forms, and synchronises `stream` before returning. On success *out holds
 * the plan; on failure *out is NULL and nothing is leaked. */
moco_status moco_plan(const moco_shape* shapes, int32_t nshapes, const void* const* templates_dev,
                      void* stream, moco_plan_t* out);

/* Replaces shape `shape_idx`'s template (same dtype and size) and recomputes
 * what depends on it, on `stream` (no allocation, no synchronisation). */
moco_status moco_set_template(moco_plan_t plan, int32_t shape_idx, const void* template_dev, void* stream);

/* Aligns every frame of every stack (Section 2: exhaustive search over the
 * window on the searched grid, then, when a level is used, the 3x3 jitter
 * at full resolution). Stacks may use different shapes of the plan. */
moco_status moco_align_stack(moco_plan_t plan, const moco_stack* stacks, int32_t nstacks, void* stream);

/* The searched-grid cost surface f_{s,t} of T frames, FP64 [T][2w-1][2w-1]
 * (Section 2's f, box-mean units). */
moco_status moco_cost_surface(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              double* cost_dev, void* stream);

/* Soft-min over shifts of each frame's cost surface (not in the paper; the
 * differentiable form): tau_f = tau_scale * median_{s,t} f (the exact middle
 * of the (2w-1)^2 values), L_f = -tau_f log sum_{s,t} exp(-f_{s,t} / tau_f).
 * Writes loss_dev[T] and weights_dev[T][2w-1][2w-1] = dL_f / df_{s,t}
 * (the softmax weights; tau held constant). cost_dev from moco_cost_surface. */
moco_status moco_softmin(moco_plan_t plan, int32_t shape_idx, const double* cost_dev, int64_t T,
                         double tau_scale, double* loss_dev, float* weights_dev, void* stream);

/* Adjoint of Section 2's f (not in the paper; the differentiable form), for
 * shapes with levels == 0: given G = grad_scale * grad_cost_dev
 * ([T][2w-1][2w-1] floats, dL/df_{s,t}), accumulates
 *   grad_template_dev[m][n] += dL/db  (float; the caller zeroes it first)
 * and, if grad_frames_dev is non-null, overwrites grad_frames_dev[T][m][n]
 * with dL/da. Uses the plan's current template. The template side's
 * correlation runs through FFTs on FFT-form plans (one inverse transform of
 * the sum over frames) and as a direct FP32 contraction otherwise; both sum
 * with FP32 atomics, so the last bits vary from run to run.
 * MOCO_ERR_UNSUPPORTED when levels != 0 or the window needs more shared
 * memory than a CTA has (w > 56). */
moco_status moco_cost_backward(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                               const float* grad_cost_dev, float grad_scale, float* grad_template_dev,
                               float* grad_frames_dev, void* stream);

/* The differentiable form's forward pass and template adjoint in one call
 * (shapes with levels == 0): the cost surface (as moco_cost_surface) into
 * cost_dev [T][2w-1][2w-1] FP64, the soft-min (as moco_softmin) into
 * loss_dev [T] and weights_dev [T][2w-1][2w-1], and
 *   grad_template_dev[m][n] += grad_scale * d(sum_f L_f)/db
 * (as moco_cost_backward with grad_cost = the weights). On FFT-form plans
 * each batch's row spectra serve both the search and the adjoint (computed
 * once); otherwise the three steps run one after another. All pointers are
 * caller-owned device memory; no allocation, no synchronisation. */
moco_status moco_softmin_grad(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              double tau_scale, float grad_scale, double* cost_dev, double* loss_dev,
                              float* weights_dev, float* grad_template_dev, void* stream);

/* End-to-end alignment from host memory: copies frames_host [T][m][n] to the
 * device in batches, aligns them and copies shifts [T][2] back to
 * shifts_host, overlapping copies with compute on `stream` and a second
 * internal stream. Returns after the last shift has landed in host memory. */
moco_status moco_align_host(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_host, int64_t T,
                            int32_t* shifts_host, void* stream);

/* Synchronises the plan's device and reports whether any bounded device-side
 * wait of the plan's kernels gave up since the last check (MOCO_ERR_TIMEOUT,
 * flag then cleared); MOCO_OK otherwise. */
moco_status moco_plan_status(moco_plan_t plan);

/* Check of the timeout path: launches on `stream` one CTA whose bounded
 * mbarrier wait (the same wait the staged kernels use) is never satisfied; it
 * gives up after about a second, records the timeout in shape shape_idx's
 * device status word and returns, with no copy in flight. The next
 * moco_plan_status then reports MOCO_ERR_TIMEOUT and clears the word; the
 * plan and the CUDA context stay usable. Asynchronous; no allocation. */
moco_status moco_selftest_wait(moco_plan_t plan, int32_t shape_idx, void* stream);

/* Measured arithmetic peaks (instrumentation; the paper has no counterpart):
 * the rate at which this device issues the operation the search's
 * compute-bound kernels are limited by, for roofline fractions against a
 * measured rather than a nominal number.
 *   MOCO_PEAK_FP32_FMA: FP32 fused multiply-adds; *ops_per_s in flop/s
 *     (2 per instruction). Bounds the FFT form's transforms.
 *   MOCO_PEAK_DP2A: 32-bit integer dot products (dp2a: two 16-bit values
 *     times two bytes plus an accumulator); *ops_per_s in instructions/s.
 *     Bounds the exact full-resolution sums of the upsampling step.
 * One resident wave of CTAs on every SM runs 16 independent chains per
 * thread for about 20 ms (best of three launches, CUDA events on `stream`,
 * after one warm-up launch). sink_dev: 4 bytes of caller-owned device
 * memory the kernels may write (the results never reach it in practice).
 * Synchronises `stream`; allocates nothing on the device. */
typedef enum { MOCO_PEAK_FP32_FMA = 0, MOCO_PEAK_DP2A = 1 } moco_peak_kind;
moco_status moco_alu_peak(int32_t kind, uint32_t* sink_dev, double* ops_per_s, void* stream);

/* The correction step: applies each frame's shift (Section 2: the found
 * shifts "motion correct" the video; the paper gives no formula, this is the
 * library's definition). For frames_dev [T][m][n] uint16 (shape shape_idx,
 * n % 8 == 0, 16-byte aligned) and shifts_dev [T][2] int32 (s, t) as
 * returned by moco_align_stack (any values; a shift past the frame leaves no
 * source pixel):
 *   corrected_dev [T][m][n] uint16 (nullable, 16-byte aligned):
 *       corrected[f][i][j] = frames[f][i + s_f][j + t_f] where 0 <= i + s_f < m
 *       and 0 <= j + t_f < n, else fill;
 *   mean_dev [m][n] double (nullable): per pixel, the sum of the in-frame
 *       source pixels over all frames divided by their count, from the exact
 *       integer sum in FP64; fill where no frame covers the pixel (all of the
 *       image when T == 0).
 * Enqueued on `stream`; no allocation (the sums live in the plan), no
 * synchronisation. Two calls on one shape must not overlap on the GPU when
 * both ask for the mean (they share the plan's sums). */
moco_status moco_apply_shifts(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              const int32_t* shifts_dev, uint16_t fill, uint16_t* corrected_dev, double* mean_dev,
                              void* stream);

/* The closed-loop single-frame mode (Section 1: real-time, closed-loop
 * experiments): a handle that aligns one frame at a time from host memory.
 * moco_stream_create registers frame_host (m x n uint16 of shape shape_idx)
 * and shift_host (2 int32); both should be page-locked (cudaHostAlloc) for
 * the shortest copies, and must stay valid until the handle is destroyed.
 * It allocates one frame and one shift on the device and captures, once,
 * the copy of frame_host to the device, the plan's alignment of that frame
 * (moco_align_stack with T = 1) and the copy of the shift to shift_host into
 * a CUDA graph (running the step once eagerly first).
 * moco_stream_align replays that graph on `stream` and waits for it: on
 * return shift_host holds (s, t) of the frame that was in frame_host, which
 * the caller may then overwrite with the next frame. The handle shares the
 * plan's batch scratch: it must not run concurrently with other calls on the
 * same plan. The plan must outlive the handle. */
typedef struct moco_stream_s* moco_stream_t;
moco_status moco_stream_create(moco_plan_t plan, int32_t shape_idx, const uint16_t* frame_host, int32_t* shift_host,
                               moco_stream_t* out);
moco_status moco_stream_align(moco_stream_t handle, void* stream);
moco_status moco_stream_destroy(moco_stream_t handle);

/* The full-resolution 3x3 refinement on its own, allocating nothing (the
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc, such as code inside a host application that owns all device
 * memory, or a real-time loop that must never block in the allocator).
 * frames_dev [T][m][n] and template_dev [m][n] are uint16, 16-byte aligned,
 * n % 8 == 0; coarse_dev [T][2] holds each frame's optimum (s_c, t_c) on the
 * 2x2-box grid; shifts_dev [T][2] receives the best of (2 s_c + u, 2 t_c + v),
 * u, v in {-1, 0, 1}, by exact integer sums and the same tie-break as
 * moco_align_stack. Every candidate needs a non-empty overlap with the
 * frame, |2 s_c| + 1 < m and |2 t_c| + 1 < n (a searched-grid optimum always
 * has it); a frame whose coarse shift breaks that gets (INT32_MIN, INT32_MIN)
 * in shifts_dev (checked on the device: the call itself still returns MOCO_OK).
 * Its scratch is one static device array sized for at most 8192 frames per
 * call (608 KiB, held by every GPU that loads this library until the process
 * exits); larger T returns MOCO_ERR_INVALID_ARG. Every call looks the array's
 * address up in the current context (cudaGetSymbolAddress); the first call on
 * a device also loads the library's device code there and should come before
 * any stream capture. Every call shares the array and clears the part it
 * uses first, on `stream`; calls that overlap on the GPU (different streams,
 * or different host threads on one device) race on it. */
moco_status moco_jitter_noalloc(const uint16_t* frames_dev, int64_t T, int32_t m, int32_t n,
                                const uint16_t* template_dev, const int32_t* coarse_dev, int32_t* shifts_dev,
                                void* stream);

/* Fills *info for shape `shape_idx`. */
moco_status moco_plan_query(moco_plan_t plan, int32_t shape_idx, moco_shape_info* info);

/* Frees everything the plan owns (synchronises the plan's device first). */
moco_status moco_plan_destroy(moco_plan_t plan);

/* Per-kernel timing (instrumentation; the paper has no counterpart). */
typedef struct {
    char name[32];     /* kernel name, e.g. "k_cols" */
    int64_t launches;  /* launches recorded since the last reset */
    double total_ms;   /* summed device time of those launches (CUDA events) */
} moco_kernel_stat;

/* Enables (max_launches > 0) or disables (0) per-kernel timing on the plan:
 * every later launch is bracketed by two CUDA events recorded on its stream,
 * up to max_launches launches. Allocates the event pool here (not in the
 * timed calls); synchronises the plan's device. */
moco_status moco_profile_enable(moco_plan_t plan, int32_t max_launches);

/* Synchronises the plan's device and reports up to `capacity` kernels that
 * were launched since the last reset (*count receives how many); reset != 0
 * clears the record. Returns MOCO_ERR_INVALID_ARG if profiling is off. */
moco_status moco_profile_read(moco_plan_t plan, moco_kernel_stat* stats, int32_t capacity, int32_t* count,
                              int32_t reset);

/* A static, human-readable name for a status. */
const char* moco_status_string(moco_status status);

/* Text of the last error recorded by a call in this thread ("" if none). */
const char* moco_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MOCO_H_ */
