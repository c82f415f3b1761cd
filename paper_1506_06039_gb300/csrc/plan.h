// Plan state shared by the host-side translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"
#include "moco.h"

namespace moco {

// Optional per-kernel timing: CUDA events recorded on the launching stream
// around every kernel launch (enabled by moco_profile_enable).
enum KernelId { K_FRAME_ROWS = 0, K_ENERGY, K_COLS, K_ROWS_INV, K_JITTER, K_COPY_SHIFTS, K_SOFTMIN,
                K_BACKWARD, K_DIRECT, K_APPLY, K_JITTER_LEVEL, K_ADJ_ROWS, K_ADJ_COLS, K_ADJ_INV, K_COUNT };
extern const char* const kKernelNames[K_COUNT];

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<int, size_t>> marks;  // kernel id, index of its start event
    bool truncated = false;
    void begin(int kid, cudaStream_t st) {
        if (!on) return;
        if (used + 2 > pool.size()) { truncated = true; return; }
        cudaEventRecord(pool[used], st);
        marks.push_back({kid, used});
    }
    void end(cudaStream_t st) {
        if (!on || marks.empty() || marks.back().second != used) return;
        cudaEventRecord(pool[used + 1], st);
        used += 2;
    }
};

// Everything one shape of a plan owns. All device pointers are carved from
// the single allocation `base` (bytes long).
struct ShapePlan {
    moco_shape desc{};
    int levels = 0, mc = 0, nc = 0, w = 0, wm1 = 0, W = 0;
    int Nr = 0, Nc = 0, ncv = 0, ldx = 0;
    int form = MOCO_XCORR_FFT_FP32;
    bool has_fft = true, has_direct = false;  // which forms' buffers exist
    int ncp = 0, nqc = 0;                     // direct form: padded row length, 64-column chunks
    float tuned_ms[3] = {0, 0, 0};            // autotuner timings per form (ms per frame batch)
    bool tuned = false;                       // form fixed: template changes prepare only its tables
    int group = 1;
    int stage_frames = 1;  // frames per host staging buffer
    int num_sms = 0;       // of the plan's device
    bool f32 = false;
    double unit = 1.0;
    int64_t x_fstride = 0, y_fstride = 0;
    void* base = nullptr;
    size_t bytes = 0;
    // template-derived data
    void* tmpl = nullptr;
    int32_t* coff_i = nullptr;
    float* coff_f = nullptr;
    float2* twr = nullptr;  // 2*Nr four-step twiddles: forward order, then inverse order
    float2* twc = nullptr;  // 2*Nc, same layout
    float2* bspec = nullptr;
    double* Sb = nullptr;
    double* inv_area = nullptr;
    float2* Sb2 = nullptr;  // Sb as FP32 pairs (hi, lo), W^2
    float* ia32 = nullptr;  // unit / Area, W^2
    u64* bsq = nullptr;  // with a level: prefix table of b^2, (m+1) x (n+1)
    int32_t* tlev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // template level images 1 .. levels-1
    u64* apply_sum = nullptr;           // m x n: the correction step's per-pixel sums
    unsigned int* apply_cnt = nullptr;  // m x n: and counts
    // direct form
    float* bprime = nullptr;        // mc x nc offset template
    void* dtiles = nullptr;         // Toeplitz tiles (hi, lo)
    void* planes_hi = nullptr;      // group x mc x ncp BF16
    void* planes_lo = nullptr;
    float* hbuf = nullptr;          // group x W x W cross term
    unsigned int* dev_err = nullptr;  // set by a device-side wait that gave up
    // per-group scratch
    float2* X = nullptr;
    float2* Y = nullptr;
    u64* rowE = nullptr;
    u64* colE = nullptr;
    u64* tot = nullptr;
    uint32_t* corners = nullptr;
    u64* Sa = nullptr;
    int32_t* coarse = nullptr;
    int32_t* coarse2 = nullptr;  // levels > 1: the refinement's other buffer
    double* fbest = nullptr;
    float* margin = nullptr;
    float* grad_acc = nullptr;         // m x n (adjoint scratch)
    float* grad_Q = nullptr;           // W x W
    float2* grad_spec = nullptr;       // ncv x Nr (FFT form): sum_f A_f conj(Q_f) of the adjoint
    u64* jit_acc = nullptr;            // group x 9
    unsigned int* jit_ticket = nullptr;  // group
    // staging for moco_align_host (double-buffered)
    uint16_t* stage[2] = {nullptr, nullptr};
    int32_t* stage_shifts[2] = {nullptr, nullptr};
    Profiler* prof = nullptr;  // the owning plan's profiler
};

constexpr int64_t kMultiJitFrames = 32768;  // frames per launch of the several-stack refinement

struct DeviceGuard {
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    int prev_ = 0;
};

moco_status fail(moco_status s, const std::string& msg);
moco_status cuda_fail(cudaError_t e, const char* what);

}  // namespace moco

struct moco_plan_s {
    int device = 0;
    std::vector<moco::ShapePlan> shapes;
    cudaStream_t aux = nullptr;  // host staging copies (moco_align_host)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    moco::Profiler prof;
    void* scratch = nullptr;  // per-batch scratch shared by all shapes
    size_t scratch_bytes = 0;
    // the several-stack refinement (moco_align_stack): kMultiJitFrames frames per launch
    void* mj_base = nullptr;
    moco::u64* mj_acc = nullptr;
    unsigned int* mj_ticket = nullptr;
    int num_sms = 0;
};
