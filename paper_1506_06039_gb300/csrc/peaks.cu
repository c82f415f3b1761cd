// moco_alu_peak: the measured issue rate of the two arithmetic pipes the
// search's kernels are bound by (instrumentation; the paper has no
// counterpart). FP32 fused multiply-adds bound the transforms of the FFT
// form; the 16 x 8-bit integer dot product (dp2a) bounds the exact
// full-resolution sums of the upsampling step. Each thread runs kChains
// independent dependency chains so that the pipe, not the latency of one
// chain, sets the rate; one resident wave of CTAs covers every SM.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "moco.h"

namespace moco {

moco_status fail(moco_status s, const std::string& msg);
moco_status cuda_fail(cudaError_t e, const char* what);

namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;

// KIND 0: x = x * a + b in FP32 (2 flop per instruction).
// KIND 1: acc = dp2a.lo(x, y) + acc (one 32-bit integer dot product).
// The result reaches memory only when it equals a value the chains never
// produce in practice, which the compiler cannot know: the work stays.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_alu_peak(int iters, uint32_t seed, uint32_t* __restrict__ sink) {
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (KIND == 0) {
        float x[kChains];
        const float a = 0.999999f + 1e-9f * (float)(seed & 7u), b = 1e-7f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = (float)((id + k) & 63u);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += x[k];
        if (__float_as_uint(s) == seed) sink[0] = id;
    } else {
        uint32_t acc[kChains];
        const uint32_t xs = 0x00030001u * (seed | 1u);
        const uint32_t ys = 0x01020304u ^ seed;
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = id * 7u + (uint32_t)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = __dp2a_lo(xs + (uint32_t)k, ys, acc[k]);
        }
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s ^= acc[k];
        if (s == seed) sink[0] = id;
    }
}

}  // namespace
}  // namespace moco

using namespace moco;

// Declared in include/moco.h.
extern "C" moco_status moco_alu_peak(int32_t kind, uint32_t* sink_dev, double* ops_per_s, void* stream) {
    if (kind != MOCO_PEAK_FP32_FMA && kind != MOCO_PEAK_DP2A) return fail(MOCO_ERR_INVALID_ARG, "bad kind");
    if (!sink_dev || !ops_per_s) return fail(MOCO_ERR_INVALID_ARG, "null sink or result");
    if (reinterpret_cast<uintptr_t>(sink_dev) & 3) return fail(MOCO_ERR_INVALID_ARG, "sink must be 4-byte aligned");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ctas = sms * kPeakCtasPerSm;
    // About 20 ms per timed launch at this part's rates (~40 T FMA/s, ~20 T dp2a/s).
    const int iters = kind == MOCO_PEAK_FP32_FMA ? 1 << 18 : 1 << 17;
    auto launch = [&](int it) {
        if (kind == MOCO_PEAK_FP32_FMA) k_alu_peak<0><<<ctas, kPeakThreads, 0, st>>>(it, 0x3f800001u, sink_dev);
        else k_alu_peak<1><<<ctas, kPeakThreads, 0, st>>>(it, 0x7fffffffu, sink_dev);
        return cudaGetLastError();
    };
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch(iters / 8);  // warm-up (clocks up, code loaded)
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = launch(iters);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "moco_alu_peak");
    const double instr = (double)ctas * kPeakThreads * (double)iters * kChains;
    *ops_per_s = instr * (kind == MOCO_PEAK_FP32_FMA ? 2.0 : 1.0) / (best * 1e-3);
    return MOCO_OK;
}
