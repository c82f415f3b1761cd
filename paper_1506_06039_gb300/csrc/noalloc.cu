// moco_jitter_noalloc: the full-resolution 3x3 refinement without any
// allocation, for callers that cannot call cudaMalloc (for example code
// running inside a host framework that owns all device memory and forbids
// allocation after start-up, or a real-time loop that must not block in the
// allocator). Its scratch (nine exact sums and one ticket per frame) lives
// in a file-scope device array that every GPU which loads this library
// keeps until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "kernels.cuh"
#include "moco.h"

namespace moco {

moco_status fail(moco_status s, const std::string& msg);
moco_status cuda_fail(cudaError_t e, const char* what);

namespace {

constexpr int64_t kNoallocMaxFrames = 8192;
// Per frame: 9 u64 sums, then (after all sums) one 32-bit ticket:
// 8192 * (9 * 8 + 4) bytes = 608 KiB.
constexpr int64_t kNoallocWords = kNoallocMaxFrames * 9 + kNoallocMaxFrames / 2;
static_assert(kNoallocWords * 8 == 608 * 1024, "the size stated in include/moco.h");
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocWords];

// Device address of the scratch array in the current context. Looked up on
// every call (a host-side table lookup once the module is loaded): a cached
// address would go stale if the caller reset the device or tore down its
// primary context, after which the module loads again, possibly elsewhere.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace moco

using namespace moco;

extern "C" moco_status moco_jitter_noalloc(const uint16_t* frames_dev, int64_t T, int32_t m, int32_t n,
                                           const uint16_t* template_dev, const int32_t* coarse_dev,
                                           int32_t* shifts_dev, void* stream) {
    if (T < 0) return fail(MOCO_ERR_INVALID_ARG, "T < 0");
    if (T > kNoallocMaxFrames)
        return fail(MOCO_ERR_INVALID_ARG, "T exceeds the " + std::to_string(kNoallocMaxFrames) +
                                              " frames the static scratch of moco_jitter_noalloc holds");
    if (m < 2 || n < 8 || n % 8 != 0 || m > 4096 || n > 4096)
        return fail(MOCO_ERR_INVALID_ARG, "need 2 <= m <= 4096, 8 <= n <= 4096 and n % 8 == 0");
    if (T == 0) return MOCO_OK;
    if (!frames_dev || !template_dev || !coarse_dev || !shifts_dev)
        return fail(MOCO_ERR_INVALID_ARG, "null frames, template, coarse or shifts");
    if ((reinterpret_cast<uintptr_t>(frames_dev) & 15) || (reinterpret_cast<uintptr_t>(template_dev) & 15))
        return fail(MOCO_ERR_INVALID_ARG, "frames and template must be 16-byte aligned");
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    u64* acc = static_cast<u64*>(base);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(acc + 9 * kNoallocMaxFrames);
    // launch_jitter clears the T frames' sums and tickets before the kernel.
    // No template table without a plan: the kernel sums b^2 itself.
    e = launch_jitter(frames_dev, (int64_t)m * n, T, template_dev, m, n, nullptr, coarse_dev, shifts_dev, nullptr, acc,
                      ticket, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "moco_jitter_noalloc");
    return MOCO_OK;
}
