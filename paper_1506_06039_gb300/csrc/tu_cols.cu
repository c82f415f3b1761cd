// Column pass: k_cols (forward column FFT, template product, inverse kept on
// the window rows) and its spectrum-only form for template preparation.
#include <algorithm>

#include "fft_sizes.h"
#include "internal.h"
#include "kernels.cuh"

namespace moco {

// The streaming form whenever one of its CTAs fits on an SM (two fit up to
// N = 288 at 256 searched rows; longer transforms run one per SM, still
// hiding each frame's copy under the previous frame's transforms).
constexpr size_t kColsStreamSmemMax = 227 * 1024;

// Frame slices of one resident wave of the streaming form (0 when it does
// not apply): every CTA then walks about T / slices frames.
template <int N>
static cudaError_t cols_stream_slices(int ldx, int ncv, int* slices) {
    *slices = 0;
    const size_t smem = cols_stream_smem<N>(ldx);
    if (smem > kColsStreamSmemMax) return cudaSuccess;
    const void* fn = (const void*)k_cols_stream<N>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cols_threads<N>(), smem)) != cudaSuccess)
        return e;
    *slices = std::max(1, std::max(1, per_sm) * sms / ((ncv + kColsVC - 1) / kColsVC));
    return cudaSuccess;
}

template <int N>
static cudaError_t cols_n(bool spectrum, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv,
                          int64_t nimg, const float2* tw, const float2* bspec, float2* Y, int64_t y_fstride,
                          int wm1, float scale, unsigned int* err, cudaStream_t st) {
    if (!spectrum) {
        // The streaming form pays off once each of its CTAs walks several frames.
        int slices = 0;
        cudaError_t e = cols_stream_slices<N>(ldx, ncv, &slices);
        if (e != cudaSuccess) return e;
        if (slices > 0 && nimg >= 4 * (int64_t)slices) {
            const dim3 grid((unsigned)((ncv + kColsVC - 1) / kColsVC), (unsigned)slices);
            k_cols_stream<N><<<grid, cols_threads<N>(), cols_stream_smem<N>(ldx), st>>>(
                X, x_fstride, ldx, mc, ncv, nimg, tw, bspec, Y, y_fstride, wm1, err);
            return cudaGetLastError();
        }
    }
    const size_t smem = sizeof(float2) * (kColsVC * fft_ld<N>() + 2 * N);
    const void* fn = spectrum ? (const void*)k_cols<N, true> : (const void*)k_cols<N, false>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const int threads = cols_threads<N>();
    dim3 grid((unsigned)nimg, (unsigned)((ncv + kColsVC - 1) / kColsVC));
    if (spectrum)
        k_cols<N, true><<<grid, threads, smem, st>>>(X, x_fstride, ldx, mc, ncv, tw, bspec, Y, y_fstride, wm1, scale);
    else
        k_cols<N, false><<<grid, threads, smem, st>>>(X, x_fstride, ldx, mc, ncv, tw, bspec, Y, y_fstride, wm1, scale);
    return cudaGetLastError();
}

cudaError_t launch_cols(int N, bool spectrum, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv,
                        int64_t nimg, const float2* tw, const float2* bspec, float2* Y, int64_t y_fstride,
                        int wm1, float scale, unsigned int* err, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
#define MOCO_CASE(NN) \
    case NN:          \
        return cols_n<NN>(spectrum, X, x_fstride, ldx, mc, ncv, nimg, tw, bspec, Y, y_fstride, wm1, scale, err, st);
    switch (N) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

}  // namespace moco
