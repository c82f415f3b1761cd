// Column pass: k_cols (forward column FFT, template product, inverse kept on
// the window rows) and its spectrum-only form for template preparation.
#include "fft_sizes.h"
#include "internal.h"
#include "kernels.cuh"

namespace moco {

template <int N>
static cudaError_t cols_n(bool spectrum, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv,
                          int64_t nimg, const float2* tw, const float2* bspec, float2* Y, int64_t y_fstride,
                          int wm1, float scale, cudaStream_t st) {
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
                        int wm1, float scale, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
#define MOCO_CASE(NN) \
    case NN:          \
        return cols_n<NN>(spectrum, X, x_fstride, ldx, mc, ncv, nimg, tw, bspec, Y, y_fstride, wm1, scale, st);
    switch (N) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

}  // namespace moco
