// Row passes: k_frame_rows (forward) and k_rows_inv (inverse + combine + argmin).
#include "fft_sizes.h"
#include "internal.h"
#include "kernels.cuh"

namespace moco {

// Staging the chunk's frame rows in shared memory: two CTAs per SM up to
// 112 KiB each (228 KiB, 1 KiB reserved per CTA); wider frames (1024
// columns: 128 KiB of staged rows per chunk) run one staged CTA per SM,
// which still hides the copies that the unstaged loader waits for.
constexpr size_t kStagedSmemMax = 227 * 1024;

template <int N, bool F32>
static cudaError_t frame_rows_n(const void* src, int64_t src_fstride, int64_t nimg, int m, int n, int levels,
                                int mc, int nc, const int32_t* coff_i, const float* coff_f, const float2* tw,
                                float2* X, int64_t x_fstride, int ldx, u64* rowE, u64* colE, u64* tot,
                                uint32_t* corners, int wm1, unsigned int* err, int64_t capacity, cudaStream_t st) {
    const size_t smem = sizeof(float2) * ((kRC / 2) * fft_ld<N>() + N) + sizeof(u64) * (kRC + nc);
    const size_t smem_staged = frame_rows_smem_base<N, F32>(nc) + frame_rows_stage_bytes(n, levels);
    // A single image (the template, a closed-loop frame) is split over one CTA
    // per chunk of rows when the buffers have a slot per chunk for the partial
    // sums, which k_merge_chunks then adds up.
    const int chunks = (mc + kRC - 1) / kRC;
    const int split = (nimg == 1 && chunks > 1 && chunks <= capacity) ? 1 : 0;
    const unsigned grid = split ? (unsigned)chunks : (unsigned)nimg;
    cudaError_t e;
    // (the staged loader gives each searched column its own thread)
    if (!F32 && n % 8 == 0 && levels <= 1 && nc <= kRowsThreads && smem_staged <= kStagedSmemMax) {
        const void* fn = (const void*)k_frame_rows<N, false, false, true>;
        if ((e = ensure_smem(fn, smem_staged)) != cudaSuccess) return e;
        k_frame_rows<N, false, false, true><<<grid, kRowsThreads, smem_staged, st>>>(
            src, src_fstride, m, n, levels, mc, nc, coff_i, coff_f, tw, X, x_fstride, ldx, rowE, colE, tot, corners,
            wm1, nullptr, nullptr, 0, err, split);
    } else {
        const void* fn = (const void*)k_frame_rows<N, F32>;
        if ((e = ensure_smem(fn, smem)) != cudaSuccess) return e;
        k_frame_rows<N, F32><<<grid, kRowsThreads, smem, st>>>(src, src_fstride, m, n, levels, mc, nc, coff_i, coff_f,
                                                              tw, X, x_fstride, ldx, rowE, colE, tot, corners, wm1,
                                                              nullptr, nullptr, 0, nullptr, split);
    }
    if ((e = cudaGetLastError()) != cudaSuccess || !split) return e;
    k_merge_chunks<F32><<<1, 256, 0, st>>>(colE, tot, chunks, nc, wm1);
    return cudaGetLastError();
}

cudaError_t launch_frame_rows(int N, bool f32, const void* src, int64_t src_fstride, int64_t nimg, int m,
                              int n, int levels, int mc, int nc, const int32_t* coff_i, const float* coff_f,
                              const float2* tw, float2* X, int64_t x_fstride, int ldx, u64* rowE, u64* colE,
                              u64* tot, uint32_t* corners, int wm1, unsigned int* err, int64_t capacity,
                              cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
#define MOCO_CASE(NN)                                                                                        \
    case NN:                                                                                                 \
        return f32 ? frame_rows_n<NN, true>(src, src_fstride, nimg, m, n, levels, mc, nc, coff_i, coff_f,    \
                                            tw, X, x_fstride, ldx, rowE, colE, tot, corners, wm1, err,       \
                                            capacity, st)                                                    \
                   : frame_rows_n<NN, false>(src, src_fstride, nimg, m, n, levels, mc, nc, coff_i,           \
                                             coff_f, tw, X, x_fstride, ldx, rowE, colE, tot, corners, wm1,   \
                                             err, capacity, st);
    switch (N) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

template <int N>
static cudaError_t rows_inv_n(const float2* Y, int64_t y_fstride, int ncv, int wm1, int64_t nimg,
                              const float2* tw, const u64* rowE, const u64* colE, const u64* tot,
                              const uint32_t* corners, int mc, int nc, const float2* Sb2, const float* ia32,
                              double* cost, int32_t* coarse, double* fbest, float* margin,
                              cudaStream_t st) {
    const size_t smem = rows_inv_smem<N>(wm1);
    const void* fn = (const void*)k_rows_inv<N>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const int threads = rows_inv_threads<N>();  // at least four warps (one per corner quadrant)
    k_rows_inv<N><<<(unsigned)nimg, threads, smem, st>>>(Y, y_fstride, ncv, wm1, tw, rowE, colE, tot, corners, mc,
                                                         nc, Sb2, ia32, cost, coarse, fbest, margin);
    return cudaGetLastError();
}

size_t rows_inv_smem_bytes(int N, int wm1) {
#define MOCO_CASE(NN) \
    case NN: return rows_inv_smem<NN>(wm1);
    switch (N) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default: return ~(size_t)0;
    }
#undef MOCO_CASE
}

cudaError_t launch_rows_inv(int N, const float2* Y, int64_t y_fstride, int ncv, int wm1, int64_t nimg,
                            const float2* tw, const u64* rowE, const u64* colE, const u64* tot,
                            const uint32_t* corners, int mc, int nc, const float2* Sb2, const float* ia32,
                            double* cost, int32_t* coarse, double* fbest, float* margin, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
#define MOCO_CASE(NN) \
    case NN:          \
        return rows_inv_n<NN>(Y, y_fstride, ncv, wm1, nimg, tw, rowE, colE, tot, corners, mc, nc, Sb2, ia32, cost, \
                              coarse, fbest, margin, st);
    switch (N) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

}  // namespace moco
