// Internal launchers shared by the translation units of the engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace moco {

typedef unsigned long long u64;

// FFT lengths this build instantiates (each a product N1 * N2 of register
// codelet sizes); fft_size_for returns the smallest one >= needed, or 0.
int fft_size_for(int needed);
bool fft_size_supported(int N);
bool fft_split(int N, int* n1, int* n2);  // the four-step factors N = N1 * N2
int fft_split_max(int N);  // max(N1, N2): threads per row of a four-step stage

// capacity: image slots in colE and tot (a single image is split over chunk
// CTAs when it covers their count).
cudaError_t launch_frame_rows(int N, bool f32, const void* src, int64_t src_fstride, int64_t nimg, int m,
                              int n, int levels, int mc, int nc, const int32_t* coff_i, const float* coff_f,
                              const float2* tw, float2* X, int64_t x_fstride, int ldx, u64* rowE, u64* colE,
                              u64* tot, uint32_t* corners, int wm1, unsigned int* err, int64_t capacity,
                              cudaStream_t st);

cudaError_t launch_cols(int N, bool spectrum, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv,
                        int64_t nimg, const float2* tw, const float2* bspec, float2* Y, int64_t y_fstride,
                        int wm1, float scale, unsigned int* err, cudaStream_t st);

// Sa2 [nimg][W^2] and Sb2 [W^2]: exact energies as FP32 pairs (hi, lo);
// ia32 [W^2]: unit / Area.
// Dynamic shared memory of k_rows_inv for transform length N (all-ones if N
// is not a supported length).
size_t rows_inv_smem_bytes(int N, int wm1);
cudaError_t launch_rows_inv(int N, const float2* Y, int64_t y_fstride, int ncv, int wm1, int64_t nimg,
                            const float2* tw, const u64* rowE, const u64* colE, const u64* tot,
                            const uint32_t* corners, int mc, int nc, const float2* Sb2, const float* ia32,
                            double* cost, int32_t* coarse, double* fbest, float* margin, cudaStream_t st);

cudaError_t launch_energy(bool f32, bool out_double, const u64* rowE, const u64* colE, const u64* tot,
                          const uint32_t* corners, int64_t nimg, int mc, int nc, int wm1, void* out, int flip,
                          cudaStream_t st);

// acc: nimg x 9 u64 and ticket: nimg u32 of scratch (cleared here).
// bsq: the template's b^2 prefix table (launch_sq_prefix), or nullptr to sum
// b^2 inside the kernel.
cudaError_t launch_jitter(const uint16_t* frames, int64_t fstride, int64_t nimg, const uint16_t* tmpl, int m,
                          int n, const u64* bsq, const int32_t* coarse, int32_t* shifts, double* ffinal, u64* acc,
                          unsigned int* ticket, cudaStream_t st);

// One run of one stack's frames for launch_jitter_multi: T frames from
// `frames` (stride fstride), their searched-grid optima in coarse [T][2]
// (may equal shifts: each frame's optimum is read before its result is
// written), results in shifts [T][2] and ffinal [T] (nullable).
struct JitSegment {
    const uint16_t* frames;
    int64_t fstride, T;
    const uint16_t* tmpl;
    const u64* bsq;
    const int32_t* coarse;
    int32_t* shifts;
    double* ffinal;
    int m, n;
};
// The refinement of every segment in persistent launches, each of at most
// kJitSegs segments holding at most `capacity` frames; acc (9 u64 per frame)
// and ticket (one u32 per frame) are scratch for `capacity` frames. Every
// segment needs a b^2 prefix table (bsq) and at most `capacity` frames
// (cudaErrorInvalidValue otherwise).
cudaError_t launch_jitter_multi(const JitSegment* segs, int nseg, u64* acc, unsigned int* ticket, int64_t capacity,
                                int num_sms, cudaStream_t st);

// More than one level: level-l images (int32 box sums of 2^l x 2^l pixels)
// and the 3x3 refinement on level l of the doubled level-(l+1) optimum.
size_t level_image_elems(int m, int n, int l);
cudaError_t launch_box_level(const uint16_t* img, int m, int n, int l, int32_t* out, cudaStream_t st);
// acc: nimg x 9 u64 and ticket: nimg u32 of scratch (cleared here).
cudaError_t launch_jitter_level(const uint16_t* frames, int64_t fstride, int64_t nimg, int m, int n, int l,
                                const int32_t* bl, const int32_t* cin, int32_t* cout, u64* acc,
                                unsigned int* ticket, cudaStream_t st);

// The correction step: corrected frames and/or the corrected mean image;
// sum (u64) and cnt (u32) are m*n scratch, cleared here.
cudaError_t launch_apply(const uint16_t* frames, int64_t fstride, int64_t T, int m, int n, const int32_t* shifts,
                         uint16_t fill, uint16_t* corrected, double* mean, u64* sum, unsigned int* cnt,
                         int num_sms, cudaStream_t st);

// P[(m+1) x (n+1)], P[i][j] = sum over i' < i, j' < j of tmpl^2 (exact u64).
cudaError_t launch_sq_prefix(const uint16_t* tmpl, int m, int n, u64* P, cudaStream_t st);

cudaError_t launch_copy_shifts(const int32_t* coarse, int32_t* shifts, const double* fbest, double* ffinal,
                               int64_t T, cudaStream_t st);

// The template offset c (two kernels: per-slice sums into part[0 .. nparts),
// then their sum in order; part is scratch of at least one u64).
cudaError_t launch_template_offset(bool f32, const void* tmpl, int m, int n, int levels, int32_t* coff_i,
                                   float* coff_f, u64* part, int64_t nparts, cudaStream_t st);

cudaError_t launch_softmin(const double* cost, int64_t T, int K, double tau_scale, double* loss, float* weights,
                           cudaStream_t st);

// Shared memory the adjoint kernels need for half-window wm1.
size_t grad_smem_bytes(int wm1);

// Adjoint of f (levels = 0): grad_template += dL/db, grad_frames = dL/da
// (if non-null). acc (m*n floats) and Q (W*W floats) are scratch. With corr
// set the correlation part of dL/db is formed here by the tiled direct
// contraction; with corr clear acc already holds it (the FFT route below).
cudaError_t launch_grad(const uint16_t* frames, int64_t T, int m, int n, int wm1, const float* G, float scale,
                        const double* inv_area, const int32_t* coff, const void* tmpl, int tmpl_f32, int corr,
                        float* acc, float* Q, float* grad_template, float* grad_frames, cudaStream_t st);

// The correlation part of dL/db through FFTs (FFT form, levels = 0):
// QX[f][v][k] = row spectra of q_f = scale * G_f / Area (k = s + w - 1);
// Acc (ncv x Nr, four-step order, zero before the first group) += sum_f
// DFT_cols(X_f) * conj(DFT_cols(QX_f)); the inverse writes acc[r][j] for
// r < mc, j < nc, through Yt (mc x ncv complex scratch).
cudaError_t launch_q_rows(int Nc, const float* G, const double* inv_area, float scale, int wm1, int64_t T,
                          const float2* twc, float2* QX, cudaStream_t st);
cudaError_t launch_adj_cols(int Nr, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv, const float2* QX,
                            int wm1, int64_t T, const float2* twr, float2* Acc, unsigned int* err, cudaStream_t st);
cudaError_t launch_adj_inverse(int Nr, int Nc, const float2* Acc, int ncv, int mc, int nc, const float2* twr,
                               const float2* twc, float2* Yt, float* out, cudaStream_t st);

// ---- the direct (tensor-core) form -----------------------------------------
size_t direct_tiles_bytes(int mc, int ncp, int W);  // the template-row table the Toeplitz tiles are built from
size_t direct_smem(int W);
cudaError_t launch_frame_planes(bool f32, const void* src, int64_t src_fstride, int64_t nimg, int m, int n, int levels,
                                int mc, int nc, const int32_t* coff_i, const float* coff_f, const float2* tw,
                                u64* rowE, u64* colE, u64* tot, uint32_t* corners, int wm1, void* p_hi, void* p_lo,
                                int ldp, cudaStream_t st);
cudaError_t launch_toeplitz(bool f32, const void* tmpl, int m, int n, int levels, int mc, int nc, int ncp, int wm1,
                            const int32_t* coff_i, const float* coff_f, float* bprime, void* tiles, cudaStream_t st);
// K splits of one direct-form launch (1 .. kDirSplitMax): each writes a
// partial h slab of T * W * W floats, which launch_combine_h adds in order.
constexpr int kDirSplits = 8;
int direct_ksplit(int W, int64_t T, int mc, int nqc, int num_sms);
cudaError_t launch_direct(const void* a_hi, const void* a_lo, int64_t T, int mc, int ncp, int nqc, int wm1,
                          const void* tiles, float* h, int ksplit, unsigned int* err, cudaStream_t st);
cudaError_t launch_combine_h(const float* h, int ksplit, int64_t nimg, int wm1, const float2* Sa2, const float2* Sb2,
                             const float* ia32, double* cost, int32_t* coarse, double* fbest, float* margin,
                             cudaStream_t st);

// out[k] = (hi, lo): hi the nearest float of x[k], lo the rounded remainder.
cudaError_t launch_pair_from_double(const double* x, float2* out, int64_t count, cudaStream_t st);

// Sets the dynamic shared-memory limit of `func` on the current device once.
cudaError_t ensure_smem(const void* func, size_t bytes);

// One CTA whose bounded mbarrier wait is never satisfied: sets *err after
// about a second and returns (the timeout path's check).
cudaError_t launch_wait_selftest(unsigned int* err, cudaStream_t st);

}  // namespace moco
