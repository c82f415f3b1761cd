// The correlation part of the template adjoint through FFTs:
//   acc[i][j] = sum_f sum_st q_f[s][t] a'_f[i+s][j+t]
//             = IDFT2( sum_f DFT2(a'_f) * conj(DFT2(q_f)) )[i][j]
// with q_f[s][t] placed at ((s mod Nr), (t mod Nc)) and the plan's zero-padded
// sizes Nr >= m + w - 1, Nc >= n + w - 1 (no wrap-around reaches [0,m) x [0,n)).
// The frames' row spectra come from the forward frame pass (k_frame_rows, X);
//   k_q_rows     : row spectra of each frame's (2w-1)^2 weight table  -> QX
//   k_adj_cols   : column transforms of X and QX, sum over a chunk of frames
//                  of A * conj(Q) in registers, atomically added  -> Acc
//   k_adj_icols  : inverse column transforms of Acc (rows [0, m))  -> Yt
//   k_adj_irows  : inverse real row transforms (columns [0, n))    -> acc
// Both forward column transforms leave the same (four-step) output order, in
// which the product is taken and Acc is kept; the inverse takes that order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fft_sizes.h"
#include "internal.h"
#include "kernels.cuh"

namespace moco {

constexpr int kAdjFramesPerCta = 16;
constexpr size_t kAdjStreamSmemMax = 113 * 1024 + 512;  // two CTAs per SM

// One CTA per frame: the 2w-1 rows of q_f (q = scale * G * inv_area), two
// rows per complex transform of length N (= Nc), spectra split and written
// as QX[f][v][k], v in [0, N/2], k in [0, W) (k = s + w - 1).
template <int N>
__global__ void __launch_bounds__(kRowsThreads)
k_q_rows(const float* __restrict__ G, const double* __restrict__ inv_area, float scale, int wm1,
         const float2* __restrict__ tw_g, float2* __restrict__ QX) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    constexpr int NH = N / 2;
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // (kRC/2) x LD
    float2* tw = buf + (kRC / 2) * LD;                   // N: forward table
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int W = 2 * wm1 + 1, K = W * W;
    const int64_t f = blockIdx.x;
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[i];
    const float* g = G + f * K;
    float2* qx = QX + f * (int64_t)(NH + 1) * W;
    const int npairs = (W + 1) / 2;
    for (int p0 = 0; p0 < npairs; p0 += kRC / 2) {
        const int np = min(kRC / 2, npairs - p0);
        __syncthreads();
        for (int task = tid; task < np * N; task += nthr) {
            const int pi = task / N, c = task - pi * N;
            const int t = c <= wm1 ? c : (c >= N - wm1 ? c - N : 0x7fffffff);  // shift t at column c
            float va = 0.f, vb = 0.f;
            if (t != 0x7fffffff) {
                const int ka = 2 * (p0 + pi), kb = ka + 1;
                const int ti = t + wm1;
                va = scale * g[ka * W + ti] * (float)inv_area[ka * W + ti];
                if (kb < W) vb = scale * g[kb * W + ti] * (float)inv_area[kb * W + ti];
            }
            buf[pi * LD + sk<N>(c)] = make_float2(va, vb);
        }
        __syncthreads();
        fft4_fwd<N>(buf, LD, np, tw, tid, nthr);
        for (int task = tid; task < (NH + 1) * np; task += nthr) {
            const int v = task / np, pi = task - v * np;
            const float2 zk = buf[pi * LD + sk<N>(spec_pos<N>(v))];
            const float2 zn = cconj(buf[pi * LD + sk<N>(spec_pos<N>(v == 0 ? 0 : N - v))]);
            const int ka = 2 * (p0 + pi), kb = ka + 1;
            qx[(int64_t)v * W + ka] = cscale(cadd(zk, zn), 0.5f);
            if (kb < W) {
                const float2 d = csub(zk, zn);
                qx[(int64_t)v * W + kb] = make_float2(0.5f * d.y, -0.5f * d.x);
            }
        }
    }
}

// Grid (column blocks of kColsVC, chunks of kAdjFramesPerCta frames). Thread
// p owns position p of every column of the block and keeps its sum.
template <int N>
__global__ void __launch_bounds__(cols_threads<N>(), cols_threads<N>() <= 320 ? 2 : 1)
k_adj_cols(const float2* __restrict__ X, int64_t x_fstride, int ldx, int mc, int ncv, const float2* __restrict__ QX,
           int wm1, int64_t T, const float2* __restrict__ tw_g, float2* __restrict__ Acc) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    float2* bufA = reinterpret_cast<float2*>(smem_raw);  // kColsVC x LD
    float2* bufQ = bufA + kColsVC * LD;                  // kColsVC x LD
    float2* tw = bufQ + kColsVC * LD;                    // N: forward table
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int W = 2 * wm1 + 1;
    const int v0 = blockIdx.x * kColsVC, nv = min(kColsVC, ncv - v0);
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[i];
    float2 acc[kColsVC];
#pragma unroll
    for (int vi = 0; vi < kColsVC; ++vi) acc[vi] = make_float2(0.f, 0.f);
    const int64_t f_begin = (int64_t)blockIdx.y * kAdjFramesPerCta;
    const int64_t f_end = (T < f_begin + kAdjFramesPerCta) ? T : f_begin + kAdjFramesPerCta;
    for (int64_t f = f_begin; f < f_end; ++f) {
        __syncthreads();
        const float2* xs = X + f * x_fstride + (int64_t)v0 * ldx;
        const float2* qs = QX + f * (int64_t)ncv * W + (int64_t)v0 * W;
        for (int i = tid; i < N; i += nthr) {
            const int ski = sk<N>(i);
            // row i of the column holds shift s = i (i <= wm1) or i - N (i >= N - wm1)
            const int k = i <= wm1 ? i + wm1 : (i >= N - wm1 ? i - N + wm1 : -1);
#pragma unroll
            for (int vi = 0; vi < kColsVC; ++vi) {
                if (vi >= nv) break;
                bufA[vi * LD + ski] = i < mc ? xs[(int64_t)vi * ldx + i] : make_float2(0.f, 0.f);
                bufQ[vi * LD + ski] = k >= 0 ? qs[(int64_t)vi * W + k] : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        fft4_fwd<N>(bufA, LD, nv, tw, tid, nthr);
        fft4_fwd<N>(bufQ, LD, nv, tw, tid, nthr);
        if (tid < N) {
            const int skp = sk<N>(tid);
#pragma unroll
            for (int vi = 0; vi < kColsVC; ++vi) {
                if (vi >= nv) break;
                const float2 a = bufA[vi * LD + skp], q = bufQ[vi * LD + skp];
                acc[vi].x += a.x * q.x + a.y * q.y;  // a * conj(q)
                acc[vi].y += a.y * q.x - a.x * q.y;
            }
        }
    }
    if (tid < N) {
#pragma unroll
        for (int vi = 0; vi < kColsVC; ++vi) {
            if (vi >= nv) break;
            float* dst = reinterpret_cast<float*>(Acc + (int64_t)(v0 + vi) * N + tid);
            atomicAdd(dst, acc[vi].x);
            atomicAdd(dst + 1, acc[vi].y);
        }
    }
}

// The same sum with persistent CTAs: grid (column blocks, frame slices),
// CTA (x, y) owns columns [v0, v0 + nv) (ncv split evenly over gridDim.x)
// and walks frames f = y, y + gridDim.y, ..., keeping its sums in registers
// and adding them once at the end. Each frame's X block (contiguous) arrives
// by one bulk copy issued when the previous frame's first stage has read the
// staging buffer; q's few nonzero rows are read straight from QX. The
// bounded wait on the copy sets *err and ends the CTA (after the copy).
template <int N>
__host__ __device__ constexpr size_t adj_stream_smem(int ldx) {
    return sizeof(float2) * ((size_t)kColsVC * ldx + 2 * (size_t)kColsVC * fft_ld<N>() + N);
}

template <int N>
__global__ void __launch_bounds__(cols_threads<N>(), 2)
k_adj_cols_stream(const float2* __restrict__ X, int64_t x_fstride, int ldx, int mc, int ncv,
                  const float2* __restrict__ QX, int wm1, int64_t T, const float2* __restrict__ tw_g,
                  float2* __restrict__ Acc, unsigned int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    float2* stg = reinterpret_cast<float2*>(smem_raw);  // kColsVC x ldx (ldx even)
    float2* bufA = stg + kColsVC * ldx;                  // kColsVC x LD
    float2* bufQ = bufA + kColsVC * LD;                  // kColsVC x LD
    float2* tw = bufQ + kColsVC * LD;                    // N: forward table
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int W = 2 * wm1 + 1;
    const int v0 = (int)((int64_t)blockIdx.x * ncv / gridDim.x);
    const int nv = (int)((int64_t)(blockIdx.x + 1) * ncv / gridDim.x) - v0;  // <= kColsVC (host)
    const uint32_t bytes = (uint32_t)(sizeof(float2) * nv * ldx);
    int64_t f = blockIdx.y;
    if (f >= T) return;  // the same for the whole CTA
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        fence_async_smem();
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(stg, X + f * x_fstride + (int64_t)v0 * ldx, bytes, &bar);
    }
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[i];
    float2 acc[kColsVC];
#pragma unroll
    for (int vi = 0; vi < kColsVC; ++vi) acc[vi] = make_float2(0.f, 0.f);
    uint32_t phase = 0;
    for (; f < T; f += gridDim.y) {
        __syncthreads();  // set-up / the previous frame's products are read from the buffers
        if (!mbar_wait(&bar, phase, err)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (tid == 0) mbar_wait(&bar, phase, err);  // the copy in flight lands before the CTA ends
            return;
        }
        phase ^= 1u;
        fft4_fwd_stage1_from<N>(stg, ldx, mc, bufA, LD, nv, tw, tid, nthr);
        // row i of q's column holds shift s = i (i <= wm1) or i - N (i >= N - wm1)
        const float2* qs = QX + f * (int64_t)ncv * W + (int64_t)v0 * W;
        fft4_fwd_stage1_gen<N>(
            [&](int r, int i) {
                const int k = i <= wm1 ? i + wm1 : (i >= N - wm1 ? i - N + wm1 : -1);
                return k >= 0 ? qs[(int64_t)r * W + k] : make_float2(0.f, 0.f);
            },
            bufQ, LD, nv, tw, tid, nthr);
        __syncthreads();
        if (tid == 0 && f + gridDim.y < T) {
            fence_async_smem();  // this frame's reads of the staging buffer come before the next copy
            mbar_expect_tx(&bar, bytes);
            bulk_g2s(stg, X + (f + gridDim.y) * x_fstride + (int64_t)v0 * ldx, bytes, &bar);
        }
        fft4_fwd_stage2<N>(bufA, LD, nv, tid, nthr);
        fft4_fwd_stage2<N>(bufQ, LD, nv, tid, nthr);
        if (tid < N) {
            const int skp = sk<N>(tid);
#pragma unroll
            for (int vi = 0; vi < kColsVC; ++vi) {
                if (vi >= nv) break;
                const float2 a = bufA[vi * LD + skp], q = bufQ[vi * LD + skp];
                acc[vi].x += a.x * q.x + a.y * q.y;  // a * conj(q)
                acc[vi].y += a.y * q.x - a.x * q.y;
            }
        }
    }
    if (tid < N) {
#pragma unroll
        for (int vi = 0; vi < kColsVC; ++vi) {
            if (vi >= nv) break;
            float* dst = reinterpret_cast<float*>(Acc + (int64_t)(v0 + vi) * N + tid);
            atomicAdd(dst, acc[vi].x);
            atomicAdd(dst + 1, acc[vi].y);
        }
    }
}

// Inverse column transforms of Acc (columns of the block), rows [0, mc)
// scaled by `scale`, written transposed: Yt[r][v].
template <int N>
__global__ void __launch_bounds__(cols_threads<N>())
k_adj_icols(const float2* __restrict__ Acc, int ncv, int mc, const float2* __restrict__ tw_g, float scale,
            float2* __restrict__ Yt) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // kColsVC x LD
    float2* tw = buf + kColsVC * LD;                     // N: inverse table
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int v0 = blockIdx.x * kColsVC, nv = min(kColsVC, ncv - v0);
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[N + i];
    for (int p = tid; p < N; p += nthr) {
        const int skp = sk<N>(p);
        for (int vi = 0; vi < nv; ++vi) buf[vi * LD + skp] = Acc[(int64_t)(v0 + vi) * N + p];
    }
    __syncthreads();
    fft4_inv<N>(buf, LD, nv, tw, tid, nthr);
    for (int task = tid; task < mc * kColsVC; task += nthr) {
        const int r = task / kColsVC, vi = task % kColsVC;
        if (vi >= nv) continue;
        Yt[(int64_t)r * ncv + v0 + vi] = cscale(buf[vi * LD + sk<N>(r)], scale);
    }
}

// Inverse real row transforms (length N = Nc) of Yt's rows, two rows per
// complex transform (kRC/2 pairs per CTA), columns [0, nc) -> out[r][j].
template <int N>
__global__ void __launch_bounds__(kRowsThreads)
k_adj_irows(const float2* __restrict__ Yt, int ncv, int mc, int nc, const float2* __restrict__ tw_g,
            float* __restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    constexpr int NH = N / 2;
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // (kRC/2) x LD
    float2* tw = buf + (kRC / 2) * LD;                   // N: inverse table
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[N + i];
    const int pair0 = blockIdx.x * (kRC / 2);
    const int npairs = (mc + 1) / 2;
    const int np = min(kRC / 2, npairs - pair0);
    for (int task = tid; task < np * N; task += nthr) {
        const int pi = task / N, k = task - pi * N;
        const int ra = 2 * (pair0 + pi), rb = ra + 1;
        const int kk = k <= NH ? k : N - k;
        float2 A = Yt[(int64_t)ra * ncv + kk];
        float2 B = rb < mc ? Yt[(int64_t)rb * ncv + kk] : make_float2(0.f, 0.f);
        if (k == 0 || k == NH) { A.y = 0.f; B.y = 0.f; }
        if (k > NH) { A.y = -A.y; B.y = -B.y; }
        buf[pi * LD + sk<N>(spec_pos<N>(k))] = make_float2(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    fft4_inv<N>(buf, LD, np, tw, tid, nthr);
    for (int task = tid; task < np * nc; task += nthr) {
        const int pi = task / nc, j = task - pi * nc;
        const int ra = 2 * (pair0 + pi);
        const float2 z = buf[pi * LD + sk<N>(j)];
        out[(int64_t)ra * nc + j] = z.x;
        if (ra + 1 < mc) out[(int64_t)(ra + 1) * nc + j] = z.y;
    }
}

template <int N>
static cudaError_t adj_rows_n(int which, const float* G, const double* inv_area, float scale, int wm1, int64_t T,
                              const float2* tw, float2* QX, const float2* Yt, int ncv, int mc, int nc, float* out,
                              cudaStream_t st) {
    const size_t smem = sizeof(float2) * ((kRC / 2) * fft_ld<N>() + N);
    if (which == 0) {
        cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_q_rows<N>), smem);
        if (e != cudaSuccess) return e;
        k_q_rows<N><<<(unsigned)T, kRowsThreads, smem, st>>>(G, inv_area, scale, wm1, tw, QX);
    } else {
        cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_adj_irows<N>), smem);
        if (e != cudaSuccess) return e;
        const int blocks = ((mc + 1) / 2 + kRC / 2 - 1) / (kRC / 2);
        k_adj_irows<N><<<(unsigned)blocks, kRowsThreads, smem, st>>>(Yt, ncv, mc, nc, tw, out);
    }
    return cudaGetLastError();
}

template <int N>
static cudaError_t adj_cols_n(int which, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv,
                              const float2* QX, int wm1, int64_t T, const float2* tw, float2* Acc, float scale,
                              float2* Yt, unsigned int* err, cudaStream_t st) {
    const int threads = cols_threads<N>();
    const unsigned vblocks = (unsigned)((ncv + kColsVC - 1) / kColsVC);
    if (which == 0) {
        // Persistent form when two CTAs fit on an SM and each walks several frames.
        const size_t ssm = adj_stream_smem<N>(ldx);
        if (ssm <= kAdjStreamSmemMax) {
            const void* fn = reinterpret_cast<const void*>(k_adj_cols_stream<N>);
            cudaError_t e = ensure_smem(fn, ssm);
            if (e != cudaSuccess) return e;
            int dev = 0, sms = 0, per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, ssm)) != cudaSuccess) return e;
            const int64_t slices = std::max(1, std::max(1, per_sm) * sms / (int)vblocks);
            if (T >= 4 * slices) {
                k_adj_cols_stream<N><<<dim3(vblocks, (unsigned)slices), threads, ssm, st>>>(X, x_fstride, ldx, mc, ncv,
                                                                                         QX, wm1, T, tw, Acc, err);
                return cudaGetLastError();
            }
        }
        const size_t smem = sizeof(float2) * (2 * kColsVC * fft_ld<N>() + N);
        cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_adj_cols<N>), smem);
        if (e != cudaSuccess) return e;
        dim3 grid(vblocks, (unsigned)((T + kAdjFramesPerCta - 1) / kAdjFramesPerCta));
        k_adj_cols<N><<<grid, threads, smem, st>>>(X, x_fstride, ldx, mc, ncv, QX, wm1, T, tw, Acc);
    } else {
        const size_t smem = sizeof(float2) * (kColsVC * fft_ld<N>() + N);
        cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_adj_icols<N>), smem);
        if (e != cudaSuccess) return e;
        k_adj_icols<N><<<vblocks, threads, smem, st>>>(Acc, ncv, mc, tw, scale, Yt);
    }
    return cudaGetLastError();
}

cudaError_t launch_q_rows(int Nc, const float* G, const double* inv_area, float scale, int wm1, int64_t T,
                          const float2* twc, float2* QX, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
#define MOCO_CASE(NN) \
    case NN: return adj_rows_n<NN>(0, G, inv_area, scale, wm1, T, twc, QX, nullptr, 0, 0, 0, nullptr, st);
    switch (Nc) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

cudaError_t launch_adj_cols(int Nr, const float2* X, int64_t x_fstride, int ldx, int mc, int ncv, const float2* QX,
                            int wm1, int64_t T, const float2* twr, float2* Acc, unsigned int* err, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
#define MOCO_CASE(NN) \
    case NN: return adj_cols_n<NN>(0, X, x_fstride, ldx, mc, ncv, QX, wm1, T, twr, Acc, 0.f, nullptr, err, st);
    switch (Nr) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

cudaError_t launch_adj_inverse(int Nr, int Nc, const float2* Acc, int ncv, int mc, int nc, const float2* twr,
                               const float2* twc, float2* Yt, float* out, cudaStream_t st) {
    const float scale = (float)(1.0 / ((double)Nr * (double)Nc));
    cudaError_t e = cudaErrorInvalidValue;
#define MOCO_CASE(NN) \
    case NN: e = adj_cols_n<NN>(1, nullptr, 0, 0, mc, ncv, nullptr, 0, 0, twr, const_cast<float2*>(Acc), scale, Yt, nullptr, st); break;
    switch (Nr) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default: break;
    }
#undef MOCO_CASE
    if (e != cudaSuccess) return e;
#define MOCO_CASE(NN) \
    case NN: return adj_rows_n<NN>(1, nullptr, nullptr, 0.f, 0, 0, twc, nullptr, Yt, ncv, mc, nc, out, st);
    switch (Nc) {
        MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef MOCO_CASE
}

}  // namespace moco
