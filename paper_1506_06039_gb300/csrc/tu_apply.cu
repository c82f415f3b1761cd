// The correction step: apply each frame's found shift (Section 2, the
// aligned shifts "motion correct" the video).
//   corrected[f][i][j] = a_f[i + s_f][j + t_f] inside the frame, else fill
//   mean[i][j]         = sum of the in-frame source pixels / their count (FP64
//                        from the exact integer sum; fill where no frame
//                        covers the pixel)
// k_apply: grid (pixel tiles, frame chunks). A thread owns 8 consecutive
// pixels of one row (16 bytes) and walks the frames of its chunk; the source
// columns j + t start at an offset o = t mod 8 that is the same for the whole
// frame, so two aligned 16-byte loads and a switch on o (uniform across the
// CTA) give the 8 values. Per-pixel sums (exact in 32 bits for up to 65536
// frames) and counts stay in registers and are added to the plan's 64-bit
// accumulators once per chunk. k_apply_mean then divides.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "kernels.cuh"

namespace moco {

constexpr int kApplyThreads = 256;

// Half-words O .. O+7 of the 16 half-words in (q0, q1), as 4 packed words.
template <int O>
__device__ __forceinline__ void apply_extract(const uint4& q0, const uint4& q1, uint32_t (&v)[4]) {
    const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (O % 2 == 0) v[k] = w[O / 2 + k];
        else v[k] = __byte_perm(w[O / 2 + k], w[O / 2 + k + 1], 0x5432);
    }
}

static __global__ void __launch_bounds__(kApplyThreads)
k_apply(const uint16_t* __restrict__ frames, int64_t fstride, int64_t T, int m, int n,
        const int32_t* __restrict__ shifts, uint16_t fill, int frames_per_chunk, uint16_t* __restrict__ corrected,
        u64* __restrict__ sum, unsigned int* __restrict__ cnt) {
    const int G = n / 8;
    const int64_t task = (int64_t)blockIdx.x * kApplyThreads + threadIdx.x;
    if (task >= (int64_t)m * G) return;
    const int i = (int)(task / G), j0 = 8 * (int)(task - (int64_t)(task / G) * G);
    const int64_t f_begin = (int64_t)blockIdx.y * frames_per_chunk;
    const int64_t f_end = min(T, f_begin + frames_per_chunk);
    uint32_t acc[8], num[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k] = 0;
        num[k] = 0;
    }
    const uint32_t fill2 = (uint32_t)fill | ((uint32_t)fill << 16);
    // Four frames per iteration: all their loads are issued before any is used.
    constexpr int kF = 4;
    for (int64_t fb = f_begin; fb < f_end; fb += kF) {
        uint4 q0[kF], q1[kF];
        int c[kF];
        bool row_in[kF];
#pragma unroll
        for (int u = 0; u < kF; ++u) {
            const int64_t f = fb + u;
            q0[u] = make_uint4(0, 0, 0, 0);
            q1[u] = make_uint4(0, 0, 0, 0);
            row_in[u] = false;
            c[u] = 0;
            if (f < f_end) {
                // Shifts beyond the frame are clamped: every source pixel is outside.
                const int s = max(-m, min(m, shifts[2 * f])), t = max(-n, min(n, shifts[2 * f + 1]));
                const int r = i + s;
                c[u] = j0 + t;  // first source column
                const int o = c[u] & 7, cb = c[u] - o;
                row_in[u] = r >= 0 && r < m;
                if (row_in[u]) {
                    const uint16_t* src = frames + f * fstride + (int64_t)r * n;
                    if (cb >= 0 && cb + 8 <= n) q0[u] = __ldg(reinterpret_cast<const uint4*>(src + cb));
                    if (o != 0 && cb + 8 >= 0 && cb + 16 <= n)
                        q1[u] = __ldg(reinterpret_cast<const uint4*>(src + cb + 8));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kF; ++u) {
            const int64_t f = fb + u;
            if (f >= f_end) break;
            uint32_t v[4];
            switch (c[u] & 7) {
                case 0: apply_extract<0>(q0[u], q1[u], v); break;
                case 1: apply_extract<1>(q0[u], q1[u], v); break;
                case 2: apply_extract<2>(q0[u], q1[u], v); break;
                case 3: apply_extract<3>(q0[u], q1[u], v); break;
                case 4: apply_extract<4>(q0[u], q1[u], v); break;
                case 5: apply_extract<5>(q0[u], q1[u], v); break;
                case 6: apply_extract<6>(q0[u], q1[u], v); break;
                default: apply_extract<7>(q0[u], q1[u], v); break;
            }
            // Pixels whose source lies outside the frame take the fill value.
            uint32_t inside = 0;  // bit k: pixel j0 + k has an in-frame source
            if (row_in[u]) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (c[u] + k >= 0 && c[u] + k < n) inside |= 1u << k;
            }
            if (inside != 0xffu) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t keep = (((inside >> (2 * k)) & 1u) ? 0x0000ffffu : 0u) |
                                          (((inside >> (2 * k + 1)) & 1u) ? 0xffff0000u : 0u);
                    v[k] = (v[k] & keep) | (fill2 & ~keep);
                }
            }
            if (corrected)
                *reinterpret_cast<uint4*>(corrected + f * (int64_t)m * n + (int64_t)i * n + j0) =
                    make_uint4(v[0], v[1], v[2], v[3]);
            if (sum) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t in = (inside >> k) & 1u;
                    const uint32_t x = (k & 1) ? (v[k / 2] >> 16) : (v[k / 2] & 0xffffu);
                    acc[k] += in ? x : 0u;
                    num[k] += in;
                }
            }
        }
    }
    if (sum) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (num[k]) {
                atomicAdd(&sum[(int64_t)i * n + j0 + k], (u64)acc[k]);
                atomicAdd(&cnt[(int64_t)i * n + j0 + k], num[k]);
            }
    }
}

static __global__ void k_apply_mean(const u64* __restrict__ sum, const unsigned int* __restrict__ cnt, int64_t mn,
                                    uint16_t fill, double* __restrict__ mean) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= mn) return;
    mean[p] = cnt[p] ? (double)sum[p] / (double)cnt[p] : (double)fill;
}

cudaError_t launch_apply(const uint16_t* frames, int64_t fstride, int64_t T, int m, int n, const int32_t* shifts,
                         uint16_t fill, uint16_t* corrected, double* mean, u64* sum, unsigned int* cnt,
                         int num_sms, cudaStream_t st) {
    if (T < 0 || (!corrected && !mean)) return cudaSuccess;
    const int64_t mn = (int64_t)m * n;
    if (mean) {
        cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(u64) * mn, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * mn, st);
        if (e != cudaSuccess) return e;
    }
    if (T == 0) {  // no frame covers any pixel: the mean is the fill value
        if (!mean) return cudaSuccess;
        k_apply_mean<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(sum, cnt, mn, fill, mean);
        return cudaGetLastError();
    }
    const int64_t tiles = ((int64_t)m * (n / 8) + kApplyThreads - 1) / kApplyThreads;
    // Enough frame chunks for ~8 CTAs per SM; at most 65536 frames per chunk
    // keeps the 32-bit per-pixel sums exact.
    int64_t chunks = std::max<int64_t>(1, (8ll * num_sms + tiles - 1) / tiles);
    chunks = std::min<int64_t>(chunks, T);
    int64_t fpc = (T + chunks - 1) / chunks;
    if (fpc > 65536) fpc = 65536;
    chunks = (T + fpc - 1) / fpc;
    if (chunks > 65535 || tiles > 0x7fffffff) return cudaErrorInvalidValue;
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    k_apply<<<grid, kApplyThreads, 0, st>>>(frames, fstride, T, m, n, shifts, fill, (int)fpc, corrected,
                                            mean ? sum : nullptr, mean ? cnt : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !mean) return e;
    k_apply_mean<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(sum, cnt, mn, fill, mean);
    return cudaGetLastError();
}

}  // namespace moco
