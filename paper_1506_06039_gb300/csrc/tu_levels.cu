// More than one level (Section 2: the resolution is "multiplied by two
// multiple times"; Section 3: three or four downsamplings cause severe
// errors). Level l is the 2x2 sum of level l - 1, i.e. the sum of the
// 2^l x 2^l full-resolution pixels behind each of its pixels. After the
// exhaustive search on level L, each level l = L-1 .. 1 refines the doubled
// optimum by the 3x3 search with exact sums (k_jitter_level); level 0 is
// k_jitter's full-resolution pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "kernels.cuh"

namespace moco {

constexpr int kLevelThreads = 256;

// Level-l image of a uint16 image: out[i][j] = box sum, (m >> l) x (n >> l).
static __global__ void k_box_level(const uint16_t* __restrict__ img, int m, int n, int l, int32_t* __restrict__ out) {
    const int ml = m >> l, nl = n >> l;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)ml * nl) return;
    const int i = (int)(p / nl), j = (int)(p % nl);
    out[p] = (int32_t)box_sum_l(img, n, i, j, l);
}

// The nine candidates (2 sc + u - 1, 2 tc + v - 1) of level l: exact int64
// S = sum over D of (a_l[i+s][j+t] - b_l[i][j])^2 on level l's (ml x nl)
// images. Grid (bands of kLevelRows level rows, frames): a CTA forms the
// frame's level rows its band needs (kLevelRows + 2) from the full-
// resolution frame in shared memory, sums its band, and adds the nine sums to
// the frame's accumulators; the frame's last CTA (ticket) takes the minimum
// of S / Area with the tie-break, compared as exact rationals. acc and ticket
// are zero on entry. b_l is the plan's level image.
constexpr int kLevelRows = 16;

static __global__ void __launch_bounds__(kLevelThreads)
k_jitter_level(const uint16_t* __restrict__ frames, int64_t fstride, int m, int n, int l,
               const int32_t* __restrict__ bl, const int32_t* __restrict__ cin, int32_t* __restrict__ cout,
               u64* __restrict__ acc_g, unsigned int* __restrict__ ticket) {
    extern __shared__ __align__(16) int32_t arows[];  // (kLevelRows + 2) x nl
    __shared__ long long red[kLevelThreads / 32][9];
    __shared__ bool last;
    const int ml = m >> l, nl = n >> l;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t f = blockIdx.y;
    const uint16_t* a = frames + f * fstride;
    const int s0 = 2 * cin[2 * f], t0 = 2 * cin[2 * f + 1];
    const int i0 = blockIdx.x * kLevelRows, rows = min(kLevelRows, ml - i0);
    // level rows i0 + s0 - 1 .. i0 + rows + s0 (zero outside; masked below)
    for (int rr = warp; rr < rows + 2; rr += kLevelThreads / 32) {
        const int ar = i0 + s0 - 1 + rr;
        const bool in = ar >= 0 && ar < ml;  // the same for the whole warp
        for (int j = lane; j < nl; j += 32) arows[rr * nl + j] = in ? (int32_t)box_sum_l(a, n, ar, j, l) : 0;
    }
    __syncthreads();
    long long acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0;
    for (int ri = warp; ri < rows; ri += kLevelThreads / 32) {
        const int i = i0 + ri;
        for (int j = lane; j < nl; j += 32) {
            const int32_t b = bl[(int64_t)i * nl + j];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ar = i + s0 - 1 + u;
                if (ar < 0 || ar >= ml) continue;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int ac = j + t0 - 1 + v;
                    if (ac < 0 || ac >= nl) continue;
                    const long long d = (long long)(arows[(ri + u) * nl + ac] - b);
                    acc[u * 3 + v] += d * d;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        long long v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (tid < 9) {
        long long sum = 0;
        for (int wi = 0; wi < kLevelThreads / 32; ++wi) sum += red[wi][tid];
        atomicAdd(&acc_g[f * 9 + tid], (u64)sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&ticket[f], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    int bk = -1, bs = 0, bt = 0;
    u64 bS = 0, bA = 1;
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) {
            const int s = s0 + u - 1, t = t0 + v - 1;
            const u64 S = atomicAdd(&acc_g[f * 9 + u * 3 + v], 0ull);
            const u64 A = (u64)(ml - abs(s)) * (u64)(nl - abs(t));
            bool take = bk < 0;
            if (!take) {
                int eq;
                if (ratio_lt(S, A, bS, bA, &eq)) take = true;
                else if (eq) {
                    const int k1 = abs(s) + abs(t), k2 = abs(bs) + abs(bt);
                    take = (k1 < k2) || (k1 == k2 && (s < bs || (s == bs && t < bt)));
                }
            }
            if (take) { bk = u * 3 + v; bS = S; bA = A; bs = s; bt = t; }
        }
    cout[2 * f] = bs;
    cout[2 * f + 1] = bt;
}

size_t level_image_elems(int m, int n, int l) { return (size_t)(m >> l) * (size_t)(n >> l); }

cudaError_t launch_box_level(const uint16_t* img, int m, int n, int l, int32_t* out, cudaStream_t st) {
    const int64_t count = (int64_t)(m >> l) * (n >> l);
    if (count <= 0) return cudaSuccess;
    k_box_level<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(img, m, n, l, out);
    return cudaGetLastError();
}

cudaError_t launch_jitter_level(const uint16_t* frames, int64_t fstride, int64_t nimg, int m, int n, int l,
                                const int32_t* bl, const int32_t* cin, int32_t* cout, u64* acc,
                                unsigned int* ticket, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(u64) * 9 * nimg, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int) * nimg, st);
    if (e != cudaSuccess) return e;
    const int ml = m >> l, nl = n >> l;
    const size_t smem = sizeof(int32_t) * (size_t)(kLevelRows + 2) * nl;  // <= 18 x 2048 x 4 bytes
    e = ensure_smem(reinterpret_cast<const void*>(k_jitter_level), smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((ml + kLevelRows - 1) / kLevelRows), (unsigned)nimg);
    k_jitter_level<<<grid, kLevelThreads, smem, st>>>(frames, fstride, m, n, l, bl, cin, cout, acc, ticket);
    return cudaGetLastError();
}

}  // namespace moco
