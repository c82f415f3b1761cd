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

// The nine candidates (2 sc + u - 1, 2 tc + v - 1) of level LV: exact int64
// S = sum over D of (a_l[i+s][j+t] - b_l[i][j])^2 on level LV's (ml x nl)
// images. Grid (bands of kLevelRows level rows, frames): a CTA forms the
// frame's level rows its band needs (kLevelRows + 2) from the full-
// resolution frame in shared memory, sums its band (four neighbouring level
// pixels per lane at a time; a candidate whose frame pixel lies outside the
// frame contributes zero, by a select), and adds the
// nine sums to the frame's accumulators; on the frame's last CTA (ticket)
// the lanes of one warp take the minimum of S / Area with the tie-break,
// compared as exact rationals. acc and ticket are zero on entry. b_l is the
// plan's level image.
// Band height in level rows (taller bands, 64 rows at 512^2, were slower:
// fewer CTAs per frame to hide the latency of the box sums' loads).
constexpr int kLevelRows = 16;

template <int LV>
static __global__ void __launch_bounds__(kLevelThreads)
k_jitter_level(const uint16_t* __restrict__ frames, int64_t fstride, int m, int n,
               const int32_t* __restrict__ bl, const int32_t* __restrict__ cin, int32_t* __restrict__ cout,
               u64* __restrict__ acc_g, unsigned int* __restrict__ ticket) {
    extern __shared__ __align__(16) int32_t arows[];  // (kLevelRows + 2) x nl
    __shared__ u64 red[kLevelThreads / 32][9];
    __shared__ bool last;
    const int ml = m >> LV, nl = n >> LV;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t f = blockIdx.y;
    const uint16_t* a = frames + f * fstride;
    const int s0 = 2 * cin[2 * f], t0 = 2 * cin[2 * f + 1];
    const int i0 = blockIdx.x * kLevelRows, rows = min(kLevelRows, ml - i0);
    // level rows i0 + s0 - 1 .. i0 + rows + s0 (zero outside; masked below)
    for (int rr = warp; rr < rows + 2; rr += kLevelThreads / 32) {
        const int ar = i0 + s0 - 1 + rr;
        const bool in = ar >= 0 && ar < ml;  // the same for the whole warp
        if (!in) {
            for (int j = lane; j < nl; j += 32) arows[rr * nl + j] = 0;
            continue;
        }
#pragma unroll 4
        for (int j = lane; j < nl; j += 32) arows[rr * nl + j] = (int32_t)box_sum_vec<LV>(a, n, ar, j);  // loads of four in flight
    }
    __syncthreads();
    u64 acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0;
    // Each lane takes four neighbouring level pixels of a row at a time: their
    // windows span six frame columns per window row, loaded (and clamped and
    // checked) once for all twelve of the row's candidates.
    for (int ri = warp; ri < rows; ri += kLevelThreads / 32) {
        const int i = i0 + ri;
        const int32_t* brow = bl + (int64_t)i * nl;
        for (int j0 = 4 * lane; j0 < nl; j0 += 128) {
            int32_t b[4];
            bool pv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                pv[p] = j0 + p < nl;
                b[p] = 0;
                if (pv[p]) b[p] = __ldg(brow + j0 + p);
            }
            int cj[6];
            bool cv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int ac = j0 + t0 - 1 + c;
                cv[c] = (unsigned)ac < (unsigned)nl;
                cj[c] = min(max(ac, 0), nl - 1);
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ar = i + s0 - 1 + u;
                if (ar < 0 || ar >= ml) continue;  // the same for the whole warp
                const int32_t* ap = arows + (ri + u) * nl;
                int32_t av[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) av[c] = ap[cj[c]];
#pragma unroll
                for (int v = 0; v < 3; ++v)
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const int32_t d = (cv[p + v] && pv[p]) ? av[p + v] - b[p] : 0;
                        add_sq(acc[u * 3 + v], d);
                    }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        u64 v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (tid < 9) {
        u64 sum = 0;
        for (int wi = 0; wi < kLevelThreads / 32; ++wi) sum += red[wi][tid];
        atomicAdd(&acc_g[f * 9 + tid], sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&ticket[f], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last || warp != 0) return;
    __threadfence();
    u64 S = 0, A = 1;
    int s = 0, t = 0;
    if (lane < 9) {
        s = s0 + lane / 3 - 1;
        t = t0 + lane % 3 - 1;
        A = (u64)(ml - abs(s)) * (u64)(nl - abs(t));
        S = ld_relaxed_u64(acc_g + f * 9 + lane);
    }
    u64 bS = 0, bA = 1;
    int bs = 0, bt = 0;
    choose_nine(S, A, s, t, bS, bA, bs, bt);
    if (lane == 0) {
        cout[2 * f] = bs;
        cout[2 * f + 1] = bt;
    }
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
    dim3 grid((unsigned)((ml + kLevelRows - 1) / kLevelRows), (unsigned)nimg);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t r = ensure_smem(reinterpret_cast<const void*>(kern), smem);
        if (r != cudaSuccess) return r;
        kern<<<grid, kLevelThreads, smem, st>>>(frames, fstride, m, n, bl, cin, cout, acc, ticket);
        return cudaSuccess;
    };
    switch (l) {  // refinement levels 1 .. 3 (at most four levels in all)
        case 1: e = run(k_jitter_level<1>); break;
        case 2: e = run(k_jitter_level<2>); break;
        case 3: e = run(k_jitter_level<3>); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace moco
