// The differentiable form (not in the paper): a soft-min over shifts of
// Section 2's cost f, and the adjoint of f with respect to the template and
// the frames.
//
//   L_f = -tau_f log sum_{s,t} exp(-f_st / tau_f),  tau_f = scale * median_st f_st
//   dL_f/df_st = softmax weight g_st (tau held constant)
//
// f_st = (1/A_st) sum_{(i,j) in D_st} (a[i+s][j+t] - b[i][j])^2, so with
// q_st = G_st / A_st (G = dL/df):
//   dL/db[i][j] = -2 sum_f sum_st q_f,st a'_f[i+s][j+t] + 2 b'[i][j] sum_st Q_st 1[0<=i+s<m] 1[0<=j+t<n]
//   dL/da_f[k][l] = 2 a'_f[k][l] sum_st q_f,st 1[0<=k-s<m] 1[0<=l-t<n] - 2 sum_st q_f,st b'[k-s][l-t]
// with Q = sum_f q_f, a' = a - c, b' = b - c (the plan's offset; f does not
// depend on it), and a', b' taken as zero outside the image (that zero
// carries the 1[(i,j) in D_st] of each sum). The template side's correlation
// sum runs through FFTs where the plan has the FFT form (tu_adjoint.cu) and
// as the tiled direct FP32 contraction below otherwise; the frame side's is
// a direct contraction per frame; the indicator sums are rectangle sums of a
// 2-D prefix table of q (or Q).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace moco {

constexpr int kSoftminThreads = 256;
constexpr int kGradTile = 32;          // output tile edge
constexpr int kGradThreads = 256;      // 8 x 32: each thread 4 outputs of one row
constexpr int kGradFramesPerCta = 16;  // frames per CTA of the template adjoint

// Order-preserving map of doubles to unsigned keys (and back).
__device__ __forceinline__ unsigned long long dkey(double x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

// Order-preserving map of floats to unsigned keys (and back).
__device__ __forceinline__ unsigned int fkey(float x) {
    const unsigned int u = __float_as_uint(x);
    return (u >> 31) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned int k) {
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// One step of the radix select: hist holds the counts of the current digit
// among the keys that match the prefix; the digit of the element of rank
// *rank (0-based) is found by warp 0 (lane L owns bins 8L .. 8L + 7: a scan
// of the lanes' totals, then the owning lane walks its eight bins), and
// *rank becomes the rank within that digit. Returns the digit (all threads,
// after the call's barrier).
__device__ __forceinline__ unsigned int radix_digit(const unsigned int* hist, int* s_rank, unsigned int* s_digit) {
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        unsigned int c[8], tot = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = hist[lane * 8 + j];
            tot += c[j];
        }
        unsigned int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned int excl = incl - tot;
        const unsigned int r = (unsigned int)*s_rank;
        const unsigned int own = __ballot_sync(0xffffffffu, r >= excl && r < incl);
        if (lane == __ffs(own) - 1) {
            unsigned int rr = r - excl, b = lane * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (c[j] > rr) break;
                rr -= c[j];
                ++b;
            }
            *s_rank = (int)rr;
            *s_digit = b;
        }
    }
    __syncthreads();
    return *s_digit;
}

// One CTA per frame: the exact median (the element of rank K/2) by 8-bit
// radix select on order-preserving keys (32-bit keys when every cost of the
// frame is a float value, as the search's own costs are; 64-bit otherwise),
// then the stable log-sum-exp and the softmax weights (exponentials in FP32,
// their sum in FP64).
static __global__ void __launch_bounds__(kSoftminThreads)
k_softmin(const double* __restrict__ cost, int K, double tau_scale, double* __restrict__ loss,
          float* __restrict__ weights) {
    __shared__ unsigned int hist[256];
    __shared__ int s_rank;
    __shared__ unsigned int s_digit;
    __shared__ double s_red[32];
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t f = blockIdx.x;
    const double* c = cost + f * K;
    if (tid == 0) s_rank = K / 2;
    int exact = 1;
    for (int k = tid; k < K; k += nthr) exact &= ((double)(float)c[k] == c[k]);
    exact = __syncthreads_and(exact);
    double med;
    if (exact) {
        unsigned int prefix = 0, mask = 0;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += nthr) hist[i] = 0;
            __syncthreads();
            for (int k = tid; k < K; k += nthr) {
                const unsigned int key = fkey((float)c[k]);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            prefix |= radix_digit(hist, &s_rank, &s_digit) << shift;
            mask |= 255u << shift;
            __syncthreads();  // s_digit is read before the next pass writes it
        }
        med = (double)fkey_inv(prefix);
    } else {
        unsigned long long prefix = 0, mask = 0;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += nthr) hist[i] = 0;
            __syncthreads();
            for (int k = tid; k < K; k += nthr) {
                const unsigned long long key = dkey(c[k]);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            prefix |= (unsigned long long)radix_digit(hist, &s_rank, &s_digit) << shift;
            mask |= 255ull << shift;
            __syncthreads();
        }
        med = dkey_inv(prefix);
    }
    const double tau = tau_scale * med;
    double vmin = INFINITY;
    for (int k = tid; k < K; k += nthr) vmin = vmin < c[k] ? vmin : c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, vmin, o);
        vmin = vmin < other ? vmin : other;
    }
    if ((tid & 31) == 0) s_red[tid >> 5] = vmin;
    __syncthreads();
    if (tid == 0) {
        double v = s_red[0];
        for (int i = 1; i < (nthr + 31) / 32; ++i) v = v < s_red[i] ? v : s_red[i];
        s_red[0] = v;
    }
    __syncthreads();
    const double fmin_v = s_red[0];
    __syncthreads();
    float* wf = weights + f * K;
    if (!(tau > 0.0)) {
        // tau = 0 (a median of zero): the soft-min is the min; the weight is
        // shared equally by the minimisers.
        int cnt = 0;
        for (int k = tid; k < K; k += nthr) cnt += (c[k] == fmin_v);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int i = 0; i < (nthr + 31) / 32; ++i) t += s_cnt[i];
            s_cnt[0] = t;
            loss[f] = fmin_v;
        }
        __syncthreads();
        const float wv = 1.0f / (float)s_cnt[0];
        for (int k = tid; k < K; k += nthr) wf[k] = (c[k] == fmin_v) ? wv : 0.0f;
        return;
    }
    const double itau = 1.0 / tau;
    double z = 0.0;
    for (int k = tid; k < K; k += nthr) z += (double)expf(-(float)((c[k] - fmin_v) * itau));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = z;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < (nthr + 31) / 32; ++i) t += s_red[i];
        s_red[0] = t;
        loss[f] = fmin_v - tau * log(t);
    }
    __syncthreads();
    const float iZ = (float)(1.0 / s_red[0]);
    for (int k = tid; k < K; k += nthr) wf[k] = expf(-(float)((c[k] - fmin_v) * itau)) * iZ;
}

// Q[k] += scale * inv_area[k] * sum_f G[f][k] (k < K) over one chunk of
// kQsumFrames frames: grid (k blocks, frame chunks); Q is zero on entry.
constexpr int kQsumFrames = 32;
static __global__ void k_grad_qsum(const float* __restrict__ G, int64_t T, int K, const double* __restrict__ inv_area,
                            float scale, float* __restrict__ Q) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t f0 = (int64_t)blockIdx.y * kQsumFrames, f1 = (T < f0 + kQsumFrames) ? T : f0 + kQsumFrames;
    float s = 0.f;
    for (int64_t f = f0; f < f1; ++f) s += G[f * K + k];
    atomicAdd(&Q[k], s * (float)inv_area[k] * scale);
}

// 2-D inclusive prefix of a W x W table into P ((W+1) x (W+1), P[0][*] =
// P[*][0] = 0), by one block in shared memory.
__device__ __forceinline__ void prefix2d(const float* src, float* P, int W, int tid, int nthr) {
    const int L = W + 1;
    for (int i = tid; i < L * L; i += nthr) {
        const int a = i / L, b = i - a * L;
        P[i] = (a > 0 && b > 0) ? src[(a - 1) * W + (b - 1)] : 0.f;
    }
    __syncthreads();
    for (int a = tid; a < L; a += nthr) {
        float s = 0.f;
        for (int b = 0; b < L; ++b) { s += P[a * L + b]; P[a * L + b] = s; }
    }
    __syncthreads();
    for (int b = tid; b < L; b += nthr) {
        float s = 0.f;
        for (int a = 0; a < L; ++a) { s += P[a * L + b]; P[a * L + b] = s; }
    }
    __syncthreads();
}

// Sum of q over s in [slo, shi], t in [tlo, thi] (shift indices, inclusive).
__device__ __forceinline__ float rect(const float* P, int W, int wm1, int slo, int shi, int tlo, int thi) {
    const int L = W + 1;
    const int a0 = slo + wm1, a1 = shi + wm1 + 1, b0 = tlo + wm1, b1 = thi + wm1 + 1;
    if (a1 <= a0 || b1 <= b0) return 0.f;
    return P[a1 * L + b1] - P[a0 * L + b1] - P[a1 * L + b0] + P[a0 * L + b0];
}

// Correlation part of dL/db: acc[i][j] += sum_{f in chunk} sum_st q_f,st a'_f[i+s][j+t]
// for one kGradTY x kGradTX tile; q_f = scale * G_f * inv_area. Grid
// (tiles_x, tiles_y, chunks of kGradTmplFrames frames). Each of the 16 x 16
// threads owns 4 rows x 8 columns of outputs; for every shift row s it slides
// 12-value windows of its four halo rows along t, four taps at a time from
// 16-byte shared loads (q's rows are zero-padded to Wp, a multiple of 4, so
// the last taps add zeros).
constexpr int kGradTY = 64, kGradTX = 128, kGradTmplFrames = 8;

__host__ __device__ constexpr int grad_wp(int W) { return (W + 3) / 4 * 4; }

static __global__ void __launch_bounds__(kGradThreads)
k_grad_tmpl(const uint16_t* __restrict__ frames, int64_t T, int m, int n, int wm1, const float* __restrict__ G,
            const double* __restrict__ inv_area, float scale, const int32_t* __restrict__ coff,
            float* __restrict__ acc_out) {
    extern __shared__ __align__(16) float sm[];
    const int W = 2 * wm1 + 1, K = W * W, Wp = grad_wp(W);
    const int Hy = kGradTY + 2 * wm1, Hx = kGradTX + Wp;  // halo rows, padded halo row length
    float* halo = sm;                                      // Hy x Hx
    float* q = sm + Hy * Hx;                               // W x Wp
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * kGradTY, j0 = blockIdx.x * kGradTX;
    const int ty = tid >> 4, tx = tid & 15;  // outputs (ty*4 + r, tx*8 + x)
    const float c = (float)*coff;
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int x = 0; x < 8; ++x) acc[r][x] = 0.f;
    const int64_t f_begin = (int64_t)blockIdx.z * kGradTmplFrames;
    const int64_t f_end = (T < f_begin + kGradTmplFrames) ? T : f_begin + kGradTmplFrames;
    for (int64_t f = f_begin; f < f_end; ++f) {
        __syncthreads();
        const uint16_t* a = frames + f * (int64_t)m * n;
        for (int r = tid >> 5; r < Hy; r += kGradThreads / 32) {
            const int ai = i0 - wm1 + r;
            for (int cc = tid & 31; cc < Hx; cc += 32) {
                const int aj = j0 - wm1 + cc;
                halo[r * Hx + cc] = (cc < kGradTX + W - 1 && ai >= 0 && ai < m && aj >= 0 && aj < n)
                                        ? (float)a[(int64_t)ai * n + aj] - c : 0.f;
            }
        }
        for (int k = tid; k < W * Wp; k += kGradThreads) {
            const int si = k / Wp, ti = k - si * Wp;
            q[k] = ti < W ? scale * G[f * K + si * W + ti] * (float)inv_area[si * W + ti] : 0.f;
        }
        __syncthreads();
        for (int s = 0; s < W; ++s) {
            const float* qrow = q + s * Wp;
            float win[4][12];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float* hp = halo + (ty * 4 + r + s) * Hx + tx * 8;
                const float4 v0 = *reinterpret_cast<const float4*>(hp);
                const float4 v1 = *reinterpret_cast<const float4*>(hp + 4);
                win[r][0] = v0.x; win[r][1] = v0.y; win[r][2] = v0.z; win[r][3] = v0.w;
                win[r][4] = v1.x; win[r][5] = v1.y; win[r][6] = v1.z; win[r][7] = v1.w;
            }
            for (int t0 = 0; t0 < Wp; t0 += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(qrow + t0);
                const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float4 v = *reinterpret_cast<const float4*>(halo + (ty * 4 + r + s) * Hx + tx * 8 + t0 + 8);
                    win[r][8] = v.x; win[r][9] = v.y; win[r][10] = v.z; win[r][11] = v.w;
#pragma unroll
                    for (int dt = 0; dt < 4; ++dt)
#pragma unroll
                        for (int x = 0; x < 8; ++x) acc[r][x] = fmaf(qv[dt], win[r][x + dt], acc[r][x]);
#pragma unroll
                    for (int x = 0; x < 8; ++x) win[r][x] = win[r][x + 4];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int j = j0 + tx * 8 + x;
            if (i < m && j < n) atomicAdd(&acc_out[(int64_t)i * n + j], acc[r][x]);
        }
    }
}

// dL/db[i][j] += -2 acc[i][j] + 2 b'[i][j] * sum of Q over the shifts whose
// overlap contains (i, j).
static __global__ void __launch_bounds__(256)
k_grad_tmpl_finish(const float* __restrict__ acc, const float* __restrict__ Q, int m, int n, int wm1,
                   const void* __restrict__ tmpl, int tmpl_f32, const int32_t* __restrict__ coff,
                   float* __restrict__ grad) {
    extern __shared__ __align__(16) float P[];
    const int W = 2 * wm1 + 1;
    prefix2d(Q, P, W, threadIdx.x, blockDim.x);
    const float c = (float)*coff;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (int64_t)m * n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / n), j = (int)(p % n);
        const float bv = tmpl_f32 ? static_cast<const float*>(tmpl)[p] : (float)static_cast<const uint16_t*>(tmpl)[p];
        const float cover = rect(P, W, wm1, max(-wm1, -i), min(wm1, m - 1 - i), max(-wm1, -j), min(wm1, n - 1 - j));
        grad[p] += -2.f * acc[p] + 2.f * (bv - c) * cover;
    }
}

// dL/da_f for one 32 x 32 tile of one frame. Grid (tiles_x, tiles_y, T).
static __global__ void __launch_bounds__(kGradThreads)
k_grad_frames(const uint16_t* __restrict__ frames, int m, int n, int wm1, const float* __restrict__ G,
              const double* __restrict__ inv_area, float scale, const void* __restrict__ tmpl, int tmpl_f32,
              const int32_t* __restrict__ coff, float* __restrict__ grad_frames) {
    extern __shared__ __align__(16) float sm[];
    const int W = 2 * wm1 + 1, K = W * W, L = W + 1;
    const int H = kGradTile + 2 * wm1;
    float* halo = sm;         // H x H: b' around the tile
    float* q = sm + H * H;    // K, stored flipped: qf[(wm1-s)][(wm1-t)]
    float* P = q + K;         // (W+1)^2 prefix of q (unflipped)
    float* qraw = P + L * L;  // K
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * kGradTile, j0 = blockIdx.x * kGradTile;
    const int64_t f = blockIdx.z;
    const float c = (float)*coff;
    for (int k = tid; k < H * H; k += kGradThreads) {
        const int r = k / H, cc = k - r * H;
        const int bi = i0 - wm1 + r, bj = j0 - wm1 + cc;
        float v = 0.f;
        if (bi >= 0 && bi < m && bj >= 0 && bj < n) {
            const int64_t p = (int64_t)bi * n + bj;
            v = (tmpl_f32 ? static_cast<const float*>(tmpl)[p] : (float)static_cast<const uint16_t*>(tmpl)[p]) - c;
        }
        halo[k] = v;
    }
    for (int k = tid; k < K; k += kGradThreads) {
        const float qv = scale * G[f * K + k] * (float)inv_area[k];
        qraw[k] = qv;
        q[K - 1 - k] = qv;  // flip both shift axes
    }
    __syncthreads();
    prefix2d(qraw, P, W, tid, kGradThreads);
    // sum_st q_st b'[k-s][l-t] = sum_{s',t'} qflip[s'][t'] b'[k-wm1+s'][l-wm1+t']
    const int ty = tid >> 3, tx = (tid & 7) * 4;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int s = 0; s < W; ++s) {
        const float* hrow = halo + (ty + s) * H + tx;
        const float* qrow = q + s * W;
        float seg[4];
#pragma unroll
        for (int x = 0; x < 3; ++x) seg[x] = hrow[x];
        for (int t = 0; t < W; ++t) {
            seg[3] = hrow[t + 3];
            const float qv = qrow[t];
#pragma unroll
            for (int x = 0; x < 4; ++x) acc[x] = fmaf(qv, seg[x], acc[x]);
#pragma unroll
            for (int x = 0; x < 3; ++x) seg[x] = seg[x + 1];
        }
    }
    const int k = i0 + ty;
    const uint16_t* a = frames + f * (int64_t)m * n;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int l = j0 + tx + x;
        if (k < m && l < n) {
            // shifts (s, t) with (k - s, l - t) inside the template
            const float cover = rect(P, W, wm1, max(-wm1, k - m + 1), min(wm1, k), max(-wm1, l - n + 1), min(wm1, l));
            const float av = (float)a[(int64_t)k * n + l] - c;
            grad_frames[f * (int64_t)m * n + (int64_t)k * n + l] = 2.f * av * cover - 2.f * acc[x];
        }
    }
}

}  // namespace moco
