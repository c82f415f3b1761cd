// Device kernels of the translation search (Section 2 of the paper).
//
// For one frame a and the template b (both on the searched grid, offset by
// the plan's integer c) every shift max(|s|,|t|) < w gets
//     Area(D_st) f_st = Sa_st + Sb_st - 2 h_st                  (Section 2)
// with Sa, Sb the energies of a and b over D_st (exact int64 here, the
// paper's dynamic-programming sums restricted to the window) and h the
// cross-correlation, computed through zero-padded 2-D FFTs (Section 2):
//   k_frame_rows : 2x2 box (exact integer 4-sum), subtract c, energies of the
//                  edge strips and corners, real row FFTs (length Nc) -> X
//   k_cols       : column FFT (length Nr), x conj(template spectrum), inverse
//                  column FFT kept on the 2w-1 needed rows -> Y
//   k_rows_inv   : inverse row FFTs kept on the 2w-1 needed columns -> h;
//                  Sa for every shift from totals, edge strips and corners
//                  (energy_frame); f = (Sa + Sb - 2h) / Area in FP32 from
//                  exact energies; argmin with tie-break
//   k_energy     : the same energies stored (template, direct form)
//   k_jitter     : Section 2's upsampling step: the 3x3 candidates around the
//                  doubled optimum, exact int64 sums at full resolution
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "fft.cuh"
#include "ptx.cuh"

namespace moco {

typedef unsigned long long u64;

constexpr int kRowsThreads = 512;
constexpr int kRC = 32;          // searched-grid rows per chunk of k_frame_rows
constexpr int kColsVC = 16;      // spectral columns per CTA of k_cols
constexpr int kInvPC = 16;       // row pairs per chunk of k_rows_inv
constexpr int kEnergyThreads = 256;
constexpr int kJitterThreads = 256;

template <bool F32>
struct AccT { typedef u64 type; };
template <>
struct AccT<true> { typedef double type; };

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t lo16(uint32_t w) { return w & 0xffffu; }
// d^2 exactly, |d| < 2^32: one 32x32 -> 64-bit unsigned multiply.
__device__ __forceinline__ u64 sq64(int32_t d) {
    const uint32_t a = (uint32_t)abs(d);
    return (u64)a * (u64)a;
}
__device__ __forceinline__ uint32_t hi16(uint32_t w) { return w >> 16; }
// acc + (low half-word of w) + (high half-word of w), one dp2a.
__device__ __forceinline__ uint32_t add_halves(uint32_t w, uint32_t acc) {
    asm("dp2a.lo.u32.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(w), "r"(0x0101u));
    return acc;
}
// Sum of the 2^LV x 2^LV full-resolution pixels behind level-LV pixel (r, c)
// (LV >= 1; below 2^32 for LV <= 4): each of the block's 2^LV rows read by one
// aligned 4-, 8- or 16-byte load (two at LV = 4; n % 8 == 0, the image
// 16-byte aligned).
template <int LV>
__device__ __forceinline__ uint32_t box_sum_vec(const uint16_t* __restrict__ img, int n, int r, int c) {
    constexpr int B = 1 << LV;
    const uint16_t* p0 = img + ((int64_t)r << LV) * n + ((int64_t)c << LV);
    uint32_t s = 0;
#pragma unroll
    for (int dr = 0; dr < B; ++dr) {
        const uint16_t* p = p0 + (int64_t)dr * n;
        if constexpr (B == 2) {
            s = add_halves(__ldg(reinterpret_cast<const uint32_t*>(p)), s);
        } else if constexpr (B == 4) {
            const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
            s = add_halves(q.x, add_halves(q.y, s));
        } else {
#pragma unroll
            for (int h = 0; h < B / 8; ++h) {
                const uint4 q = __ldg(reinterpret_cast<const uint4*>(p) + h);
                s = add_halves(q.x, add_halves(q.y, add_halves(q.z, add_halves(q.w, s))));
            }
        }
    }
    return s;
}
// The same at a level known at run time (1 <= L <= 4).
__device__ __forceinline__ uint32_t box_sum_l(const uint16_t* __restrict__ img, int n, int r, int c, int L) {
    switch (L) {  // the same for every thread of a launch
        case 1: return box_sum_vec<1>(img, n, r, c);
        case 2: return box_sum_vec<2>(img, n, r, c);
        case 3: return box_sum_vec<3>(img, n, r, c);
        default: return box_sum_vec<4>(img, n, r, c);
    }
}
// acc += d * d exactly (|d| < 2^31), one 32 x 32 -> 64-bit multiply-add.
__device__ __forceinline__ void add_sq(u64& acc, int32_t d) {
    asm("mad.wide.s32 %0, %1, %1, %0;" : "+l"(acc) : "r"(d));
}

// ---------------------------------------------------------------------------
// k_frame_rows: one CTA per image (frame or template).
//
// src        : images, element stride src_fstride between them; uint16
//              (frames, U16 template) or float (F32 template, levels = 0)
// levels     : 1 = one 2x2 box level (4-sum), 0 = none
// coff       : the plan's integer offset c (int32 for U16, float for F32)
// X          : X[f*x_fstride + v*ldx + r], v in [0, Nc/2], r in [0, mc): the
//              row DFT of the offset searched-grid rows
// rowE, colE : per-row / per-column energies (only the 2(w-1) edge rows and
//              columns are written), tot: total energy, all as 64-bit words
//              (u64 for integer images, double for F32)
// corners    : the four (w-1)x(w-1) corner blocks of the offset image
//              (int32 or float bits), [f][q][ri][ci], q = 2*bottom + right
//
// PLANES (the direct form): no FFT; the offset searched-grid image is written
// as BF16 hi and lo planes instead, planes[f][r][c] with row length ldp
// (columns nc .. ldp-1 written as zeros).
// STAGED (uint16 frames, FFT mode; n % 8 == 0): the full-resolution rows of
// each chunk of kRC searched rows are brought into shared memory by bulk
// asynchronous copies (one mbarrier), the next chunk's while this chunk's
// transforms run; the loader then reads shared memory. A wait that gives up
// (about a second) sets *err and ends the CTA after one more bounded wait.
template <int N, bool F32IN>
__host__ __device__ constexpr size_t frame_rows_smem_base(int nc) {
    return (sizeof(float2) * ((kRC / 2) * fft_ld<N>() + N) + sizeof(typename AccT<F32IN>::type) * (kRC + nc) + 127) /
           128 * 128;
}
__host__ __device__ constexpr size_t frame_rows_stage_bytes(int n, int levels) {
    return (size_t)(levels ? 2 : 1) * kRC * n * 2;
}
constexpr uint32_t kStageCopyBytes = 16384;  // bulk copies of at most 16 KiB each

// Staged passes at N >= 512 hold more than half of an SM's shared memory
// (n > 2 (N_prev - 127) columns of staged rows beside the transform buffer):
// one CTA per SM, so the registers are not capped for two.
template <int N, bool STAGED>
__host__ __device__ constexpr int frame_rows_min_blocks() { return STAGED && N >= 512 ? 1 : 2; }

template <int N, bool F32IN, bool PLANES = false, bool STAGED = false>
__global__ void __launch_bounds__(kRowsThreads, frame_rows_min_blocks<N, STAGED>())
k_frame_rows(const void* __restrict__ src, int64_t src_fstride, int m, int n, int levels, int mc,
             int nc, const int32_t* __restrict__ coff_i, const float* __restrict__ coff_f,
             const float2* __restrict__ tw_g, float2* __restrict__ X, int64_t x_fstride, int ldx,
             u64* __restrict__ rowE, u64* __restrict__ colE, u64* __restrict__ tot,
             uint32_t* __restrict__ corners, int wm1, __nv_bfloat16* __restrict__ p_hi = nullptr,
             __nv_bfloat16* __restrict__ p_lo = nullptr, int ldp = 0, unsigned int* __restrict__ err = nullptr,
             int split = 0) {
    static_assert(!STAGED || (!F32IN && !PLANES), "staging is for uint16 frames in FFT mode");
    typedef typename AccT<F32IN>::type Acc;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();                      // skewed, padded row
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // (kRC/2) x LD
    float2* tw = buf + (kRC / 2) * LD;                   // N: forward table
    Acc* rowacc = reinterpret_cast<Acc*>(tw + N);        // kRC
    Acc* colacc = rowacc + kRC;                          // nc
    __shared__ Acc red[32];
    __shared__ __align__(8) uint64_t stage_bar;
    __shared__ int s_abort;
    __shared__ int spos[PLANES ? 1 : N];  // buffer slot of spectral index k
    const uint16_t* stage = reinterpret_cast<const uint16_t*>(smem_raw + frame_rows_smem_base<N, F32IN>(nc));
    // Issues the bulk copies of the chunk at searched row c0 (one thread).
    auto issue_chunk = [&](int c0) {
        const int rows = min(kRC, mc - c0) * (levels ? 2 : 1);
        const uint32_t bytes = (uint32_t)rows * (uint32_t)n * 2u;
        const unsigned char* g = reinterpret_cast<const unsigned char*>(static_cast<const uint16_t*>(src) +
                                                                        (split ? 0 : blockIdx.x) * src_fstride +
                                                                        (int64_t)c0 * (levels ? 2 : 1) * n);
        unsigned char* d = smem_raw + frame_rows_smem_base<N, F32IN>(nc);
        mbar_expect_tx(&stage_bar, bytes);
        for (uint32_t off = 0; off < bytes; off += kStageCopyBytes)
            bulk_g2s(d + off, g + off, min(kStageCopyBytes, bytes - off), &stage_bar);
    };

    const int tid = threadIdx.x, nthr = blockDim.x;
    // split: one image, one chunk of kRC searched rows per CTA; its partial
    // total and edge-column energies go to slot blockIdx.x.
    const int64_t f = split ? 0 : blockIdx.x;
    const int r_begin = split ? (int)blockIdx.x * kRC : 0;
    const int r_end = split ? min(mc, r_begin + kRC) : mc;
    const int64_t slot_out = blockIdx.x;
    if (STAGED) {
        if (tid == 0) {
            mbar_init(&stage_bar, 1);
            s_abort = 0;
            fence_async_smem();
            issue_chunk(r_begin);
        }
    }
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[i];
    if (!PLANES)
        for (int k = tid; k < N; k += nthr) spos[k] = sk<N>(spec_pos<N>(k));
    for (int i = tid; i < nc; i += nthr) colacc[i] = 0;
    for (int i = tid; i < kRC; i += nthr) rowacc[i] = 0;

    const int CW = (levels ? 4 : 8);  // searched-grid values per thread per row
    const int G = nc / CW;             // column groups per row
    const int RPI = nthr / G;          // rows per pass (host guarantees G <= nthr)
    const bool active = tid < RPI * G;
    const int g = tid % G, rl0 = tid / G;
    Acc tacc = 0;
    const int32_t ci_off = F32IN ? 0 : *coff_i;
    const float cf_off = F32IN ? *coff_f : 0.f;
    const size_t wm1sq = (size_t)wm1 * wm1;

    // FFT-mode loader: a thread owns one column c of a row pair (rows 2p and
    // 2p+1 of the chunk, packed as one complex value), so consecutive threads
    // write consecutive 8-byte words of the transform buffer. Its column set
    // is the same in every chunk: edge-column energies stay in registers.
    const int CS = (nc + nthr - 1) / nthr;  // column slots per thread (nc > nthr)
    const int PPI = nc <= nthr ? nthr / nc : 1;
    const bool warp_rows = (nc % 32 == 0);  // every warp then shares one row pair
    Acc colreg[4] = {0, 0, 0, 0};

    for (int r0 = r_begin; r0 < r_end; r0 += kRC) {
        const int rows = min(kRC, mc - r0), nfft = (rows + 1) >> 1;
        if constexpr (!PLANES) {
            for (int i = tid; i < nfft * (N - nc); i += nthr) {
                const int pr = i / (N - nc), cc = nc + (i - pr * (N - nc));
                buf[pr * LD + sk<N>(cc)] = make_float2(0.f, 0.f);
            }
            if (STAGED) {
                __syncthreads();  // s_abort and the barrier's set-up are visible
                if (!mbar_wait(&stage_bar, (uint32_t)(((r0 - r_begin) / kRC) & 1), err)) s_abort = 1;
                __syncthreads();
                if (s_abort) {
                    if (tid == 0) mbar_wait(&stage_bar, (uint32_t)(((r0 - r_begin) / kRC) & 1), err);
                    return;
                }
            }
            if constexpr (STAGED) {
                // Staged uint16 frames (the host guarantees nc <= nthr): one
                // column c per thread, row pairs p0, p0 + PPI, ... of the chunk.
                // The 2x2 box sums come from dp2a, the float value from the
                // exact 2^23 bias (|d| < 2^19), the squares from 64-bit
                // multiply-adds; an edge row's sum over a warp is two 32-bit
                // reductions of the 18-bit halves of d^2 (< 2^36).
                const int c = tid % nc, p0 = tid / nc;
                if (p0 < PPI) {
                    const int skc = sk<N>(c);
                    const bool ecol = c < wm1 || c >= nc - wm1;
                    const int hw = n >> 1;
                    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(stage);
                    const int bias = 0x4B400000 - ci_off;  // float bits of 2^23 + 2^22 + d
                    // Only chunks that hold an edge row (r < w-1 or r >= mc-(w-1))
                    // have per-row energies or corner values to record.
                    const bool edge_chunk = r0 < wm1 || r0 + rows > mc - wm1;
                    if (levels && !edge_chunk && rows == kRC) {
                        // A full chunk without edge rows (most of them): box sums,
                        // values and the energies of the total and the edge
                        // columns only, by pointers that step a row pair at a time.
                        const uint32_t* q = s32 + (size_t)(4 * p0) * hw + c;
                        float2* bq = buf + p0 * LD + skc;
                        const int qstep = 4 * PPI * hw, bstep = PPI * LD;
#pragma unroll 4
                        for (int pr = p0; pr < nfft; pr += PPI, q += qstep, bq += bstep) {
                            const int s0 = (int)add_halves(q[0], add_halves(q[hw], 0u));
                            const int s1 = (int)add_halves(q[2 * hw], add_halves(q[3 * hw], 0u));
                            *bq = make_float2(__int_as_float(s0 + bias) - 12582912.0f,
                                              __int_as_float(s1 + bias) - 12582912.0f);
                            const int d0 = s0 - ci_off, d1 = s1 - ci_off;
                            add_sq(tacc, d0);
                            add_sq(tacc, d1);
                            if (ecol) {
                                add_sq(colreg[0], d0);
                                add_sq(colreg[0], d1);
                            }
                        }
                    } else if (levels && rows == kRC && warp_rows) {
                        // A full chunk with edge rows: the same, plus each edge row's
                        // energy (a warp holds one row pair: two 32-bit warp sums of
                        // the 18-bit halves of d^2, added by lane 0) and, in the edge
                        // columns, its corner values.
                        const uint32_t* q = s32 + (size_t)(4 * p0) * hw + c;
                        float2* bq = buf + p0 * LD + skc;
                        const int qstep = 4 * PPI * hw, bstep = PPI * LD;
                        const int cj = c >= nc - wm1 ? c - (nc - wm1) : c, qc = c >= nc - wm1 ? 1 : 0;
                        for (int pr = p0; pr < nfft; pr += PPI, q += qstep, bq += bstep) {
                            const int s0 = (int)add_halves(q[0], add_halves(q[hw], 0u));
                            const int s1 = (int)add_halves(q[2 * hw], add_halves(q[3 * hw], 0u));
                            *bq = make_float2(__int_as_float(s0 + bias) - 12582912.0f,
                                              __int_as_float(s1 + bias) - 12582912.0f);
                            const int d0 = s0 - ci_off, d1 = s1 - ci_off;
                            add_sq(tacc, d0);
                            add_sq(tacc, d1);
                            if (ecol) {
                                add_sq(colreg[0], d0);
                                add_sq(colreg[0], d1);
                            }
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int rr = r0 + 2 * pr + h;  // the same for the whole warp
                                const bool top = rr < wm1, bot = rr >= mc - wm1;
                                if (!(top || bot)) continue;
                                const int dh = h ? d1 : d0;
                                const u64 eh = (u64)((long long)dh * dh);
                                const uint32_t lo = __reduce_add_sync(0xffffffffu, (uint32_t)(eh & 0x3ffffu));
                                const uint32_t hi = __reduce_add_sync(0xffffffffu, (uint32_t)(eh >> 18));
                                if ((tid & 31) == 0) atomicAdd(&rowacc[2 * pr + h], ((u64)hi << 18) + lo);
                                if (ecol) {
                                    const int ri = top ? rr : rr - (mc - wm1);
                                    corners[(f * 4 + (bot ? 2 : 0) + qc) * wm1sq + (size_t)ri * wm1 + cj] = (uint32_t)dh;
                                }
                            }
                        }
                    } else
                    for (int pr = p0; pr < nfft; pr += PPI) {
                        const int rl = 2 * pr;
                        const bool has1 = rl + 1 < rows;  // the same for the whole warp
                        int s0, s1;
                        if (levels) {
                            const uint32_t* q = s32 + (2 * rl) * hw + c;
                            s0 = (int)add_halves(q[0], add_halves(q[hw], 0u));
                            s1 = has1 ? (int)add_halves(q[2 * hw], add_halves(q[3 * hw], 0u)) : ci_off;
                        } else {
                            s0 = stage[rl * n + c];
                            s1 = has1 ? (int)stage[(rl + 1) * n + c] : ci_off;
                        }
                        const int d0 = s0 - ci_off, d1 = s1 - ci_off;  // d1 = 0 past the last row
                        buf[pr * LD + skc] = make_float2(__int_as_float(s0 + bias) - 12582912.0f,
                                                         __int_as_float(s1 + bias) - 12582912.0f);
                        add_sq(tacc, d0);
                        add_sq(tacc, d1);
                        if (ecol) {
                            add_sq(colreg[0], d0);
                            add_sq(colreg[0], d1);
                        }
                        if (edge_chunk)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (h == 1 && !has1) break;
                            const int rr = r0 + rl + h;
                            const bool top = rr < wm1, bot = rr >= mc - wm1;
                            if (!(top || bot)) continue;
                            const int dh = h ? d1 : d0;
                            const u64 eh = (u64)((long long)dh * dh);
                            if (warp_rows) {
                                const uint32_t lo = __reduce_add_sync(0xffffffffu, (uint32_t)(eh & 0x3ffffu));
                                const uint32_t hi = __reduce_add_sync(0xffffffffu, (uint32_t)(eh >> 18));
                                if ((tid & 31) == 0) atomicAdd(&rowacc[rl + h], ((u64)hi << 18) + lo);
                            } else {
                                atomicAdd(&rowacc[rl + h], eh);
                            }
                            if (ecol) {
                                const int ri = top ? rr : rr - (mc - wm1);
                                const int cj = c >= nc - wm1 ? c - (nc - wm1) : c;
                                const int q = (bot ? 2 : 0) + (c >= nc - wm1 ? 1 : 0);
                                corners[(f * 4 + q) * wm1sq + (size_t)ri * wm1 + cj] = (uint32_t)dh;
                            }
                        }
                    }
                }
            } else
#pragma unroll
            for (int slot = 0; slot < 4; ++slot) {
                if (slot >= CS) break;
                int c, p0;
                if (nc <= nthr) {
                    c = tid % nc;
                    p0 = tid / nc;
                    if (p0 >= PPI) break;
                } else {
                    c = tid + slot * nthr;
                    p0 = 0;
                    if (c >= nc) break;
                }
                const bool left = c < wm1, right = c >= nc - wm1;
                for (int pr = p0; pr < nfft; pr += PPI) {
                    const int rl = 2 * pr, r = r0 + rl;
                    const bool has1 = rl + 1 < rows;
                    float v[2];
                    if (!F32IN) {
                        const uint16_t* base = static_cast<const uint16_t*>(src) + f * src_fstride;
                        int32_t iv[2] = {0, 0};
                        if (levels) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                if (h == 1 && !has1) break;
                                uint32_t w0, w1;
                                if (STAGED) {
                                    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(stage);
                                    w0 = s32[(2 * (rl + h)) * (n / 2) + c];
                                    w1 = s32[(2 * (rl + h) + 1) * (n / 2) + c];
                                } else if (levels > 1) {
                                    iv[h] = (int32_t)box_sum_l(base, n, r + h, c, levels);
                                    continue;
                                } else {
                                    w0 = __ldg(reinterpret_cast<const uint32_t*>(base + (int64_t)(2 * (r + h)) * n + 2 * c));
                                    w1 = __ldg(reinterpret_cast<const uint32_t*>(base + (int64_t)(2 * (r + h) + 1) * n + 2 * c));
                                }
                                iv[h] = (int32_t)(lo16(w0) + hi16(w0) + lo16(w1) + hi16(w1));
                            }
                        } else if (STAGED) {
                            iv[0] = (int32_t)stage[rl * n + c];
                            if (has1) iv[1] = (int32_t)stage[(rl + 1) * n + c];
                        } else {
                            iv[0] = (int32_t)__ldg(base + (int64_t)r * n + c);
                            if (has1) iv[1] = (int32_t)__ldg(base + (int64_t)(r + 1) * n + c);
                        }
                        v[0] = (float)(iv[0] - ci_off);
                        v[1] = has1 ? (float)(iv[1] - ci_off) : 0.f;
                    } else {
                        const float* base = static_cast<const float*>(src) + f * src_fstride;
                        v[0] = __ldg(base + (int64_t)r * n + c) - cf_off;
                        v[1] = has1 ? __ldg(base + (int64_t)(r + 1) * n + c) - cf_off : 0.f;
                    }
                    buf[pr * LD + sk<N>(c)] = make_float2(v[0], v[1]);
                    Acc e[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (F32IN) e[h] = (Acc)((double)v[h] * (double)v[h]);
                        else e[h] = (Acc)sq64((int32_t)v[h]);
                    }
                    tacc += e[0] + e[1];
                    if (left || right) colreg[slot] += e[0] + e[1];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rr = r + h;
                        if (h == 1 && !has1) break;
                        const bool top = rr < wm1, bot = rr >= mc - wm1;
                        if (!(top || bot)) continue;
                        if (warp_rows) {
                            const Acc sum = warp_sum(e[h]);
                            if ((tid & 31) == 0) atomicAdd(&rowacc[rl + h], sum);
                        } else {
                            atomicAdd(&rowacc[rl + h], e[h]);
                        }
                        if (left || right) {
                            const int ri = top ? rr : rr - (mc - wm1);
                            const int cj = right ? c - (nc - wm1) : c;
                            const int q = (bot ? 2 : 0) + (right ? 1 : 0);
                            const uint32_t bits = F32IN ? __float_as_uint(v[h]) : (uint32_t)(int32_t)v[h];
                            corners[(f * 4 + q) * wm1sq + (size_t)ri * wm1 + cj] = bits;
                        }
                    }
                }
            }
        } else {
        __syncthreads();
        if (active) {
            for (int rl = rl0; rl < rows; rl += RPI) {
                const int r = r0 + rl;
                float val[8];
                if (!F32IN) {
                    const uint16_t* base = static_cast<const uint16_t*>(src) + f * src_fstride;
                    int32_t iv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (levels) {
                        const uint4 p0 = __ldg(reinterpret_cast<const uint4*>(base + (int64_t)(2 * r) * n + 8 * g));
                        const uint4 p1 = __ldg(reinterpret_cast<const uint4*>(base + (int64_t)(2 * r + 1) * n + 8 * g));
                        const uint32_t w0[4] = {p0.x, p0.y, p0.z, p0.w}, w1[4] = {p1.x, p1.y, p1.z, p1.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            iv[k] = (int32_t)(lo16(w0[k]) + hi16(w0[k]) + lo16(w1[k]) + hi16(w1[k]));
                    } else {
                        const uint4 p0 = __ldg(reinterpret_cast<const uint4*>(base + (int64_t)r * n + 8 * g));
                        const uint32_t w0[4] = {p0.x, p0.y, p0.z, p0.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            iv[2 * k] = (int32_t)lo16(w0[k]);
                            iv[2 * k + 1] = (int32_t)hi16(w0[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) val[k] = (float)(iv[k] - ci_off);  // |d| < 2^19: exact
                } else {
                    const float* base = static_cast<const float*>(src) + f * src_fstride;
                    const float4 q0 = __ldg(reinterpret_cast<const float4*>(base + (int64_t)r * n + 8 * g));
                    const float4 q1 = __ldg(reinterpret_cast<const float4*>(base + (int64_t)r * n + 8 * g + 4));
                    val[0] = q0.x - cf_off; val[1] = q0.y - cf_off; val[2] = q0.z - cf_off; val[3] = q0.w - cf_off;
                    val[4] = q1.x - cf_off; val[5] = q1.y - cf_off; val[6] = q1.z - cf_off; val[7] = q1.w - cf_off;
                }
                const bool top = r < wm1, bot = r >= mc - wm1;
                Acc rs = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (k >= CW) break;
                    const int c = g * CW + k;
                    Acc e;
                    if (F32IN) e = (Acc)((double)val[k] * (double)val[k]);
                    else e = (Acc)sq64((int32_t)val[k]);
                    rs += e;
                    const bool left = c < wm1, right = c >= nc - wm1;
                    if (left || right) {
                        atomicAdd(&colacc[c], e);  // column energies: edge columns only
                        if (top || bot) {
                            const int ri = top ? r : r - (mc - wm1);
                            const int cj = right ? c - (nc - wm1) : c;
                            const int q = (bot ? 2 : 0) + (right ? 1 : 0);
                            const uint32_t bits = F32IN ? __float_as_uint(val[k]) : (uint32_t)(int32_t)val[k];
                            corners[(f * 4 + q) * wm1sq + (size_t)ri * wm1 + cj] = bits;
                        }
                    }
                }
                tacc += rs;
                if (top || bot) atomicAdd(&rowacc[rl], rs);
                if constexpr (PLANES) {
                    if (g == 0)  // the padding columns nc .. ldp-1 must read as zero
                        for (int c = nc; c < ldp; ++c) {
                            p_hi[(f * mc + r) * (int64_t)ldp + c] = __float2bfloat16_rn(0.f);
                            p_lo[(f * mc + r) * (int64_t)ldp + c] = __float2bfloat16_rn(0.f);
                        }
                    __nv_bfloat16* ph = p_hi + (f * mc + r) * (int64_t)ldp + g * CW;
                    __nv_bfloat16* pl = p_lo + (f * mc + r) * (int64_t)ldp + g * CW;
                    // CW (4 or 8) consecutive values per plane: one 8- or 16-byte store each
                    // (ldp and g * CW are multiples of CW, the planes 256-byte aligned)
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int k = 0; k < 8; k += 2) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(val[k]), h1 = __float2bfloat16_rn(val[k + 1]);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(val[k] - __bfloat162float(h0));
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(val[k + 1] - __bfloat162float(h1));
                        hw[k / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        lw[k / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                    }
                    if (CW == 4) {
                        *reinterpret_cast<uint2*>(ph) = make_uint2(hw[0], hw[1]);
                        *reinterpret_cast<uint2*>(pl) = make_uint2(lw[0], lw[1]);
                    } else {
                        *reinterpret_cast<uint4*>(ph) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(pl) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                } else {
                    float* dst = reinterpret_cast<float*>(buf + (rl >> 1) * LD) + (rl & 1);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (k < CW) dst[2 * (g * CW + k)] = val[k];
                }
            }
        }
        }
        __syncthreads();
        if (STAGED && tid == 0 && r0 + kRC < r_end) {
            fence_async_smem();  // this chunk's reads of the stage come before the next copies
            issue_chunk(r0 + kRC);
        }
        if constexpr (!PLANES) {
        fft4_fwd<N>(buf, LD, nfft, tw, tid, nthr);
        // Two real rows were packed as one complex row: split the spectra.
        constexpr int NH = N / 2 + 1;
        constexpr int PC = kRC / 2;  // row pairs of a full chunk
        for (int task = tid; task < NH * PC; task += nthr) {
            const int v = task / PC, fi = task % PC;
            if (fi >= nfft) continue;
            const float2 zk = buf[fi * LD + spos[v]];
            const float2 zn = cconj(buf[fi * LD + spos[v == 0 ? 0 : N - v]]);
            const float2 x1 = cscale(cadd(zk, zn), 0.5f);
            const float2 d = csub(zk, zn);
            const float2 x2 = make_float2(0.5f * d.y, -0.5f * d.x);
            float2* out = X + f * x_fstride + (int64_t)v * ldx + r0 + 2 * fi;
            if (2 * fi + 1 < rows)
                *reinterpret_cast<float4*>(out) = make_float4(x1.x, x1.y, x2.x, x2.y);
            else
                out[0] = x1;
        }
        }
        for (int rl = tid; rl < rows; rl += nthr) {
            const int r = r0 + rl;
            if (r < wm1 || r >= mc - wm1) {
                Acc v = rowacc[rl];
                rowE[f * mc + r] = *reinterpret_cast<u64*>(&v);
            }
            rowacc[rl] = 0;
        }
        __syncthreads();
    }
    if constexpr (!PLANES) {
#pragma unroll
        for (int slot = 0; slot < 4; ++slot) {
            if (slot >= CS) break;
            int c;
            if (nc <= nthr) {
                c = tid % nc;
                if (tid / nc >= PPI) break;
            } else {
                c = tid + slot * nthr;
                if (c >= nc) break;
            }
            if (c < wm1 || c >= nc - wm1) atomicAdd(&colacc[c], colreg[slot]);
        }
    }
    __syncthreads();
    tacc = warp_sum(tacc);
    if ((tid & 31) == 0) red[tid >> 5] = tacc;
    __syncthreads();
    if (tid == 0) {
        Acc s = 0;
        for (int i = 0; i < (nthr + 31) / 32; ++i) s += red[i];
        tot[slot_out] = *reinterpret_cast<u64*>(&s);
    }
    for (int c = tid; c < nc; c += nthr)
        if (c < wm1 || c >= nc - wm1) {
            Acc v = colacc[c];
            colE[slot_out * nc + c] = *reinterpret_cast<u64*>(&v);
        }
}

// After a split single-image k_frame_rows: the slots' partial totals and
// edge-column energies summed, in slot order, into slot 0.
template <bool F32>
__global__ void k_merge_chunks(u64* __restrict__ colE, u64* __restrict__ tot, int chunks, int nc, int wm1) {
    typedef typename AccT<F32>::type Acc;
    for (int c = threadIdx.x; c <= nc; c += blockDim.x) {
        if (c < nc && !(c < wm1 || c >= nc - wm1)) continue;
        u64* p = c < nc ? colE + c : tot;
        const int64_t stride = c < nc ? nc : 1;
        Acc s = 0;
        for (int k = 0; k < chunks; ++k) {
            const u64 b = p[k * stride];
            s += *reinterpret_cast<const Acc*>(&b);
        }
        p[0] = *reinterpret_cast<u64*>(&s);
    }
}

// ---------------------------------------------------------------------------
// k_energy: Sa[s][t] = sum over the a-side of D_st of a'^2 for every shift.
// The a-side of D_st keeps rows [max(0,s), mc+min(0,s)) and columns
// [max(0,t), nc+min(0,t)), i.e. everything but an edge strip of |s| rows and
// one of |t| columns, so
//     Sa = Tot - ExR(s) - ExC(t) + Corner(s,t)
// where the corner term is a 2-D prefix sum over one (w-1)^2 corner block
// (the recurrence of Section 2 restricted to the window). With flip set the
// result is stored at (-s,-t): the template's energy over the b-side of D.
// OUT_DOUBLE stores doubles (exact for integer images); otherwise (uint16
// frames) each exact integer energy is stored as an FP32 pair hi + lo with
// hi = the nearest float and lo = the rounded remainder (|error| <= 8 for
// energies below 2^53, i.e. 2^-48 relative), which the FP32 combine uses.
// The energies of one frame for every shift, computed by the whole block:
// emit(s, t, Sa) once per shift (s, t), |s|, |t| <= wm1. qp corner tables
// (1 or 4) are built per pass: their squares, a prefix along each table row
// (one thread per row), then along each column (one thread per column), so a
// pass takes three barriers. smem (energy_smem): exR, exC (W each) and qp
// tables of w rows x PL of Acc. Every thread of the block must call it (it
// synchronises).
__host__ __device__ constexpr int energy_pl(int wm1) { return (wm1 + 1) | 1; }  // odd row stride
__host__ __device__ constexpr size_t energy_smem(int wm1, size_t acc_bytes, int qp) {
    return acc_bytes * (2 * (2 * wm1 + 1) + (size_t)qp * (wm1 + 1) * energy_pl(wm1));
}
// Quadrants per pass: all four while their tables stay within 64 KiB.
__host__ __device__ constexpr int energy_qp(int wm1, size_t acc_bytes) {
    return energy_smem(wm1, acc_bytes, 4) <= 64 * 1024 ? 4 : 1;
}

template <bool F32, typename Emit>
__device__ __forceinline__ void energy_frame(const u64* __restrict__ rE, const u64* __restrict__ cE, u64 tot_bits,
                                             const uint32_t* __restrict__ corners_f, int mc, int nc, int wm1,
                                             unsigned char* smem, Emit emit) {
    typedef typename AccT<F32>::type Acc;
    const int W = 2 * wm1 + 1, w = wm1 + 1, PL = energy_pl(wm1);
    const int qp = energy_qp(wm1, sizeof(Acc));
    Acc* exR = reinterpret_cast<Acc*>(smem);  // W
    Acc* exC = exR + W;                       // W
    Acc* P = exC + W;                         // qp x w x PL
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    auto ld = [](const u64* p) { u64 v = *p; return *reinterpret_cast<Acc*>(&v); };
    // Edge strips: exR[wm1 + k] = energy of the first k rows, exR[wm1 - k] of
    // the last k rows (k = 1 .. wm1); the same for columns. Warps 0-3.
    if (warp < 4) {
        const u64* src = warp < 2 ? rE : cE;
        const int len = warp < 2 ? mc : nc;
        Acc* dst = warp < 2 ? exR : exC;
        const bool from_end = warp & 1;
        Acc carry = 0;
        if (lane == 0) dst[wm1] = 0;
        for (int k0 = 0; k0 < wm1; k0 += 32) {
            const int k = k0 + lane;  // k + 1 rows or columns
            Acc v = k < wm1 ? ld(src + (from_end ? len - 1 - k : k)) : Acc(0);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Acc u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            v += carry;
            if (k < wm1) dst[from_end ? wm1 - 1 - k : wm1 + 1 + k] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    const Acc T = *reinterpret_cast<const Acc*>(&tot_bits);
    const size_t wm1sq = (size_t)wm1 * wm1;
    for (int q0 = 0; q0 < 4; q0 += qp) {
        const int rows = qp * w;  // table rows of this pass: (q - q0) * w + a
        __syncthreads();
        // P_q[a][b] = sum over the a rows nearest the corner's horizontal edge
        // and the b columns nearest its vertical edge: squares first ...
        for (int r = warp; r < rows; r += nwarps) {
            const int q = q0 + r / w, a = r % w;
            const bool bottom = q >= 2, right = q & 1;
            for (int b = lane; b < w; b += 32) {
                Acc v = 0;
                if (a > 0 && b > 0) {
                    const int ri = bottom ? wm1 - a : a - 1;  // distances from the outer edges
                    const int cj = right ? wm1 - b : b - 1;
                    const uint32_t bits = corners_f[q * wm1sq + (size_t)ri * wm1 + cj];
                    if (F32) {
                        const double x = (double)__uint_as_float(bits);
                        v = (Acc)(x * x);
                    } else {
                        const long long x = (int32_t)bits;
                        v = (Acc)(x * x);
                    }
                }
                P[r * PL + b] = v;
            }
        }
        __syncthreads();
        // ... then along each table row ...
        for (int r = tid; r < rows; r += nthr) {
            Acc* row = P + r * PL;
            Acc run = 0;
            for (int b = 0; b < w; ++b) {
                run += row[b];
                row[b] = run;
            }
        }
        __syncthreads();
        // ... and along each column.
        for (int c = tid; c < rows; c += nthr) {
            Acc* col = P + (c / w) * w * PL + c % w;
            Acc run = 0;
            for (int a = 0; a < w; ++a) {
                run += col[a * PL];
                col[a * PL] = run;
            }
        }
        __syncthreads();
        // Shifts of these quadrants: s >= 0 (top) or s < 0 (bottom), same for t.
        for (int r = warp; r < rows; r += nwarps) {
            const int q = q0 + r / w, a = r % w;
            const bool bottom = q >= 2, right = q & 1;
            if (bottom && a == 0) continue;
            const int s = bottom ? -a : a;
            for (int b = lane; b < w; b += 32) {
                if (right && b == 0) continue;
                const int t = right ? -b : b;
                emit(s, t, T - exR[s + wm1] - exC[t + wm1] + P[r * PL + b]);
            }
        }
    }
}

// x as a float, exact for x < 2^23, without a conversion instruction (the
// bits of 2^23 + x, minus 2^23).
__device__ __forceinline__ float small_u32_to_float(uint32_t x) {
    return __uint_as_float(0x4B000000u | x) - 8388608.0f;
}

// The exact energy e (< 2^53) as an FP32 pair hi + lo. e splits into three
// limbs exact in FP32, e = H 2^32 + M 2^16 + L0 (H < 2^21, M, L0 < 2^16);
// hi + r = H 2^32 + M 2^16 by an error-free sum (TwoSum) and lo = r + L0
// rounds once at |lo| <= 2^-24 |hi| + 2^16: hi + lo is e to within
// 2^-24 |lo|, far below FP32's own resolution of e. 64-bit integer
// conversions run on this part's narrow FP64 pipe; this takes only integer
// logic and FP32 additions.
__device__ __forceinline__ float2 energy_pair(u64 e) {
    const uint32_t H = (uint32_t)(e >> 32), L = (uint32_t)e;
    const float e2 = small_u32_to_float(H) * 4294967296.0f;
    const float e1 = small_u32_to_float(L >> 16) * 65536.0f;
    const float e0 = small_u32_to_float(L & 0xffffu);
    const float hi = e2 + e1;
    const float bb = hi - e2;
    const float r = (e2 - (hi - bb)) + (e1 - bb);
    return make_float2(hi, r + e0);
}

// (double)x for a float, by moving the bits (the same value: every float is a
// double); zero, subnormal, infinite and NaN inputs take the conversion
// instruction, which runs on the narrow FP64 pipe.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)x;
    const u64 bits = ((u64)(u & 0x80000000u) << 32) | ((u64)(ex + 896u) << 52) | ((u64)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// The same energies as energy_frame (integer frames), by warp sweeps instead
// of corner tables in shared memory. For corner quadrant q the table
//     P_q[a][b] = sum over the a rows and b columns nearest q's corner of a'^2
// (a, b < w) is a 2-D prefix sum of the squared corner block. Each lane owns
// K consecutive columns b = K lane + k; the rows [1, w) of a quadrant are
// split into G contiguous segments, one warp each. A warp first sums its
// segment's rows per column and turns that into a prefix along the columns
// (the segment's share of every P_q[a][b] below it), which the warps of
// later segments add as their starting carry; then it walks its rows: each
// row's squares, their prefix along the columns (lane-local, then one warp
// scan of the lane totals), added to the carry, give P_q[a][b] for the row,
// and emit(s, t, Sa) is called for each of its shifts. With a fetch functor,
// fetch(s, t) is called for every shift of the lane's next row while the
// current row is scanned (loads in flight a row ahead), and its value comes
// back as emit(s, t, Sa, value). Every thread of the block must call it (it
// synchronises once); shared memory: energy_sweep_smem(wm1, warps). Needs
// w <= 32 K and at least four warps.
__host__ __device__ constexpr int sweep_groups(int warps) { return warps >= 8 ? warps / 4 : 1; }
__host__ __device__ constexpr size_t energy_sweep_smem(int wm1, int warps) {
    return sizeof(u64) * (2 * (2 * (size_t)wm1 + 1) + 4 * (size_t)sweep_groups(warps) * (wm1 + 1));
}

// No per-shift values to fetch: emit(s, t, Sa).
struct SweepNoFetch {
    struct V {};
    __device__ __forceinline__ V operator()(int, int) const { return V{}; }
};
template <typename Emit>
struct SweepEmit3 {
    Emit& e;
    __device__ __forceinline__ void operator()(int s, int t, u64 sa, SweepNoFetch::V) const { e(s, t, sa); }
};

template <int K, typename Emit, typename Fetch>
__device__ __forceinline__ void energy_sweep_f(const u64* __restrict__ rE, const u64* __restrict__ cE, u64 T,
                                               const uint32_t* __restrict__ corners_f, int mc, int nc, int wm1,
                                               unsigned char* smem, Emit emit, Fetch fetch) {
    using V = decltype(fetch(0, 0));
    const int W = 2 * wm1 + 1, w = wm1 + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int G = sweep_groups(nwarps);
    u64* exR = reinterpret_cast<u64*>(smem);  // W
    u64* exC = exR + W;                       // W
    u64* seg = exC + W;                       // 4 x G x w
    // Edge strips (as energy_frame): exR[wm1 + k] = energy of the first k
    // rows, exR[wm1 - k] of the last k rows; the same for columns. Warps 0-3.
    if (warp < 4) {
        const u64* src = warp < 2 ? rE : cE;
        const int len = warp < 2 ? mc : nc;
        u64* dst = warp < 2 ? exR : exC;
        const bool from_end = warp & 1;
        u64 carry = 0;
        if (lane == 0) dst[wm1] = 0;
        for (int k0 = 0; k0 < wm1; k0 += 32) {
            const int k = k0 + lane;
            u64 v = k < wm1 ? src[from_end ? len - 1 - k : k] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u64 u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            v += carry;
            if (k < wm1) dst[from_end ? wm1 - 1 - k : wm1 + 1 + k] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    const int q = warp / G, g = warp - q * G;
    const bool active = q < 4;
    const bool bottom = q >= 2, right = q & 1;
    const int L = (wm1 + G - 1) / G;
    const int a0 = 1 + g * L, a1 = min(w, 1 + (g + 1) * L);
    const size_t wm1sq = (size_t)wm1 * wm1;
    const uint32_t* blk = corners_f + (size_t)(q & 3) * wm1sq;
    // Corner values of table row a at this lane's columns (0 at b = 0 and
    // b >= w), and their squares.
    auto row_raw = [&](int a, int32_t (&c)[K]) {
        const uint32_t* row = blk + (size_t)(bottom ? wm1 - a : a - 1) * wm1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = K * lane + k;
            c[k] = (b >= 1 && b < w) ? (int32_t)row[right ? wm1 - b : b - 1] : 0;
        }
    };
    auto squares = [&](const int32_t (&c)[K], u64 (&v)[K]) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (u64)((long long)c[k] * c[k]);
    };
    // Inclusive prefix of v along the columns (lane-local, then across lanes).
    auto col_prefix = [&](u64 (&v)[K]) {
#pragma unroll
        for (int k = 1; k < K; ++k) v[k] += v[k - 1];
        const u64 tot = v[K - 1];
        u64 x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const u64 excl = x - tot;
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += excl;
    };
    if (active) {
        u64 cs[K];
#pragma unroll
        for (int k = 0; k < K; ++k) cs[k] = 0ull;
        for (int a = a0; a < a1; ++a) {
            int32_t c[K];
            u64 v[K];
            row_raw(a, c);
            squares(c, v);
#pragma unroll
            for (int k = 0; k < K; ++k) cs[k] += v[k];
        }
        col_prefix(cs);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = K * lane + k;
            if (b < w) seg[((size_t)q * G + g) * w + b] = cs[k];
        }
    }
    __syncthreads();
    if (!active) return;
    u64 carry[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int b = K * lane + k;
        carry[k] = 0ull;
        if (b < w)
            for (int g2 = 0; g2 < g; ++g2) carry[k] += seg[((size_t)q * G + g2) * w + b];
    }
    // The shifts of table row a at this lane's columns: whether each exists.
    auto row_fetch = [&](int a, V (&val)[K]) {
        const int s = bottom ? -a : a;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = K * lane + k;
            if (b < w && !(right && b == 0)) val[k] = fetch(s, right ? -b : b);
        }
    };
    auto emit_row = [&](int a, const V (&val)[K]) {
        const int s = bottom ? -a : a;
        const u64 base = T - exR[s + wm1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = K * lane + k;
            if (b < w && !(right && b == 0)) {
                const int t = right ? -b : b;
                emit(s, t, base - exC[t + wm1] + carry[k], val[k]);
            }
        }
    };
    V vnext[K];  // the next row's fetched values, loaded one row ahead
    if (g == 0 && !bottom) {  // a = 0: no corner rows (s = 0 belongs to the top quadrants)
        V v0[K];
        row_fetch(0, v0);
        emit_row(0, v0);
    }
    int32_t nxt[K];  // the next row's corner values, loaded one row ahead
    if (a0 < a1) {
        row_raw(a0, nxt);
        row_fetch(a0, vnext);
    }
    for (int a = a0; a < a1; ++a) {
        int32_t c[K];
        V vcur[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            c[k] = nxt[k];
            vcur[k] = vnext[k];
        }
        if (a + 1 < a1) {
            row_raw(a + 1, nxt);
            row_fetch(a + 1, vnext);
        }
        u64 v[K];
        squares(c, v);
        col_prefix(v);
#pragma unroll
        for (int k = 0; k < K; ++k) carry[k] += v[k];
        emit_row(a, vcur);
    }
}

template <int K, typename Emit>
__device__ __forceinline__ void energy_sweep(const u64* __restrict__ rE, const u64* __restrict__ cE, u64 T,
                                             const uint32_t* __restrict__ corners_f, int mc, int nc, int wm1,
                                             unsigned char* smem, Emit emit) {
    energy_sweep_f<K>(rE, cE, T, corners_f, mc, nc, wm1, smem, SweepEmit3<Emit>{emit}, SweepNoFetch{});
}

// energy_sweep with K = ceil(w / 32) columns per lane (w <= 128).
template <typename Emit>
__device__ __forceinline__ void energy_sweep_any(const u64* __restrict__ rE, const u64* __restrict__ cE, u64 T,
                                                 const uint32_t* __restrict__ corners_f, int mc, int nc, int wm1,
                                                 unsigned char* smem, Emit emit) {
    if (wm1 < 32) energy_sweep<1>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit);
    else if (wm1 < 64) energy_sweep<2>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit);
    else if (wm1 < 96) energy_sweep<3>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit);
    else energy_sweep<4>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit);
}
template <typename Emit, typename Fetch>
__device__ __forceinline__ void energy_sweep_any_f(const u64* __restrict__ rE, const u64* __restrict__ cE, u64 T,
                                                   const uint32_t* __restrict__ corners_f, int mc, int nc, int wm1,
                                                   unsigned char* smem, Emit emit, Fetch fetch) {
    if (wm1 < 32) energy_sweep_f<1>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit, fetch);
    else if (wm1 < 64) energy_sweep_f<2>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit, fetch);
    else if (wm1 < 96) energy_sweep_f<3>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit, fetch);
    else energy_sweep_f<4>(rE, cE, T, corners_f, mc, nc, wm1, smem, emit, fetch);
}

// The template-side operands of one shift's combine.
struct CombineOps {
    float2 sb;  // Sb as an FP32 pair
    float ia;   // 1 / Area (times the unit)
};

template <bool F32, bool OUT_DOUBLE>
__global__ void __launch_bounds__(kEnergyThreads)
k_energy(const u64* __restrict__ rowE, const u64* __restrict__ colE, const u64* __restrict__ tot,
         const uint32_t* __restrict__ corners, int mc, int nc, int wm1, void* __restrict__ out,
         int flip) {
    typedef typename AccT<F32>::type Acc;
    extern __shared__ __align__(16) unsigned char esm_raw[];
    const int W = 2 * wm1 + 1;
    const int64_t f = blockIdx.x;
    if constexpr (!F32 && !OUT_DOUBLE) {
        // integer frames' energies as FP32 pairs (the direct form's combine): the warp sweep
        auto emit = [&](int s, int t, u64 val) {
            const int so = flip ? -s : s, to = flip ? -t : t;
            static_cast<float2*>(out)[f * (int64_t)W * W + (int64_t)(so + wm1) * W + (to + wm1)] = energy_pair(val);
        };
        energy_sweep_any(rowE + f * mc, colE + f * nc, tot[f], corners + f * 4 * (size_t)wm1 * wm1, mc, nc, wm1,
                         esm_raw, emit);
        return;
    }
    energy_frame<F32>(rowE + f * mc, colE + f * nc, tot[f], corners + f * 4 * (size_t)wm1 * wm1, mc, nc, wm1,
                      esm_raw, [&](int s, int t, Acc val) {
                          const int so = flip ? -s : s, to = flip ? -t : t;
                          const int64_t k = f * (int64_t)W * W + (int64_t)(so + wm1) * W + (to + wm1);
                          if (OUT_DOUBLE) {
                              static_cast<double*>(out)[k] = (double)val;
                          } else {
                              static_cast<float2*>(out)[k] = energy_pair(*reinterpret_cast<const u64*>(&val));
                          }
                      });
}

// ---------------------------------------------------------------------------
// k_cols: one CTA per (frame = blockIdx.x, kColsVC spectral columns v = blockIdx.y).
// Forward DFT along the image rows (length Nr) of X[:, v], multiplied by the
// plan's conj(template spectrum) / (Nr Nc) (stored in the forward output
// layout), inverse DFT, and only the 2w-1 rows s in [-(w-1), w-1] kept:
// Y[f*y_fstride + (s+w-1)*ncv + v]. With SPECTRUM set, the forward transform
// is written out conjugated and scaled instead (template preparation).
// Threads of a k_cols CTA: one per task of the wider four-step stage.
template <int N>
__host__ __device__ constexpr int cols_threads() {
    return (kColsVC * (Four<N>::N1 > Four<N>::N2 ? Four<N>::N1 : Four<N>::N2) + 31) / 32 * 32;
}

template <int N>
__host__ __device__ constexpr int cols_min_blocks() {
    return cols_threads<N>() <= 256 ? 4 : (cols_threads<N>() <= 320 ? 3 : 1);
}

template <int N, bool SPECTRUM>
__global__ void __launch_bounds__(cols_threads<N>(), cols_min_blocks<N>())
k_cols(const float2* __restrict__ X, int64_t x_fstride, int ldx, int mc, int ncv,
       const float2* __restrict__ tw_g, const float2* __restrict__ bspec, float2* __restrict__ Y,
       int64_t y_fstride, int wm1, float scale) {
    extern __shared__ __align__(16) unsigned char csm_raw[];
    constexpr int LD = fft_ld<N>();                      // skewed, padded row
    float2* buf = reinterpret_cast<float2*>(csm_raw);  // kColsVC x LD
    float2* tw = buf + kColsVC * LD;                     // 2N: forward, then inverse table
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int v0 = blockIdx.y * kColsVC, nv = min(kColsVC, ncv - v0);
    const int64_t f = blockIdx.x;
    for (int i = tid; i < 2 * N; i += nthr) tw[i] = tw_g[i];
    // A thread owns positions i (one slot sk(i)) of all the CTA's columns;
    // each column's loads are issued before any is stored.
    const float2* xs = X + f * x_fstride + (int64_t)v0 * ldx;
    for (int i = tid; i < N; i += nthr) {
        const int ski = sk<N>(i);
#pragma unroll
        for (int v8 = 0; v8 < kColsVC; v8 += 8) {
            float2 t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                t[u] = (v8 + u < nv && i < mc) ? xs[(int64_t)(v8 + u) * ldx + i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (v8 + u < nv) buf[(v8 + u) * LD + ski] = t[u];
        }
    }
    __syncthreads();
    if (SPECTRUM) {
        fft4_fwd<N>(buf, LD, nv, tw, tid, nthr);
        for (int p = tid; p < N; p += nthr) {
            const int skp = sk<N>(p);
#pragma unroll
            for (int vi = 0; vi < kColsVC; ++vi)
                if (vi < nv) Y[(int64_t)(v0 + vi) * N + p] = cscale(cconj(buf[vi * LD + skp]), scale);
        }
        return;
    }
    // forward first stage in place (each task reads its comb before writing it)
    fft4_fwd_stage1_gen<N>([&](int r, int n) { return buf[r * LD + sk<N>(n)]; }, buf, LD, nv, tw, tid, nthr);
    __syncthreads();
    // forward second stage, template product and inverse first stage in one pass
    fft4_fwd2_mul_inv1<N>(buf, LD, nv, bspec + (int64_t)v0 * N, N, tw + N, tid, nthr);
    fft4_inv_stage2<N>(buf, LD, nv, tid, nthr);
    const int W = 2 * wm1 + 1;
    float2* ys = Y + f * y_fstride + v0;
    for (int task = tid; task < W * kColsVC; task += nthr) {
        const int si = task / kColsVC, vi = task % kColsVC;
        if (vi >= nv) continue;
        const int pos = si - wm1 < 0 ? si - wm1 + N : si - wm1;
        ys[(int64_t)si * ncv + vi] = buf[vi * LD + sk<N>(pos)];
    }
}

// k_cols_stream: the k_cols product for many frames per CTA. Grid (column
// blocks, frame slices): CTA (x, y) owns spectral columns [v0, v1) (the ncv
// columns split evenly over gridDim.x blocks of at most kColsVC) and walks
// frames f = y, y + gridDim.y, ... Its columns' template spectrum stays in
// shared memory; each frame's block of row spectra X[f][v0 .. v1) (contiguous,
// v1 - v0 rows of ldx) arrives by one bulk copy into a staging buffer, issued
// as soon as the previous frame's first transform stage has read the buffer,
// so the copy runs under the rest of that frame's transforms. The bounded
// wait on the copy sets *err and ends the CTA (after the copy in flight).
// Row stride of the staging buffer (complex values): ldx, padded so that it
// is congruent to N2 modulo 16 (the first stage reads N2 tasks per row along
// the row, see Skew) when the padding keeps every row 16-byte aligned.
template <int N>
__host__ __device__ constexpr int cols_stage_ld(int ldx) {
    const int pad = ((Four<N>::N2 - ldx) % 16 + 16) % 16;
    return ldx + (pad % 2 == 0 ? pad : 0);
}
template <int N>
__host__ __device__ constexpr size_t cols_stream_smem(int ldx) {
    return sizeof(float2) *
           ((size_t)kColsVC * cols_stage_ld<N>(ldx) + (size_t)kColsVC * fft_ld<N>() + (size_t)kColsVC * N + 2 * N);
}

// (two CTAs per SM for the transforms of up to 320 points; one beyond, where
// shared memory holds one anyway, so the codelets keep their registers)
template <int N>
__global__ void __launch_bounds__(cols_threads<N>(), cols_threads<N>() <= 320 ? 2 : 1)
k_cols_stream(const float2* __restrict__ X, int64_t x_fstride, int ldx, int mc, int ncv, int64_t T,
              const float2* __restrict__ tw_g, const float2* __restrict__ bspec, float2* __restrict__ Y,
              int64_t y_fstride, int wm1, unsigned int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LD = fft_ld<N>();
    const int SL = cols_stage_ld<N>(ldx);              // staging row stride (even: rows 16-byte aligned)
    float2* stg = reinterpret_cast<float2*>(smem_raw);  // kColsVC x SL: the frame's block, one row per column
    float2* buf = stg + kColsVC * SL;                    // kColsVC x LD
    float2* bs = buf + kColsVC * LD;                     // kColsVC x N: template spectrum, forward output layout
    float2* tw = bs + kColsVC * N;                       // 2N: forward, then inverse table
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int v0 = (int)((int64_t)blockIdx.x * ncv / gridDim.x);
    const int nv = (int)((int64_t)(blockIdx.x + 1) * ncv / gridDim.x) - v0;  // <= kColsVC (host)
    const uint32_t row_bytes = (uint32_t)(sizeof(float2) * ldx);
    const int W = 2 * wm1 + 1;
    // The frame's rows v0 .. v0 + nv - 1 of X (contiguous in global memory)
    // into the staging rows, one bulk copy per row (one thread).
    auto issue = [&](int64_t fr) {
        mbar_expect_tx(&bar, row_bytes * (uint32_t)nv);
        const float2* g = X + fr * x_fstride + (int64_t)v0 * ldx;
        for (int vi = 0; vi < nv; ++vi) bulk_g2s(stg + vi * SL, g + (int64_t)vi * ldx, row_bytes, &bar);
    };
    int64_t f = blockIdx.y;
    if (f >= T) return;  // the same for the whole CTA
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        fence_async_smem();
        issue(f);
    }
    for (int i = tid; i < 2 * N; i += nthr) tw[i] = tw_g[i];
    for (int i = tid; i < nv * N; i += nthr) bs[i] = bspec[(int64_t)v0 * N + i];
    uint32_t phase = 0;
    for (; f < T; f += gridDim.y) {
        __syncthreads();  // set-up / the previous frame's outputs are read from buf
        if (!mbar_wait(&bar, phase, err)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (tid == 0) mbar_wait(&bar, phase, err);  // the copy in flight lands before the CTA ends
            return;
        }
        phase ^= 1u;
        fft4_fwd_stage1_from<N>(stg, SL, mc, buf, LD, nv, tw, tid, nthr);
        __syncthreads();
        if (tid == 0 && f + gridDim.y < T) {
            fence_async_smem();  // this frame's reads of the staging buffer come before the next copy
            issue(f + gridDim.y);
        }
        // forward second stage, template product and inverse first stage in one pass
        fft4_fwd2_mul_inv1<N>(buf, LD, nv, bs, N, tw + N, tid, nthr);
        fft4_inv_stage2<N>(buf, LD, nv, tid, nthr);
        float2* ys = Y + f * y_fstride + v0;
        for (int task = tid; task < W * kColsVC; task += nthr) {
            const int si = task / kColsVC, vi = task % kColsVC;
            if (vi >= nv) continue;
            const int pos = si - wm1 < 0 ? si - wm1 + N : si - wm1;
            ys[(int64_t)si * ncv + vi] = buf[vi * LD + sk<N>(pos)];
        }
    }
}

// ---------------------------------------------------------------------------
// The combine f = (Sa + Sb - 2h) / Area * unit in FP32 from the exact
// energies as FP32 pairs: Sa_hi + Sb_hi by an error-free sum (TwoSum), so
// the only roundings are h's own (the FP32 cross term), one in the
// difference and one in the final product (~1e-7 relative each).
__device__ __forceinline__ float combine_f32(float2 sa, float2 sb, float h, float ia) {
    const float s = sa.x + sb.x;
    const float bb = s - sa.x;
    const float err = (sa.x - (s - bb)) + (sb.x - bb);
    const float num = (s - 2.0f * h) + (err + (sa.y + sb.y));
    return num * ia;
}

// k_rows_inv: one CTA per frame. Inverse real DFTs along the image columns
// (length Nc) of Y's 2w-1 rows, two rows per complex transform, keeping the
// 2w-1 columns t in [-(w-1), w-1] -> h[s][t]. Then the frame's exact
// energies Sa_st (energy_frame, from the frame pass's edge sums and corner
// blocks, in the shared memory the transforms no longer need) and
//     f_st = (Sa_st + Sb_st - 2 h_st) / Area_st * unit   (combine_f32)
// and the argmin over the window with the tie-break: smallest f, then
// smallest |s|+|t|, then smallest s, then smallest t. Also the second-best
// value for the margin (f2 - f1) / f1.
struct Best {
    float f1;
    int r1;
    float f2;
};
__device__ __forceinline__ void best_push(Best& b, float f, int r) {
    if (f < b.f1 || (f == b.f1 && r < b.r1)) {
        b.f2 = fminf(b.f2, b.f1);
        b.f1 = f;
        b.r1 = r;
    } else {
        b.f2 = fminf(b.f2, f);
    }
}
__device__ __forceinline__ void best_merge(Best& a, const Best& o) {
    if (o.f1 < a.f1 || (o.f1 == a.f1 && o.r1 < a.r1)) {
        a.f2 = fminf(o.f2, a.f1);
        a.f1 = o.f1;
        a.r1 = o.r1;
    } else {
        a.f2 = fminf(a.f2, o.f1);
    }
}

// Shared memory of k_rows_inv: the transform buffer (later the energies'
// tables), the inverse roots, h.
template <int N>
__host__ __device__ constexpr int rows_inv_threads() {
    return (kInvPC * (Four<N>::N1 > Four<N>::N2 ? Four<N>::N1 : Four<N>::N2) + 31) / 32 * 32;
}
template <int N>
__host__ __device__ constexpr size_t rows_inv_region(int wm1) {
    return (sizeof(float2) * kInvPC * fft_ld<N>() > energy_sweep_smem(wm1, rows_inv_threads<N>() / 32)
                ? sizeof(float2) * kInvPC * fft_ld<N>()
                : (energy_sweep_smem(wm1, rows_inv_threads<N>() / 32) + 15) / 16 * 16);
}
template <int N>
__host__ __device__ constexpr size_t rows_inv_smem(int wm1) {
    return rows_inv_region<N>(wm1) + sizeof(float2) * N + sizeof(float) * (2 * wm1 + 1) * (2 * wm1 + 1);
}

template <int N>
__global__ void __launch_bounds__(rows_inv_threads<N>() <= 288 ? 288 : 576, rows_inv_threads<N>() <= 288 ? 3 : 1)
k_rows_inv(const float2* __restrict__ Y, int64_t y_fstride, int ncv, int wm1,
           const float2* __restrict__ tw_g, const u64* __restrict__ rowE, const u64* __restrict__ colE,
           const u64* __restrict__ tot, const uint32_t* __restrict__ corners, int mc, int nc,
           const float2* __restrict__ Sb2, const float* __restrict__ ia32, double* __restrict__ cost,
           int32_t* __restrict__ coarse, double* __restrict__ fbest, float* __restrict__ margin) {
    extern __shared__ __align__(16) unsigned char ism_raw[];
    constexpr int LD = fft_ld<N>();                      // skewed, padded row
    float2* buf = reinterpret_cast<float2*>(ism_raw);  // kInvPC x LD
    float2* tw = reinterpret_cast<float2*>(ism_raw + rows_inv_region<N>(wm1));  // N: inverse table
    const int W = 2 * wm1 + 1, WW = W * W;
    float* hbuf = reinterpret_cast<float*>(tw + N);     // W x W
    __shared__ Best red[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t f = blockIdx.x;
    for (int i = tid; i < N; i += nthr) tw[i] = tw_g[N + i];
    const float2* ys = Y + f * y_fstride;
    const int npairs = (W + 1) / 2;
    constexpr int NH = N / 2;
    for (int p0 = 0; p0 < npairs; p0 += kInvPC) {
        const int np = min(kInvPC, npairs - p0);
        __syncthreads();
        // Two real rows ra, rb = ra + 1 as one complex row: Z[k] = A[k] + i B[k]
        // from the half spectra (k <= N/2; A[N-k] = conj A[k]). Each stored
        // value is read once; four tasks' loads are issued before any store.
        constexpr int NK = NH + 1;
        const int ntask = np * NK;
        for (int t0 = tid; t0 < ntask; t0 += 4 * nthr) {
            float2 A[4], B[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int task = t0 + q * nthr;
                A[q] = make_float2(0.f, 0.f);
                B[q] = make_float2(0.f, 0.f);
                if (task < ntask) {
                    const int pi = task / NK, kk = task - pi * NK;
                    const int ra = 2 * (p0 + pi), rb = ra + 1;
                    A[q] = ys[(int64_t)ra * ncv + kk];
                    if (rb < W) B[q] = ys[(int64_t)rb * ncv + kk];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int task = t0 + q * nthr;
                if (task < ntask) {
                    const int pi = task / NK, kk = task - pi * NK;
                    float2 a = A[q], b = B[q];
                    if (kk == 0 || kk == NH) { a.y = 0.f; b.y = 0.f; }
                    buf[pi * LD + sk<N>(spec_pos<N>(kk))] = make_float2(a.x - b.y, a.y + b.x);
                    if (kk != 0 && kk != NH)  // k = N - kk: conj A + i conj B
                        buf[pi * LD + sk<N>(spec_pos<N>(N - kk))] = make_float2(a.x + b.y, b.x - a.y);
                }
            }
        }
        __syncthreads();
        fft4_inv<N>(buf, LD, np, tw, tid, nthr);
        for (int task = tid; task < np * W; task += nthr) {
            const int pi = task / W, ti = task - pi * W;
            const int pos = (ti - wm1 + N) % N;
            const float2 z = buf[pi * LD + sk<N>(pos)];
            const int ra = 2 * (p0 + pi);
            hbuf[ra * W + ti] = z.x;
            if (ra + 1 < W) hbuf[(ra + 1) * W + ti] = z.y;
        }
    }
    __syncthreads();  // the transform buffer is read for the last time above
    Best b;
    b.f1 = INFINITY;
    b.r1 = 0x7fffffff;
    b.f2 = INFINITY;
    // The frame's energies Sa (exact) straight into the combine; the sweep's
    // scratch takes the transform buffer's place. The template's Sb and
    // 1/Area of a row's shifts are loaded a row ahead.
    auto fetch = [&](int s, int t) {
        const int k = (s + wm1) * W + (t + wm1);
        return CombineOps{__ldg(Sb2 + k), __ldg(ia32 + k)};
    };
    auto emit = [&](int s, int t, u64 sa, const CombineOps& o) {
        const int k = (s + wm1) * W + (t + wm1);
        const float fv = combine_f32(energy_pair(sa), o.sb, hbuf[k], o.ia);
        if (cost) cost[f * WW + k] = f32_to_f64(fv);
        best_push(b, fv, (abs(s) + abs(t)) * WW + k);
    };
    energy_sweep_any_f(rowE + f * mc, colE + f * nc, tot[f], corners + f * 4 * (size_t)wm1 * wm1, mc, nc, wm1,
                       ism_raw, emit, fetch);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best o2;
        o2.f1 = __shfl_xor_sync(0xffffffffu, b.f1, o);
        o2.r1 = __shfl_xor_sync(0xffffffffu, b.r1, o);
        o2.f2 = __shfl_xor_sync(0xffffffffu, b.f2, o);
        best_merge(b, o2);
    }
    if ((tid & 31) == 0) red[tid >> 5] = b;
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < (nthr + 31) / 32; ++i) best_merge(b, red[i]);
        const int k = b.r1 % WW;
        const int s = k / W - wm1, t = k % W - wm1;
        coarse[2 * f] = s;
        coarse[2 * f + 1] = t;
        if (fbest) fbest[f] = (double)b.f1;
        if (margin) {
            float mg;
            if (b.f1 > 0) mg = (b.f2 - b.f1) / b.f1;
            else mg = (b.f2 > 0) ? INFINITY : 0.f;
            margin[f] = mg;
        }
    }
}

// ---------------------------------------------------------------------------
// k_jitter: the upsampling step of Section 2. For the nine candidates
// (s, t) = (2 sc + u - 1, 2 tc + v - 1), u, v in {0, 1, 2}, the exact
//     S = sum over D of (a[i+s][j+t] - b[i][j])^2
//       = sum_D a^2 + sum_D b^2 - 2 sum_D a b
// at full resolution, all nine accumulated in one pass over the frame.
//
// Products are exact 32-bit integer dot products (dp2a: two 16-bit values
// times two bytes, plus a 32-bit sum). With y = 256 y_hi + y_lo split into
// bytes, x y = 256 x y_hi + x y_lo and the two halves are summed apart. Each
// 16 x 8-bit product is below 2^24, so a band of at most 32 rows of 8
// columns sums below 2^32 exactly; the halves meet in 64 bits once per band.
//
// Frame values outside the frame are read as zero, so sum a b and sum a^2
// need no mask. sum_D b^2 depends on the template and (s, t) only: with a
// 2-D prefix table of b^2 (TABLE) the frame's last warp item reads it at four
// corners per shift; without one it is summed in the loop, a template
// position counting only when its partner lies inside the frame.
//
// Work comes in warp items (below). Each thread owns the template columns
// j0 .. j0+7 of a band of band_rows (<= kJitRows) rows and walks down it keeping the three
// frame rows r = i + 2 sc - 1 + u (u = 0, 1, 2) as 16-bit pairs, columns
// counted from lead = j0 + 2 tc - 1 (odd):
//   pw[p] = columns (lead + 2p, lead + 2p + 1), p < 5   (v = 0: pw[0..3],
//                                                        v = 2: pw[1..4])
//   rw[p] = columns (lead + 2p + 1, lead + 2p + 2), p < 4 (v = 1)
// rw are the aligned 32-bit words themselves; pw take one byte permute each.
// An aligned word (even column c, c + 1; n even) lies wholly inside or
// wholly outside the frame, so every thread runs the same code: a word
// outside is a predicated-off load that leaves zero; so is a row outside the
// frame.
// Frame and template rows arrive through a ring of asynchronous copies
// kJitRing rows ahead (below), and the loop is unrolled three times so that
// the window rotates without copies.
//
// sum a^2: each window row is summed over its v = 0 columns only; the
// frame rows that all three u share accumulate once per row, the two rows at
// each end of the band's frame range are added at the end. The groups tile
// the template row, so across a row the v = 1 and v = 2 windows differ from
// v = 0 by one or two frame columns at the two ends of the row only: the
// threads of the first and last groups subtract and add those columns'
// squares (jit_edge_columns, a warp at a time).
// In-loop sum b^2: template rows whose partner rows are valid for all three
// u accumulate once; the at most four rows valid for only some u are added
// at the end.
// Per-warp partial sums go to acc[f][9] by 64-bit atomics (two's complement
// wrap-around: the total is exact); the last warp item of a frame (ticket
// counter) adds sum_D b^2 (TABLE) and takes the minimum of S / Area with the
// tie-break, compared as exact rationals. acc and ticket are zero on entry.
constexpr int kJitRows = 32;  // band height (at most: the launcher may pick shorter bands)
static_assert(kJitRows <= 32, "32-bit dot-product sums are exact for at most 32 rows of 8 columns");

// One frame row of a thread's window. raw: the 16-byte chunks that hold
// half-words lead-1 .. lead+10, i.e. 32-bit words O .. O+5 of raw, where
// O = ((lead - 1) / 2) mod 4 is the same for every thread of a frame (lead =
// 8 j + 2 tc - 1); a ninth word when O = 3. pw as described above; rw[p] is
// raw[O + 1 + p] itself. Chunks (8 half-words from a multiple of 8; n % 8 ==
// 0) lie wholly inside or outside the frame: outside ones stay zero.
template <int O>
struct JitSlot {
    uint32_t raw[O == 3 ? 9 : 8];
    uint32_t pw[5];
};

// 2 x 32-bit partial sums (low and high byte half) of one quantity.
struct Acc2 {
    uint32_t lo, hi;
};

struct JitBand {
    const uint16_t* a;     // frame
    const uint16_t* tmpl;  // template
    int m, n, s0, j0, i_b, i_e;
    int first;             // frame row of window row 0 at the band's first template row
    int c0;                // first column of raw chunk 0 (multiple of 8, may be negative)
    uint32_t cvalid;       // bit c: raw chunk c (columns c0 + 8c .. + 7) inside the frame
};

template <int O>
__device__ __forceinline__ void jit_unpack(JitSlot<O>& x) {
#pragma unroll
    for (int p = 0; p < 5; ++p) x.pw[p] = __byte_perm(x.raw[O + p], x.raw[O + p + 1], 0x5432);
}

// Byte planes of a 16-bit pair (y0, y1): bytes (y0_lo, y1_lo, y0_hi, y1_hi).
__device__ __forceinline__ uint32_t byte_planes(uint32_t y) { return __byte_perm(y, 0u, 0x3120); }

// acc += x . y for a 16-bit pair x and the byte planes yp of a pair y
// (dp2a: the two 16-bit halves of x times bytes 0, 1 (lo) or 2, 3 (hi) of
// yp, added to the 32-bit accumulator in place).
__device__ __forceinline__ void dot_acc(uint32_t x, uint32_t yp, Acc2& acc) {
    asm("dp2a.lo.u32.u32 %0, %1, %2, %0;" : "+r"(acc.lo) : "r"(x), "r"(yp));
    asm("dp2a.hi.u32.u32 %0, %1, %2, %0;" : "+r"(acc.hi) : "r"(x), "r"(yp));
}

__device__ __forceinline__ u64 acc_value(const Acc2& a) { return (u64)a.lo + ((u64)a.hi << 8); }

// Sum of squares of one window row over its v = 0 columns 0..7 (of lead ..).
template <int O>
__device__ __forceinline__ void row_energy(const JitSlot<O>& x, Acc2& e) {
#pragma unroll
    for (int p = 0; p < 4; ++p) dot_acc(x.pw[p], byte_planes(x.pw[p]), e);
}

// Byte masks of template pair p for shift v: the template columns whose
// frame partner (column lead + 2p + v, + 1) lies inside the frame.
__device__ __forceinline__ uint32_t col_mask(uint32_t mask, int v, int p) {
    return (((mask >> (v * 8 + 2 * p)) & 1u) ? 0x00ff00ffu : 0u) |
           (((mask >> (v * 8 + 2 * p + 1)) & 1u) ? 0xff00ff00u : 0u);
}

// In-loop template energy of one row (pairs bw, planes bp) for each v.
__device__ __forceinline__ void tmpl_energy(const uint32_t (&bw)[4], const uint32_t (&bp)[4],
                                            const uint32_t (&cm)[12], Acc2 (&e)[3]) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < 4; ++p) dot_acc(bw[p], bp[p] & cm[v * 4 + p], e[v]);
}

__device__ __forceinline__ uint4 jit_tmpl_row(const JitBand& B, int i) {
    return __ldg(reinterpret_cast<const uint4*>(B.tmpl + (int64_t)i * B.n + B.j0));
}

// Shared-memory ring of rows in flight: stage q % 3 holds, per thread, the
// raw chunks of frame row first + q and (q >= 2) template row i_b + q - 2, as
// ring[((stage * 4) + c) * kJitterThreads + tid], c = 0, 1, 2 frame chunks,
// 3 template; each thread copies and reads only its own column (cp.async,
// one commit group per row), so no barrier is needed. Three stages, as many
// as the window's slots, so that the loop unrolled three times names every
// stage at compile time. Only chunks inside the frame are copied: a chunk
// outside it (the same columns for every row of a band) is zeroed in every
// stage once, when the band starts, and a row outside the frame is zeroed
// when it is taken.
constexpr int kJitRing = 3;
constexpr size_t kJitRingBytes = (size_t)kJitRing * 4 * kJitterThreads * 16;
// After the ring, one 16-byte cell per thread: the energies of its band's
// first two frame rows (taken when they arrive, added at the band's end).
constexpr size_t kJitSmemBytes = kJitRingBytes + (size_t)kJitterThreads * 16;

// The next row to copy: its frame row ar, the addresses of its first raw
// chunk (columns c0 .. c0 + 7 of row ar; read only where inside the frame)
// and of its template row's chunk, rows left to issue.
struct JitCursor {
    const uint16_t* fp;
    const uint16_t* tp;
    int ar, left;
};

template <int O, int STAGE>
__device__ __forceinline__ void jit_issue(const JitBand& B, uint4* ring, bool with_tmpl, JitCursor& cur) {
    uint4* st = ring + STAGE * 4 * kJitterThreads;
    if (cur.left > 0) {
        const bool rok = (unsigned)cur.ar < (unsigned)B.m;
#pragma unroll
        for (int c = 0; c < (O == 3 ? 3 : 2); ++c)
            cp16_if(rok && ((B.cvalid >> c) & 1u), st + c * kJitterThreads, cur.fp + 8 * c);
        if (with_tmpl) {
            cp16(st + 3 * kJitterThreads, cur.tp);
            cur.tp += B.n;
        }
        cur.fp += B.n;
        ++cur.ar;
        --cur.left;
    }
    cp_commit();
}

// The row in ring stage STAGE (its copy group complete) into slot x, zeros
// when the row lies outside the frame (rok false); its template row into *tr
// when asked.
template <int O, int STAGE>
__device__ __forceinline__ void jit_take(const uint4* ring, bool rok, JitSlot<O>& x, uint4* tr) {
    const uint4* st = ring + STAGE * 4 * kJitterThreads;
    const uint4 c0 = st[0], c1 = st[kJitterThreads];
    x.raw[0] = c0.x;
    x.raw[1] = c0.y;
    x.raw[2] = c0.z;
    x.raw[3] = c0.w;
    x.raw[4] = c1.x;
    x.raw[5] = c1.y;
    x.raw[6] = c1.z;
    x.raw[7] = c1.w;
    if (O == 3) x.raw[(O == 3) ? 8 : 0] = st[2 * kJitterThreads].x;
    if (!rok)
#pragma unroll
        for (int k = 0; k < (O == 3 ? 9 : 8); ++k) x.raw[k] = 0u;
    if (tr) *tr = st[3 * kJitterThreads];
    jit_unpack(x);
}

// Step j of a band (K = j mod 3), template row i = i_b + j: slots K, K+1
// hold frame rows i+s0-1, i+s0; slot K+2 receives row i+s0+1 (ring row j+2,
// stage (K + 2) mod 3) with template row i, and ring row j+5 is issued into
// the same stage.
template <bool TABLE, int O, int K>
__device__ __forceinline__ void jit_step(const JitBand& B, int i, uint4* ring, JitCursor& cur, JitSlot<O> (&S)[3],
                                         Acc2 (&C)[9],
                                         Acc2& M, Acc2 (&QB)[3], const uint32_t (&cm)[12]) {
    JitSlot<O>& w0 = S[K];
    JitSlot<O>& w1 = S[(K + 1) % 3];
    JitSlot<O>& w2 = S[(K + 2) % 3];
    uint4 tr;
    cp_wait<kJitRing - 1>();
    jit_take<O, (K + 2) % 3>(ring, (unsigned)(i + B.s0 + 1) < (unsigned)B.m, w2, &tr);
    const uint32_t bw[4] = {tr.x, tr.y, tr.z, tr.w};
    uint32_t bp[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) bp[p] = byte_planes(bw[p]);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        dot_acc(w0.pw[p], bp[p], C[0]);
        dot_acc(w0.raw[O + 1 + p], bp[p], C[1]);
        dot_acc(w0.pw[p + 1], bp[p], C[2]);
        dot_acc(w1.pw[p], bp[p], C[3]);
        dot_acc(w1.raw[O + 1 + p], bp[p], C[4]);
        dot_acc(w1.pw[p + 1], bp[p], C[5]);
        dot_acc(w2.pw[p], bp[p], C[6]);
        dot_acc(w2.raw[O + 1 + p], bp[p], C[7]);
        dot_acc(w2.pw[p + 1], bp[p], C[8]);
    }
    if (i <= B.i_e - 3) row_energy(w2, M);  // frame row shared by all three u
    if (!TABLE)
        if (i + B.s0 - 1 >= 0 && i + B.s0 + 1 <= B.m - 1) tmpl_energy(bw, bp, cm, QB);
    jit_issue<O, (K + 2) % 3>(B, ring, true, cur);  // the stage just read (its data is consumed)
}

// X[u*3+v] += energy e of frame row r (its v = 0 window, every v) for each
// u whose range first + u .. first + u + L - 1 holds r.
__device__ __forceinline__ void jit_add_row(int r, int first, int L, const Acc2& e, u64 (&X)[9]) {
    const u64 ev = acc_value(e);
#pragma unroll
    for (int u = 0; u < 3; ++u)
        if (r >= first + u && r <= first + u + L - 1)
#pragma unroll
            for (int v = 0; v < 3; ++v) X[u * 3 + v] += ev;
}

// The v = 1, 2 windows of a band's frame rows against v = 0: at the left end
// of the template row (group 0, bit 0 of need) they lack frame columns
// c = t0 - 1 (v = 1, 2) and c + 1 (v = 2), at the right end (group G - 1,
// bit 1) they add columns c + n and c + n + 1; each row counts for every u
// whose range first + u .. first + u + L - 1 holds it. The whole warp takes
// the bands of its lanes that hold an end group one at a time, a frame row
// per lane, so the loads of a band are in flight together. Sums mod 2^64
// (the totals are exact); values outside the frame are zero.
__device__ __forceinline__ void jit_edge_columns(const uint16_t* __restrict__ a, int m, int n, int t0, int first,
                                                 int L, uint32_t need, u64 (&X)[9]) {
    const int lane = threadIdx.x & 31;
    uint32_t todo = __ballot_sync(0xffffffffu, need != 0u);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int bf = __shfl_sync(0xffffffffu, first, src);
        const int bL = __shfl_sync(0xffffffffu, L, src);
        const uint32_t bn = __shfl_sync(0xffffffffu, need, src);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (!((bn >> side) & 1u)) continue;
            const int c = t0 - 1 + (side ? n : 0);
            for (int r = bf + lane; r <= bf + bL + 1; r += 32) {
                if (r < 0 || r >= m) continue;
                const uint16_t* row = a + (int64_t)r * n;
                const u64 a0 = (c >= 0 && c < n) ? (u64)__ldg(row + c) : 0ull;
                const u64 a1 = (c + 1 >= 0 && c + 1 < n) ? (u64)__ldg(row + c + 1) : 0ull;
                const u64 q1 = a0 * a0, q2 = q1 + a1 * a1;
                const u64 d1 = side ? q1 : 0ull - q1, d2 = side ? q2 : 0ull - q2;
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    if (r >= bf + u && r <= bf + u + bL - 1) {
                        X[u * 3 + 1] += d1;
                        X[u * 3 + 2] += d2;
                    }
            }
        }
    }
}

template <int O, int A, int B2>
__device__ __forceinline__ void jit_last_rows(const JitSlot<O> (&S)[3], int first, int L, u64 (&X)[9]) {
    Acc2 e = {0u, 0u};
    row_energy(S[A], e);
    jit_add_row(first + L, first, L, e, X);
    Acc2 f = {0u, 0u};
    row_energy(S[B2], f);
    jit_add_row(first + L + 1, first, L, f, X);
}

// The nine partial sums of one thread's band, X[u*3+v] (mod 2^64).
template <bool TABLE, int O>
__device__ __forceinline__ void jit_band(const JitBand& B, uint4* ring, uint32_t mask, u64 (&X)[9]) {
    Acc2 C[9], M = {0u, 0u}, QB[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) C[k] = Acc2{0u, 0u};
#pragma unroll
    for (int v = 0; v < 3; ++v) QB[v] = Acc2{0u, 0u};
    uint32_t cm[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) cm[k] = TABLE ? 0u : col_mask(mask, k / 4, k % 4);
    const int first = B.first, L = B.i_e - B.i_b;
    JitSlot<O> S[3];
    JitCursor cur;
    cur.ar = B.first;
    cur.fp = B.a + ((int64_t)B.first * B.n + B.c0);
    cur.tp = B.tmpl + ((int64_t)B.i_b * B.n + B.j0);
    cur.left = B.i_e - B.i_b + 2;  // rows first .. first + L + 1
#pragma unroll
    for (int c = 0; c < (O == 3 ? 3 : 2); ++c)
        if (!((B.cvalid >> c) & 1u))
#pragma unroll
            for (int q = 0; q < kJitRing; ++q) ring[(q * 4 + c) * kJitterThreads] = make_uint4(0u, 0u, 0u, 0u);
    jit_issue<O, 0>(B, ring, false, cur);
    jit_issue<O, 1>(B, ring, false, cur);
    jit_issue<O, 2>(B, ring, true, cur);
    cp_wait<kJitRing - 1>();
    jit_take<O, 0>(ring, (unsigned)first < (unsigned)B.m, S[0], nullptr);
    jit_issue<O, 0>(B, ring, true, cur);
    cp_wait<kJitRing - 1>();
    jit_take<O, 1>(ring, (unsigned)(first + 1) < (unsigned)B.m, S[1], nullptr);
    jit_issue<O, 1>(B, ring, true, cur);
    {
        // Frame rows first and first + 1 are not shared by all three u: their
        // energies wait in the thread's cell until the band's end.
        Acc2 e0 = {0u, 0u}, e1 = {0u, 0u};
        row_energy(S[0], e0);
        row_energy(S[1], e1);
        ring[kJitRing * 4 * kJitterThreads] = make_uint4(e0.lo, e0.hi, e1.lo, e1.hi);
    }
    for (int i = B.i_b;;) {
        jit_step<TABLE, O, 0>(B, i, ring, cur, S, C, M, QB, cm);
        if (++i >= B.i_e) break;
        jit_step<TABLE, O, 1>(B, i, ring, cur, S, C, M, QB, cm);
        if (++i >= B.i_e) break;
        jit_step<TABLE, O, 2>(B, i, ring, cur, S, C, M, QB, cm);
        if (++i >= B.i_e) break;
    }
    cp_wait<0>();  // the groups still open hold no copies; none stays in flight
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v)
            X[u * 3 + v] = acc_value(M) + acc_value(QB[v]) - 2ull * acc_value(C[u * 3 + v]);

    // Frame rows at the ends of the band's range first .. first + L + 1.
    // The last two are still in slots L and L + 1 (mod 3).
    switch (L % 3) {
        case 0: jit_last_rows<O, 0, 1>(S, first, L, X); break;
        case 1: jit_last_rows<O, 1, 2>(S, first, L, X); break;
        default: jit_last_rows<O, 2, 0>(S, first, L, X); break;
    }
    // The first two, from the cell (row first + 1 is row first + L when L = 1).
    {
        const uint4 q = ring[kJitRing * 4 * kJitterThreads];
        jit_add_row(first, first, L, Acc2{q.x, q.y}, X);
        if (L >= 2) jit_add_row(first + 1, first, L, Acc2{q.z, q.w}, X);
    }
    if (TABLE) return;
    // In-loop sum b^2: template rows whose partner row is valid for some but
    // not all u, i + s0 in {-1, 0, m - 1, m}.
    for (int k = 0; k < 4; ++k) {
        const int i = (k < 2 ? -1 + k : B.m - 3 + k) - B.s0;
        if (i < B.i_b || i >= B.i_e || i < 0 || i >= B.m) continue;
        const uint4 q = jit_tmpl_row(B, i);
        const uint32_t bw[4] = {q.x, q.y, q.z, q.w};
        uint32_t bp[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) bp[p] = byte_planes(bw[p]);
        Acc2 e[3] = {{0u, 0u}, {0u, 0u}, {0u, 0u}};
        tmpl_energy(bw, bp, cm, e);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int r = i + B.s0 - 1 + u;
            if (r >= 0 && r < B.m)
#pragma unroll
                for (int v = 0; v < 3; ++v) X[u * 3 + v] += acc_value(e[v]);
        }
    }
}

// sum of b^2 over the template rows [i0, i1) x columns [j0, j1) from the
// prefix table P[i][j] = sum_{i' < i, j' < j} b^2, (m+1) x (n+1).
__device__ __forceinline__ u64 rect_sum(const u64* __restrict__ P, int n, int i0, int i1, int j0, int j1) {
    if (i1 <= i0 || j1 <= j0) return 0ull;
    const int64_t ld = n + 1;
    return P[i1 * ld + j1] - P[i0 * ld + j1] - P[i1 * ld + j0] + P[i0 * ld + j0];
}

// Returns 1 when S1/A1 < S2/A2 exactly (A > 0); *eq when equal.
__device__ __forceinline__ int ratio_lt(u64 S1, u64 A1, u64 S2, u64 A2, int* eq) {
    const u64 l_lo = S1 * A2, l_hi = __umul64hi(S1, A2);
    const u64 r_lo = S2 * A1, r_hi = __umul64hi(S2, A1);
    *eq = (l_lo == r_lo) && (l_hi == r_hi);
    return (l_hi < r_hi) || (l_hi == r_hi && l_lo < r_lo);
}

// One stack's refinement: its frames, template, b^2 table (TABLE) or nullptr,
// searched-grid optima in, final shifts (and costs) out, and the per-frame
// scratch (nine sums and a ticket, zero on entry).
struct JitParams {
    const uint16_t* frames;
    int64_t fstride;
    const uint16_t* tmpl;
    const u64* bsq;
    const int32_t* coarse;
    int32_t* shifts;
    double* ffinal;
    u64* acc;
    unsigned int* ticket;
    int m, n, band_rows, witems;  // witems: warp items (32 band-and-column-group tasks) per frame
};

__device__ __forceinline__ u64 ld_relaxed_u64(const u64* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// The best of nine candidates held by lanes 0-8 of the warp (S / A with the
// tie-break: smallest ratio, then |s| + |t|, then s, then t; exact 128-bit
// cross products), taken in order by every lane from shuffles.
__device__ __forceinline__ void choose_nine(u64 S, u64 A, int s, int t, u64& bS, u64& bA, int& bs, int& bt) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const u64 Sk = __shfl_sync(0xffffffffu, S, k), Ak = __shfl_sync(0xffffffffu, A, k);
        const int sk = __shfl_sync(0xffffffffu, s, k), tk = __shfl_sync(0xffffffffu, t, k);
        bool take = (k == 0);
        if (!take) {
            int eq;
            const int lt = ratio_lt(Sk, Ak, bS, bA, &eq);
            if (lt) take = true;
            else if (eq) {
                const int k1 = abs(sk) + abs(tk), k2 = abs(bs) + abs(bt);
                take = (k1 < k2) || (k1 == k2 && (sk < bs || (sk == bs && tk < bt)));
            }
        }
        if (take) { bS = Sk; bA = Ak; bs = sk; bt = tk; }
    }
}

// Frame f's final shift from its nine complete sums (every item's additions
// visible): lane k < 9 forms candidate (u, v) = (k / 3, k % 3), its S (the
// table's b^2 added) and overlap A; every lane then takes the nine in order,
// smallest S/A first, ties to the smaller |s| + |t|, then s, then t, with
// exact 128-bit cross products. Lane 0 writes the result.
template <bool TABLE>
__device__ __forceinline__ void jitter_choose(const JitParams& P, int64_t f, int s0, int t0, bool valid) {
    const int lane = threadIdx.x & 31, m = P.m, n = P.n;
    u64 S = 0, A = 1;
    int s = 0, t = 0;
    if (lane < 9) {
        s = s0 + lane / 3 - 1;
        t = t0 + lane % 3 - 1;
        A = (u64)(m - abs(s)) * (u64)(n - abs(t));
        S = ld_relaxed_u64(P.acc + f * 9 + lane);
        if (TABLE) S += rect_sum(P.bsq, n, max(0, -s), m - max(0, s), max(0, -t), n - max(0, t));
    }
    u64 bS = 0, bA = 1;
    int bs = 0, bt = 0;
    choose_nine(S, A, s, t, bS, bA, bs, bt);
    if (lane != 0) return;
    P.shifts[2 * f] = valid ? bs : INT32_MIN;
    P.shifts[2 * f + 1] = valid ? bt : INT32_MIN;
    if (P.ffinal) P.ffinal[f] = valid ? (double)bS / (double)bA : __longlong_as_double(0x7ff8000000000000ll);
}

// The work of warp item `item` (of P.witems) of frame f: tasks item * 32 +
// lane, task = band * G + g (G = n / 8 column groups), each lane its band's
// nine partial sums; the warp adds their totals to the frame's scratch, and
// the frame's last item to finish (ticket counter) takes the minimum. Every
// lane of the warp calls it; no other warp is waited for.
template <bool TABLE>
__device__ __forceinline__ void jitter_item(const JitParams& P, int64_t f, int item, uint4* ring) {
    const int m = P.m, n = P.n, band_rows = P.band_rows;
    const uint16_t* __restrict__ frames = P.frames;
    const int64_t fstride = P.fstride;
    const int lane = threadIdx.x & 31;
    // Every candidate needs a non-empty overlap: |2 sc| + 1 < m, |2 tc| + 1 < n
    // (always so for a searched-grid optimum; checked for caller-given ones).
    // A frame outside that range is computed at (0, 0), so every index stays
    // in range, and reported as (INT32_MIN, INT32_MIN).
    const int sc = P.coarse[2 * f], tc = P.coarse[2 * f + 1];
    const bool valid = sc >= -((m - 2) >> 1) && sc <= ((m - 2) >> 1) && tc >= -((n - 2) >> 1) && tc <= ((n - 2) >> 1);
    const int s0 = valid ? 2 * sc : 0, t0 = valid ? 2 * tc : 0;
    u64 X[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = 0;
    const int G = n / 8;
    const int nb = (m + band_rows - 1) / band_rows;  // band_rows <= kJitRows
    const int task = item * 32 + lane;
    int e_first = 0, e_L = 0;  // this lane's band, for the end-column terms
    uint32_t e_need = 0;
    if (task < G * nb) {
        const int g = task % G, band = task / G;
        JitBand B;
        B.a = frames + f * fstride;
        B.tmpl = P.tmpl;
        B.m = m;
        B.n = n;
        B.s0 = s0;
        B.j0 = 8 * g;
        const int lead = B.j0 + t0 - 1;  // odd
        // Word (lead - 1) / 2 of the row is word O of chunk 0.
        const int O = ((t0 >> 1) - 1) & 3;  // the same for the whole frame
        B.c0 = lead - 1 - 2 * O;
        B.i_b = band * band_rows;
        B.i_e = min(m, B.i_b + band_rows);
        B.first = B.i_b + s0 - 1;
        B.cvalid = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (B.c0 + 8 * c >= 0 && B.c0 + 8 * c + 8 <= n) B.cvalid |= 1u << c;
        uint32_t mask = 0;  // bit v*8+k: frame column lead+k+v inside the frame
        if (!TABLE) {
#pragma unroll
            for (int v = 0; v < 3; ++v)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int c = lead + k + v;
                    if (c >= 0 && c < n) mask |= 1u << (v * 8 + k);
                }
        }
        switch (O) {
            case 0: jit_band<TABLE, 0>(B, ring, mask, X); break;
            case 1: jit_band<TABLE, 1>(B, ring, mask, X); break;
            case 2: jit_band<TABLE, 2>(B, ring, mask, X); break;
            default: jit_band<TABLE, 3>(B, ring, mask, X); break;
        }
        e_need = (g == 0 ? 1u : 0u) | (g == G - 1 ? 2u : 0u);
        e_first = B.first;
        e_L = B.i_e - B.i_b;
    }
    jit_edge_columns(frames + f * fstride, m, n, t0, e_first, e_L, e_need, X);
    u64 mine = 0;  // lane k < 9: the warp's total of sum k
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        u64 v = X[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == k) mine = v;
    }
    if (lane < 9) atomicAdd(&P.acc[f * 9 + lane], mine);
    __threadfence();  // the sums before the ticket
    __syncwarp();
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(&P.ticket[f], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t != (unsigned int)P.witems - 1) return;
    __threadfence();  // the other items' sums, seen through their tickets
    jitter_choose<TABLE>(P, f, s0, t0, valid);
}

// Grid (ceil(witems / 8), frames): warp w of CTA x takes item 8 x + w.
template <bool TABLE>
__global__ void __launch_bounds__(kJitterThreads, TABLE ? 3 : 1) k_jitter(JitParams P) {
    extern __shared__ __align__(16) unsigned char jit_smem[];
    uint4* ring = reinterpret_cast<uint4*>(jit_smem) + threadIdx.x;  // kJitSmemBytes
    const int item = blockIdx.x * (kJitterThreads / 32) + (threadIdx.x >> 5);
    if (item >= P.witems) return;  // the whole warp
    jitter_item<TABLE>(P, blockIdx.y, item, ring);
}

// The refinement of one or several stacks (shapes, templates) in one launch:
// a grid over the (stack, frame, warp item) work items of every segment,
// warp w of CTA x taking item i = 8 x + w. Item i belongs to the segment k
// with item_base[k] <= i < item_base[k + 1] (segment k covers P[k].witems
// items of each of its frames). A segment is a run of one stack's frames; its
// P pointers are already offset to the run's first frame. (A persistent form,
// resident warps striding over the items, ran slower here, and one fetching
// items from a shared counter slower still: every fetch hit one address.)
constexpr int kJitSegs = 40;  // segments per launch (the parameters stay under 4 KiB)
struct JitBatch {
    JitParams P[kJitSegs];
    int64_t item_base[kJitSegs + 1];
    int nseg;
};
static_assert(sizeof(JitBatch) <= 4096, "kernel parameters of k_jitter_multi");

static __global__ void __launch_bounds__(kJitterThreads, 3) k_jitter_multi(const __grid_constant__ JitBatch batch) {
    extern __shared__ __align__(16) unsigned char jit_smem[];
    uint4* ring = reinterpret_cast<uint4*>(jit_smem) + threadIdx.x;  // kJitSmemBytes
    const long long i = (long long)blockIdx.x * (kJitterThreads / 32) + (threadIdx.x >> 5);
    if (i >= batch.item_base[batch.nseg]) return;  // the whole warp
    int k = 0;
    while (k + 1 < batch.nseg && batch.item_base[k + 1] <= i) ++k;
    const JitParams& P = batch.P[k];
    const long long local = i - batch.item_base[k];
    jitter_item<true>(P, local / P.witems, (int)(local % P.witems), ring);
}

// Prefix table of b^2 for k_jitter, P[(m+1) x (n+1)] (exact u64), in two
// passes. k_sq_prefix_rows: one warp per row, 32-wide warp scans with a
// carry (row 0 and column 0 zero). k_sq_prefix_cols: one CTA of 32 warps per
// 32 columns; warp w owns a slice of rows: the slice's column sums, an
// exclusive sum over the earlier slices, then the slice rewritten as running
// sums (two passes over P, each coalesced along the columns).
static __global__ void __launch_bounds__(256) k_sq_prefix_rows(const uint16_t* __restrict__ tmpl, int m, int n,
                                                               u64* __restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t ld = n + 1;
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j <= n; j += blockDim.x) P[j] = 0;
    if (i >= m) return;
    u64* row = P + (int64_t)(i + 1) * ld;
    if (lane == 0) row[0] = 0;
    u64 carry = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        u64 v = 0;
        if (j < n) {
            const u64 b = tmpl[(int64_t)i * n + j];
            v = b * b;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        v += carry;
        if (j < n) row[j + 1] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

static __global__ void __launch_bounds__(1024) k_sq_prefix_cols(int m, int n, u64* __restrict__ P) {
    __shared__ u64 part[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;  // column of P
    const int64_t ld = n + 1;
    const int slice = (m + 31) / 32;
    const int r0 = 1 + w * slice, r1 = min(m + 1, r0 + slice);  // rows [r0, r1) of P
    u64 s = 0;
    if (j <= n)
        for (int r = r0; r < r1; ++r) s += P[(int64_t)r * ld + j];
    part[w][lane] = s;
    __syncthreads();
    u64 run = 0;
    for (int k = 0; k < w; ++k) run += part[k][lane];
    if (j <= n)
        for (int r = r0; r < r1; ++r) {
            run += P[(int64_t)r * ld + j];
            P[(int64_t)r * ld + j] = run;
        }
}

// For searches without a level: the searched optimum is the answer.
static __global__ void k_copy_shifts(const int32_t* __restrict__ coarse, int32_t* __restrict__ shifts,
                              const double* __restrict__ fbest, double* __restrict__ ffinal, int64_t T) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < 2 * T) shifts[i] = coarse[i];
    if (ffinal && i < T) ffinal[i] = fbest[i];
}

// ---------------------------------------------------------------------------
// Template offset c = round(mean of the searched-grid template), integer.
// U16: exact integer sum of the (box-summed) template; F32: FP64 sum of FP32
// partial sums (the rounding of the mean only needs it near). Two kernels:
// k_offset_partial, CTA b summing a slice of rows into part[b] (bits of a u64
// or a double), then k_offset_final adding the parts in order.
template <bool F32>
__global__ void __launch_bounds__(256)
k_offset_partial(const void* __restrict__ tmpl, int m, int n, int levels, u64* __restrict__ part) {
    __shared__ u64 redu[8];
    __shared__ double redd[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mc = m >> levels, nc = n >> levels;
    const int rows = mc << levels, cols = nc << levels;  // the pixels the searched grid covers
    const int i0 = (int)((int64_t)blockIdx.x * rows / gridDim.x), i1 = (int)((int64_t)(blockIdx.x + 1) * rows / gridDim.x);
    u64 su = 0;
    double sd = 0.0;
    for (int i = i0 + warp; i < i1; i += 8) {
        float rf = 0.f;
        for (int j = lane; j < cols; j += 32) {
            if (F32) rf += static_cast<const float*>(tmpl)[(int64_t)i * n + j];
            else su += static_cast<const uint16_t*>(tmpl)[(int64_t)i * n + j];
        }
        sd += (double)rf;
    }
    su = warp_sum(su);
    sd = warp_sum(sd);
    if (lane == 0) { redu[warp] = su; redd[warp] = sd; }
    __syncthreads();
    if (tid == 0) {
        u64 tu = 0;
        double td = 0.0;
        for (int k = 0; k < 8; ++k) { tu += redu[k]; td += redd[k]; }
        part[blockIdx.x] = F32 ? (u64)__double_as_longlong(td) : tu;
    }
}

template <bool F32>
__global__ void k_offset_final(const u64* __restrict__ part, int nparts, int m, int n, int levels,
                               int32_t* __restrict__ coff_i, float* __restrict__ coff_f) {
    const u64 cnt = (u64)(m >> levels) * (u64)(n >> levels);
    u64 tu = 0;
    double td = 0.0;
    for (int k = 0; k < nparts; ++k) {
        if (F32) td += __longlong_as_double((long long)part[k]);
        else tu += part[k];
    }
    if (F32) {
        const double c = rint(td / (double)cnt);
        *coff_i = (int32_t)c;
        *coff_f = (float)c;
    } else {
        const u64 c = (2 * tu + cnt) / (2 * cnt);  // round half up of the mean
        *coff_i = (int32_t)c;
        *coff_f = (float)c;
    }
}

}  // namespace moco
