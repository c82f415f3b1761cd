// The direct form of the cross term h_st (Section 2's third sum) on the 5th
// generation tensor cores:
//
//   h[f][(s,t)] = sum_{(p,q)} A[f][(p,q)] * B[(p,q)][(s,t)],
//   A[f][(p,q)] = a'_f[p][q],   B[(p,q)][(s,t)] = b'[p-s][q-t] (0 outside),
//
// a GEMM with M = frames, N = shifts and K = searched-grid pixels. a' and b'
// are integers (offset by the plan's c) up to 2^19 in magnitude; each is
// split into BF16 hi + lo (16 significant bits) and the product is formed as
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.
//
// For one K step (image row p, 64 columns from q0) and one shift row s, the
// B block is the 64 x Wp Toeplitz matrix of template row r = p - s. Builder
// warps write these blocks into shared memory each step, in the MMA's
// canonical K-major layout without swizzle (8 x 8 core matrices of 128
// bytes, 128 bytes apart along K and 1024 bytes apart along N), from a
// per-template table of the rows in 8 phase-shifted copies
// (k_toeplitz_rows), so that each 16-byte chunk is one aligned load. A
// tiles (128 frames x 64 pixels, BF16 hi and lo planes written by the frame
// pass) come in as one TMA tensor load per plane (box 64 pixels x 1 row x
// 128 frames, 128-byte swizzle: the MMA's swizzled K-major layout; frames
// past the batch read as zeros). The kernel is warp-specialised: a TMA warp,
// an MMA-issuing thread, builder warps and drain warps, three stages deep,
// meeting only on mbarriers (k_direct below); every wait is bounded (about a
// second) and sets an error flag instead of hanging.
//
// Accumulation: the tensor core's FP32 accumulator loses low bits on each
// accumulation, which over the 12 MMAs x (mc * nc / 64) K steps of a frame
// would bias h. So each group of kDirGroup K steps accumulates into a fresh
// TMEM accumulator (two of them, alternating), issuing the small hi*lo and
// lo*hi products before the hi*hi ones, and every thread adds the finished
// accumulator of its frame into round-to-nearest FP32 registers.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace moco {

// Warp roles of k_direct (ten warps): warp 0 issues the A tiles' TMA loads,
// warp 1 the MMAs (one thread each), warps 2-5 drain the accumulators (warp
// w reads TMEM lanes 32 (w % 4) .. + 31, so the four cover the 128 frames),
// warps 6-9 build the B tiles in shared memory (thread t owns B row t).
constexpr int kDirThreads = 320;
constexpr int kDirWarpTma = 0, kDirWarpMma = 1, kDirWarpDrain = 2, kDirWarpBuild = 6;
constexpr int kDirM = 128;      // frames per tile (MMA M)
constexpr int kDirK = 64;       // pixels per K step
constexpr int kDirQ = kDirK;    // columns per K step
constexpr int kDirNmax = 128;   // MMA N (shifts per tile)

__host__ __device__ inline int direct_wp(int W) { return (W + 15) / 16 * 16; }
__host__ __device__ inline int direct_ns(int W) { return kDirNmax / direct_wp(W); }
__host__ __device__ inline size_t direct_tile_bytes(int W) { return (size_t)direct_wp(W) * kDirK * 2; }
constexpr size_t kDirAStage = 2 * (size_t)kDirM * kDirK * 2;    // A tiles of a step, both planes
constexpr size_t kDirBStage = 2 * (size_t)kDirNmax * kDirK * 2; // B tiles of a step, both planes
constexpr int kDirStages = 3;  // operands are prepared up to three K steps ahead of the MMAs
constexpr int kDirGroup = 2;   // K steps summed in one TMEM accumulator before it is drained
__host__ __device__ inline size_t direct_smem_bytes(int /*W*/) {
    return 1024 + kDirStages * (kDirAStage + kDirBStage) + 64;
}

// Byte offset of element (row, k) in a K-major core-matrix tile with 64 K.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// The template rows the B (Toeplitz) tiles are built from. For template row
// r, column chunk qc and shift column ti (t = ti - (w-1)), a tile holds
// B[k][ti] = b'[r][qc*64 + k - ti + (w-1)] (zero outside [0, nc) and for
// ti >= W). A 16-byte chunk of it (8 consecutive k at one ti) is 8
// consecutive template values: the table keeps each row of b' (hi and lo
// BF16 planes) zero-padded by Wp on the left, in 8 copies shifted by one
// value each, so that every chunk is one aligned 16-byte load (which hits
// L1: a K step's tiles need NS rows of the table):
//   rows[plane][r][ph][x] = b'[r][x + ph - Wp]   (x < Lq, zero outside).
__host__ __device__ inline int direct_row_len(int W, int ncp) {
    return (direct_wp(W) + ncp + (W - 1) / 2 + 16 + 7) / 8 * 8;
}
__host__ __device__ inline size_t direct_rows_bytes(int mc, int ncp, int W) {
    return 2 * (size_t)mc * 8 * direct_row_len(W, ncp) * 2;
}

static __global__ void k_toeplitz_rows(const float* __restrict__ bprime, int mc, int nc, int ncp, int wm1,
                                       __nv_bfloat16* __restrict__ rows) {
    const int W = 2 * wm1 + 1, Wp = direct_wp(W), Lq = direct_row_len(W, ncp);
    const int64_t per_plane = (int64_t)mc * 8 * Lq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per_plane;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % Lq);
        const int ph = (int)((e / Lq) % 8);
        const int r = (int)(e / ((int64_t)Lq * 8));
        const int col = x + ph - Wp;
        const float v = (col >= 0 && col < nc) ? bprime[(int64_t)r * nc + col] : 0.f;
        __nv_bfloat16 hi, lo;
        split_bf16(v, hi, lo);
        rows[e] = hi;
        rows[per_plane + e] = lo;
    }
}

// ---- PTX wrappers ------------------------------------------------------------

// smem_u32, mbarrier, bulk-copy and cp.async wrappers: ptx.cuh.
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major, no swizzle: core matrices 128 B apart along K, 1024 B along M/N.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t a = smem_u32(p);
    return ((a >> 4) & 0x3FFFull) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46);
}
// K-major with 128-byte swizzle (as a TMA load with that swizzle writes a
// box whose rows are 128 bytes): 8-row groups 1024 bytes apart; the start
// address advances by 32 bytes per 16-element K slice within the row.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
    const uint64_t a = smem_u32(p);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// 3-D tiled TMA load of the box at (x, y, z) into shared memory, completing
// on the mbarrier's transaction count.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t direct_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Adds the accumulator at TMEM address `addr` (this warp's 32 lanes, N
// columns) into hsum (column c of this thread's lane).
__device__ __forceinline__ void drain_acc(uint32_t addr, int N, float (&hsum)[kDirNmax]) {
    tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < kDirNmax; c0 += 32) {
        if (c0 < N) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(addr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 32; ++c) hsum[c0 + c] += __uint_as_float(r[c]);
        }
    }
    tc_fence_before();
}

// ---- the GEMM ----------------------------------------------------------------
//
// Grid (N tiles, M tiles, K splits). N tile j covers shift rows s = -(w-1) +
// j*NS .. (NS = 128 / Wp of them, Wp = W rounded up to 16); M tile covers
// frames f0 .. f0 + 127; K split z covers K steps [z K / Z, (z+1) K / Z)
// (K = mc * nqc, Z = gridDim.z) and writes its partial sum to
// h[z][f][(s+w-1)*W + (t+w-1)] (FP32, z-th slab of T * W * W), which the
// combine adds up in order of z. Splitting K keeps every SM busy when the
// window is small (few N tiles) or the batch short (few M tiles).
//
// The warps meet only on mbarriers (every wait bounded: about a second, then
// the error flag and an orderly exit):
//   full_a[st]  the TMA warp's loads of step k's A tiles landed (transaction
//               count), stage st = k % kDirStages;
//   full_b[st]  the 128 builder threads stored step k's B tiles (and fenced
//               them for the tensor core's asynchronous reads);
//   empty[st]   step k's MMAs completed (tcgen05.commit): the stage is free;
//   acc_full[a] a group's MMAs into accumulator a completed (commit);
//   acc_empty[a] the 128 drain threads have read accumulator a.
// The MMA thread issues step k's 12 MMAs as soon as its operands are ready
// and, at a group's first step, the accumulator it reuses has been drained;
// loads and builds run up to three steps ahead, drains one group behind.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

static __global__ void __launch_bounds__(kDirThreads, 1)
k_direct(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo, int64_t T, int mc,
         int ncp, int nqc, int wm1, const __nv_bfloat16* __restrict__ rows, float* __restrict__ h,
         unsigned int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_a[kDirStages], full_b[kDirStages], empty[kDirStages];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int s_consumed;  // K steps whose A tiles the MMA thread has seen land
    const int W = 2 * wm1 + 1, Wp = direct_wp(W), NS = direct_ns(W), N = NS * Wp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s_first = -wm1 + (int)blockIdx.x * NS;
    const int64_t f0 = (int64_t)blockIdx.y * kDirM;
    const int kall = mc * nqc;
    const int kb = (int)((int64_t)blockIdx.z * kall / gridDim.z);
    const int ksteps = (int)((int64_t)(blockIdx.z + 1) * kall / gridDim.z) - kb;  // this split's K steps
    const int ngroups = (ksteps + kDirGroup - 1) / kDirGroup;
    h += (int64_t)blockIdx.z * T * W * W;
    constexpr uint32_t kTmemCols = 2 * kDirNmax;  // two accumulators

    if (tid == 0) {
        for (int i = 0; i < kDirStages; ++i) {
            mbar_init(&full_a[i], 1);
            mbar_init(&full_b[i], 128);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 128);
        }
        s_abort = 0;
        s_consumed = 0;
        fence_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    auto sA = [&](int st, int plane) { return dsm + st * kDirAStage + (size_t)plane * kDirM * kDirK * 2; };
    auto sB = [&](int st, int plane) {
        return dsm + kDirStages * kDirAStage + st * kDirBStage + (size_t)plane * (kDirBStage / 2);
    };
    // A bounded wait that also gives up at once when another role already has.
    auto wait = [&](uint64_t* bar, uint32_t parity) {
        if (s_abort) return false;
        if (mbar_wait(bar, parity, err)) return true;
        s_abort = 1;
        return false;
    };

    if (warp == kDirWarpTma) {
        // A tiles: one TMA tensor load per plane and step (frames past the batch read as zeros).
        if (lane == 0) {
            int issued = 0;
            for (int k = 0; k < ksteps; ++k) {
                const int st = k % kDirStages;
                if (k >= kDirStages && !wait(&empty[st], ((k / kDirStages) - 1) & 1)) break;
                const int kk = kb + k, p = kk / nqc, qc = kk - p * nqc;
                mbar_expect_tx(&full_a[st], (uint32_t)kDirAStage);
                tma_load_3d(sA(st, 0), &tmap_hi, qc * kDirQ, p, (int)f0, &full_a[st]);
                tma_load_3d(sA(st, 1), &tmap_lo, qc * kDirQ, p, (int)f0, &full_a[st]);
                issued = k + 1;
            }
            if (s_abort) {
                // Leave no copy in flight into shared memory: wait (bounded) for the
                // loads of the last stages that the MMA thread has not seen land.
                for (int k = max(s_consumed, issued - kDirStages); k < issued; ++k)
                    mbar_wait(&full_a[k % kDirStages], (k / kDirStages) & 1, err);
            }
        }
    } else if (warp == kDirWarpMma) {
        if (lane == 0) {
            const uint32_t idesc = direct_idesc(kDirM, N);
            int committed = -1;  // last step whose MMAs were committed
            for (int k = 0; k < ksteps; ++k) {
                const int st = k % kDirStages, par = (k / kDirStages) & 1;
                const int g = k / kDirGroup, acc = g & 1;
                if (!wait(&full_a[st], (uint32_t)par)) break;
                s_consumed = k + 1;
                if (!wait(&full_b[st], (uint32_t)par)) break;
                // a group's first step reuses the accumulator of group g - 2: drained?
                if (k % kDirGroup == 0 && g >= 2 && !wait(&acc_empty[acc], ((g - 2) >> 1) & 1)) break;
                tc_fence_after();
                const unsigned char* A0 = sA(st, 0);
                const unsigned char* A1 = sA(st, 1);
                const unsigned char* B0 = sB(st, 0);
                const unsigned char* B1 = sB(st, 1);
                const uint32_t d = tmem + (uint32_t)(acc * kDirNmax);
                // small terms first, then hi*hi; a fresh accumulator at each group's first step
                // per K16 slice: A 32 bytes along its swizzled row, B two core matrices (256 bytes)
                const uint32_t first = (k % kDirGroup == 0) ? 1u : 0u;
#pragma unroll
                for (int kk = 0; kk < kDirK / 16; ++kk) {
                    mma_bf16(d, smem_desc_sw128(A0 + kk * 32), smem_desc(B1 + kk * 256), idesc,
                             (kk > 0 || !first) ? 1u : 0u);
                    mma_bf16(d, smem_desc_sw128(A1 + kk * 32), smem_desc(B0 + kk * 256), idesc, 1u);
                }
#pragma unroll
                for (int kk = 0; kk < kDirK / 16; ++kk)
                    mma_bf16(d, smem_desc_sw128(A0 + kk * 32), smem_desc(B0 + kk * 256), idesc, 1u);
                mma_commit(&empty[st]);
                if (k % kDirGroup == kDirGroup - 1 || k == ksteps - 1) mma_commit(&acc_full[acc]);
                committed = k;
            }
            // On an abort, the MMAs in flight finish (bounded wait) before the tensor
            // memory is released and the CTA's shared memory goes away.
            if (s_abort && committed >= 0)
                mbar_wait(&empty[committed % kDirStages], (committed / kDirStages) & 1, err);
        }
    } else if (warp >= kDirWarpBuild) {
        // B tiles: thread n owns B row n (shift column ti of tile sl): 64 consecutive
        // template values of one row of the table at a phase and offset fixed for
        // the thread, eight aligned 16-byte loads and stores per plane and step.
        const int n = tid - kDirWarpBuild * 32;
        const int sl = n / Wp, ti = n - sl * Wp;
        const bool col = n < N && ti < W && s_first + sl <= wm1;
        const int php = (Wp - ti + wm1) & 7;
        const int x0 = Wp - ti + wm1 - php;  // a multiple of 8: aligned chunks
        const uint32_t soff = (uint32_t)((n >> 3) * 1024 + (n & 7) * 16);
        const int Lq = direct_row_len(W, ncp);
        const size_t plane_rows = (size_t)mc * 8 * Lq;
        for (int k = 0; k < ksteps; ++k) {
            const int st = k % kDirStages;
            if (k >= kDirStages && !wait(&empty[st], ((k / kDirStages) - 1) & 1)) break;
            if (n < N) {
                const int kk = kb + k, p = kk / nqc, qc = kk - p * nqc;
                const int r = p - (s_first + sl);
                const bool live = col && r >= 0 && r < mc;
#pragma unroll
                for (int plane = 0; plane < 2; ++plane) {
                    unsigned char* dst = sB(st, plane) + soff;
                    uint4 v[8];
                    if (live) {
                        const uint4* src = reinterpret_cast<const uint4*>(
                            rows + plane * plane_rows + ((size_t)r * 8 + php) * Lq + qc * kDirQ + x0);
#pragma unroll
                        for (int kc = 0; kc < 8; ++kc) v[kc] = __ldg(src + kc);
                    } else {
#pragma unroll
                        for (int kc = 0; kc < 8; ++kc) v[kc] = make_uint4(0u, 0u, 0u, 0u);
                    }
#pragma unroll
                    for (int kc = 0; kc < 8; ++kc) *reinterpret_cast<uint4*>(dst + kc * 128) = v[kc];
                }
                fence_async_smem();  // the stores, visible to the tensor core's reads
            }
            mbar_arrive(&full_b[st]);
        }
    }
    // Drain warps: FP32 sum of this thread's frame row over the groups (round to
    // nearest, in group order), then the row's h values.
    float hsum[kDirNmax];
    const bool drainer = warp >= kDirWarpDrain && warp < kDirWarpBuild;
    if (drainer) {
#pragma unroll
        for (int c = 0; c < kDirNmax; ++c) hsum[c] = 0.f;
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int g = 0; g < ngroups; ++g) {
            const int acc = g & 1;
            if (!wait(&acc_full[acc], (g >> 1) & 1)) break;
            drain_acc(lane_addr + (uint32_t)(acc * kDirNmax), N, hsum);
            mbar_arrive(&acc_empty[acc]);
        }
    }
    __syncthreads();
    if (drainer && !s_abort) {
        const int64_t f = f0 + (warp & 3) * 32 + lane;
        if (f < T) {
#pragma unroll
            for (int c = 0; c < kDirNmax; ++c) {
                const int slc = c / Wp, tc = c - slc * Wp;
                const int s = s_first + slc;
                if (c < N && tc < W && s <= wm1) h[f * (int64_t)W * W + (int64_t)(s + wm1) * W + tc] = hsum[c];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Offset searched-grid template b' = b_c - c as floats (exact for uint16).
template <bool F32>
__global__ void k_coarse_image(const void* __restrict__ src, int m, int n, int levels, int mc, int nc,
                               const int32_t* __restrict__ coff_i, const float* __restrict__ coff_f,
                               float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)mc * nc;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / nc), j = (int)(e % nc);
        float v;
        if (F32) {
            v = static_cast<const float*>(src)[(int64_t)i * n + j] - *coff_f;
        } else {
            const uint16_t* s = static_cast<const uint16_t*>(src);
            int32_t x;
            if (levels)
                x = (int32_t)s[(int64_t)(2 * i) * n + 2 * j] + s[(int64_t)(2 * i + 1) * n + 2 * j] +
                    s[(int64_t)(2 * i) * n + 2 * j + 1] + s[(int64_t)(2 * i + 1) * n + 2 * j + 1];
            else
                x = s[(int64_t)i * n + j];
            v = (float)(x - *coff_i);
        }
        out[e] = v;
    }
}

// f = (Sa + Sb - 2 h) / Area * unit with the argmin and margin, from an h
// computed by the direct form. One CTA per frame.
// h is the sum, in order, of nsplit partial slabs of slab elements each.
static __global__ void __launch_bounds__(256)
k_combine_h(const float* __restrict__ hh, int nsplit, int64_t slab, int wm1, const float2* __restrict__ Sa2,
            const float2* __restrict__ Sb2, const float* __restrict__ ia32, double* __restrict__ cost,
            int32_t* __restrict__ coarse, double* __restrict__ fbest, float* __restrict__ margin) {
    __shared__ Best red[8];
    const int W = 2 * wm1 + 1, WW = W * W;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t f = blockIdx.x;
    Best b;
    b.f1 = INFINITY;
    b.r1 = 0x7fffffff;
    b.f2 = INFINITY;
    for (int k = tid; k < WW; k += nthr) {
        const int s = k / W - wm1, t = k % W - wm1;
        float hv = hh[f * WW + k];
        for (int z = 1; z < nsplit; ++z) hv += hh[z * slab + f * WW + k];
        const float fv = combine_f32(Sa2[f * WW + k], Sb2[k], hv, ia32[k]);
        if (cost) cost[f * WW + k] = f32_to_f64(fv);
        best_push(b, fv, (abs(s) + abs(t)) * WW + k);
    }
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
        for (int i = 1; i < nthr / 32; ++i) best_merge(b, red[i]);
        const int k = b.r1 % WW;
        coarse[2 * f] = k / W - wm1;
        coarse[2 * f + 1] = k % W - wm1;
        if (fbest) fbest[f] = (double)b.f1;
        if (margin) {
            float mg;
            if (b.f1 > 0) mg = (b.f2 - b.f1) / b.f1;
            else mg = (b.f2 > 0) ? INFINITY : 0.f;
            margin[f] = mg;
        }
    }
}

}  // namespace moco
