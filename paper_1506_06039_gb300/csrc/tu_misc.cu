// Energies, jitter, template offset, and small host helpers.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "fft_sizes.h"
#include "internal.h"
#include "kernels.cuh"

namespace moco {

bool fft_size_supported(int N) {
#define MOCO_CASE(NN) if (N == NN) return true;
    MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
#undef MOCO_CASE
    return false;
}

int fft_size_for(int needed) {
    int best = 0;
#define MOCO_CASE(NN) if (NN >= needed && (best == 0 || NN < best)) best = NN;
    MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
#undef MOCO_CASE
    return best;
}

bool fft_split(int N, int* n1, int* n2) {
#define MOCO_CASE(NN) \
    if (N == NN) { *n1 = Four<NN>::N1; *n2 = Four<NN>::N2; return true; }
    MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
#undef MOCO_CASE
    return false;
}

int fft_split_max(int N) {
#define MOCO_CASE(NN) if (N == NN) return Four<NN>::N1 > Four<NN>::N2 ? Four<NN>::N1 : Four<NN>::N2;
    MOCO_FOR_EACH_FFT_SIZE(MOCO_CASE)
#undef MOCO_CASE
    return 0;
}

cudaError_t ensure_smem(const void* func, size_t bytes) {
    // The limit only ever grows: a launch with less shared memory must not
    // lower it under a launch that needs more.
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[std::make_pair(func, dev)];
    // (also below 48 KiB: the default limit counts the kernel's static shared
    // memory too, so dynamic + static may exceed it)
    if (bytes == 0 || bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    cur = bytes;
    return cudaSuccess;
}

cudaError_t launch_energy(bool f32, bool out_double, const u64* rowE, const u64* colE, const u64* tot,
                          const uint32_t* corners, int64_t nimg, int mc, int nc, int wm1, void* out, int flip,
                          cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    // exR, exC and the corner tables (8-byte Acc), or the warp sweep's carries
    const size_t smem = std::max(energy_smem(wm1, 8, energy_qp(wm1, 8)), energy_sweep_smem(wm1, kEnergyThreads / 32));
    const void* fn = f32 ? (out_double ? (const void*)k_energy<true, true> : (const void*)k_energy<true, false>)
                         : (out_double ? (const void*)k_energy<false, true> : (const void*)k_energy<false, false>);
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    if (f32) {
        if (out_double) k_energy<true, true><<<(unsigned)nimg, kEnergyThreads, smem, st>>>(rowE, colE, tot, corners, mc, nc, wm1, out, flip);
        else k_energy<true, false><<<(unsigned)nimg, kEnergyThreads, smem, st>>>(rowE, colE, tot, corners, mc, nc, wm1, out, flip);
    } else {
        if (out_double) k_energy<false, true><<<(unsigned)nimg, kEnergyThreads, smem, st>>>(rowE, colE, tot, corners, mc, nc, wm1, out, flip);
        else k_energy<false, false><<<(unsigned)nimg, kEnergyThreads, smem, st>>>(rowE, colE, tot, corners, mc, nc, wm1, out, flip);
    }
    return cudaGetLastError();
}

static __global__ void k_pair_from_double(const double* __restrict__ x, float2* __restrict__ out, int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const float hi = (float)x[k];
    out[k] = make_float2(hi, (float)(x[k] - (double)hi));
}

cudaError_t launch_pair_from_double(const double* x, float2* out, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_pair_from_double<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(x, out, count);
    return cudaGetLastError();
}

// Warp items per frame (32 band-and-column-group tasks each) and the band
// height: bands of kJitRows rows; a small batch (fewer warps than two waves of
// eight per SM) takes bands of 16 or 8 rows so that more warps share a frame.
static void jitter_shape(int m, int n, int64_t nimg, int num_sms, int* band_rows, int* witems) {
    int br = kJitRows;
    auto items_for = [&](int b) { return ((n / 8) * ((m + b - 1) / b) + 31) / 32; };
    while (br > 8 && (int64_t)items_for(br) * nimg < 2 * (int64_t)num_sms * (kJitterThreads / 32)) br /= 2;
    *band_rows = br;
    *witems = items_for(br);
}

cudaError_t launch_jitter(const uint16_t* frames, int64_t fstride, int64_t nimg, const uint16_t* tmpl, int m,
                          int n, const u64* bsq, const int32_t* coarse, int32_t* shifts, double* ffinal, u64* acc,
                          unsigned int* ticket, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(u64) * 9 * nimg, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int) * nimg, st);
    if (e != cudaSuccess) return e;
    JitParams P;
    P.frames = frames;
    P.fstride = fstride;
    P.tmpl = tmpl;
    P.bsq = bsq;
    P.coarse = coarse;
    P.shifts = shifts;
    P.ffinal = ffinal;
    P.acc = acc;
    P.ticket = ticket;
    P.m = m;
    P.n = n;
    jitter_shape(m, n, nimg, 152, &P.band_rows, &P.witems);
    constexpr int wpc = kJitterThreads / 32;  // warps (items) per CTA
    dim3 grid((unsigned)((P.witems + wpc - 1) / wpc), (unsigned)nimg);
    const void* fn = bsq ? reinterpret_cast<const void*>(k_jitter<true>) : reinterpret_cast<const void*>(k_jitter<false>);
    e = ensure_smem(fn, kJitSmemBytes);
    if (e != cudaSuccess) return e;
    if (bsq) k_jitter<true><<<grid, kJitterThreads, kJitSmemBytes, st>>>(P);
    else k_jitter<false><<<grid, kJitterThreads, kJitSmemBytes, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_jitter_multi(const JitSegment* segs, int nseg, u64* acc, unsigned int* ticket, int64_t capacity,
                                int num_sms, cudaStream_t st) {
    int k0 = 0;
    while (k0 < nseg) {
        // The next launch: up to kJitSegs segments whose frames fit the scratch.
        int ns = 0;
        int64_t frames = 0;
        while (k0 + ns < nseg && ns < kJitSegs) {
            const JitSegment& g = segs[k0 + ns];
            if (g.T > capacity || !g.bsq) return cudaErrorInvalidValue;
            if (frames + g.T > capacity) break;
            frames += g.T;
            ++ns;
        }
        JitBatch batch;
        int64_t items = 0, f = 0;
        for (int k = 0; k < ns; ++k) {
            const JitSegment& g = segs[k0 + k];
            JitParams& P = batch.P[k];
            P.frames = g.frames;
            P.fstride = g.fstride;
            P.tmpl = g.tmpl;
            P.bsq = g.bsq;
            P.coarse = g.coarse;
            P.shifts = g.shifts;
            P.ffinal = g.ffinal;
            P.acc = acc + 9 * f;
            P.ticket = ticket + f;
            P.m = g.m;
            P.n = g.n;
            // bands sized by the whole launch's frames
            jitter_shape(g.m, g.n, frames, num_sms, &P.band_rows, &P.witems);
            batch.item_base[k] = items;
            items += g.T * P.witems;
            f += g.T;
        }
        batch.nseg = ns;
        batch.item_base[ns] = items;
        k0 += ns;
        if (items == 0) continue;
        cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(u64) * 9 * frames, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int) * frames, st);
        if (e == cudaSuccess) e = ensure_smem(reinterpret_cast<const void*>(k_jitter_multi), kJitSmemBytes);
        if (e != cudaSuccess) return e;
        constexpr int wpc = kJitterThreads / 32;  // warps (items) per CTA
        k_jitter_multi<<<(unsigned)((items + wpc - 1) / wpc), kJitterThreads, kJitSmemBytes, st>>>(batch);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sq_prefix(const uint16_t* tmpl, int m, int n, u64* P, cudaStream_t st) {
    k_sq_prefix_rows<<<(m + 7) / 8, 256, 0, st>>>(tmpl, m, n, P);
    k_sq_prefix_cols<<<(n + 1 + 31) / 32, 1024, 0, st>>>(m, n, P);
    return cudaGetLastError();
}

cudaError_t launch_copy_shifts(const int32_t* coarse, int32_t* shifts, const double* fbest, double* ffinal,
                               int64_t T, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (2 * T + threads - 1) / threads;
    k_copy_shifts<<<(unsigned)blocks, threads, 0, st>>>(coarse, shifts, fbest, ffinal, T);
    return cudaGetLastError();
}

cudaError_t launch_template_offset(bool f32, const void* tmpl, int m, int n, int levels, int32_t* coff_i,
                                   float* coff_f, u64* part, int64_t nparts, cudaStream_t st) {
    const int rows = (m >> levels) << levels;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>({nparts, 64, (int64_t)std::max(1, rows)}));
    if (f32) k_offset_partial<true><<<blocks, 256, 0, st>>>(tmpl, m, n, levels, part);
    else k_offset_partial<false><<<blocks, 256, 0, st>>>(tmpl, m, n, levels, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (f32) k_offset_final<true><<<1, 1, 0, st>>>(part, blocks, m, n, levels, coff_i, coff_f);
    else k_offset_final<false><<<1, 1, 0, st>>>(part, blocks, m, n, levels, coff_i, coff_f);
    return cudaGetLastError();
}

// The timeout path's check: an mbarrier that expects one arrival nobody
// makes, waited on by the staged kernels' bounded wait (about a second by
// clock64), which then sets *err and returns. No asynchronous copy is issued,
// so nothing is in flight when the CTA exits.
__global__ void k_wait_selftest(unsigned int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_wait(&bar, 0u, err);
    }
}

cudaError_t launch_wait_selftest(unsigned int* err, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err);
    return cudaGetLastError();
}

}  // namespace moco
