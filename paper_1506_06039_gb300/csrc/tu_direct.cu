// Launchers of the direct (tensor-core) form of the cross term.
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "kernels.cuh"
#include "direct.cuh"

namespace moco {

// The driver's tensor-map encoder, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// Frame planes [T][mc][ncp] BF16 as a 3-D tensor (column, row, frame) with
// boxes of 64 columns x 1 row x kDirM frames and 128-byte swizzle.
static cudaError_t plane_map(CUtensorMap* map, const void* planes, int64_t T, int mc, int ncp) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)ncp, (cuuint64_t)mc, (cuuint64_t)T};
    const cuuint64_t strides[2] = {(cuuint64_t)ncp * 2, (cuuint64_t)mc * ncp * 2};  // bytes, dims 1 and 2
    const cuuint32_t box[3] = {(cuuint32_t)kDirK, 1, (cuuint32_t)kDirM};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t direct_tiles_bytes(int mc, int ncp, int W) { return direct_rows_bytes(mc, ncp, W); }
size_t direct_smem(int W) { return direct_smem_bytes(W); }

cudaError_t launch_frame_planes(bool f32, const void* src, int64_t src_fstride, int64_t nimg, int m, int n, int levels,
                                int mc, int nc, const int32_t* coff_i, const float* coff_f, const float2* tw,
                                u64* rowE, u64* colE, u64* tot, uint32_t* corners, int wm1, void* p_hi, void* p_lo,
                                int ldp, cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    constexpr int N = 48;  // the FFT buffer is unused in this mode
    const size_t smem = sizeof(float2) * ((kRC / 2) * fft_ld<N>() + N) + sizeof(u64) * (kRC + nc);
    const void* fn = f32 ? (const void*)k_frame_rows<N, true, true> : (const void*)k_frame_rows<N, false, true>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(p_hi);
    __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(p_lo);
    if (f32)
        k_frame_rows<N, true, true><<<(unsigned)nimg, kRowsThreads, smem, st>>>(
            src, src_fstride, m, n, levels, mc, nc, coff_i, coff_f, tw, nullptr, 0, 0, rowE, colE, tot, corners, wm1,
            hi, lo, ldp);
    else
        k_frame_rows<N, false, true><<<(unsigned)nimg, kRowsThreads, smem, st>>>(
            src, src_fstride, m, n, levels, mc, nc, coff_i, coff_f, tw, nullptr, 0, 0, rowE, colE, tot, corners, wm1,
            hi, lo, ldp);
    return cudaGetLastError();
}

cudaError_t launch_toeplitz(bool f32, const void* tmpl, int m, int n, int levels, int mc, int nc, int ncp, int wm1,
                            const int32_t* coff_i, const float* coff_f, float* bprime, void* tiles,
                            cudaStream_t st) {
    if (f32)
        k_coarse_image<true><<<256, 256, 0, st>>>(tmpl, m, n, levels, mc, nc, coff_i, coff_f, bprime);
    else
        k_coarse_image<false><<<256, 256, 0, st>>>(tmpl, m, n, levels, mc, nc, coff_i, coff_f, bprime);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_toeplitz_rows<<<1024, 256, 0, st>>>(bprime, mc, nc, ncp, wm1, static_cast<__nv_bfloat16*>(tiles));
    return cudaGetLastError();
}

int direct_ksplit(int W, int64_t T, int mc, int nqc, int num_sms) {
    // Enough K splits for two CTAs per SM (one resident per SM), each split
    // keeping at least 16 K steps; at most kDirSplits.
    const int64_t tiles = (int64_t)((W + direct_ns(W) - 1) / direct_ns(W)) * ((T + kDirM - 1) / kDirM);
    int z = 1;
    while (z < kDirSplits && tiles * z < 2 * (int64_t)num_sms && (int64_t)mc * nqc / (2 * z) >= 16) z *= 2;
    return z;
}

cudaError_t launch_direct(const void* a_hi, const void* a_lo, int64_t T, int mc, int ncp, int nqc, int wm1,
                          const void* tiles, float* h, int ksplit, unsigned int* err, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    const int W = 2 * wm1 + 1;
    const size_t smem = direct_smem_bytes(W);
    cudaError_t e = ensure_smem((const void*)k_direct, smem);
    if (e != cudaSuccess) return e;
    const int ntiles = (W + direct_ns(W) - 1) / direct_ns(W);
    const int64_t mtiles = (T + kDirM - 1) / kDirM;
    CUtensorMap map_hi, map_lo;
    if ((e = plane_map(&map_hi, a_hi, T, mc, ncp)) != cudaSuccess) return e;
    if ((e = plane_map(&map_lo, a_lo, T, mc, ncp)) != cudaSuccess) return e;
    dim3 grid((unsigned)ntiles, (unsigned)mtiles, (unsigned)ksplit);
    k_direct<<<grid, kDirThreads, smem, st>>>(map_hi, map_lo, T, mc, ncp, nqc, wm1,
                                              static_cast<const __nv_bfloat16*>(tiles),
                                              h, err);
    return cudaGetLastError();
}

cudaError_t launch_combine_h(const float* h, int ksplit, int64_t nimg, int wm1, const float2* Sa2, const float2* Sb2,
                             const float* ia32, double* cost, int32_t* coarse, double* fbest, float* margin,
                             cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    const int64_t slab = nimg * (int64_t)(2 * wm1 + 1) * (2 * wm1 + 1);
    k_combine_h<<<(unsigned)nimg, 256, 0, st>>>(h, ksplit, slab, wm1, Sa2, Sb2, ia32, cost, coarse, fbest, margin);
    return cudaGetLastError();
}

}  // namespace moco
