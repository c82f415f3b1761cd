// Launchers of the differentiable form: soft-min and the adjoint of f.
#include <algorithm>

#include "grad.cuh"
#include "internal.h"

namespace moco {

cudaError_t launch_softmin(const double* cost, int64_t T, int K, double tau_scale, double* loss, float* weights,
                           cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    k_softmin<<<(unsigned)T, kSoftminThreads, 0, st>>>(cost, K, tau_scale, loss, weights);
    return cudaGetLastError();
}

static size_t grad_tmpl_smem(int wm1) {
    const int W = 2 * wm1 + 1, Wp = grad_wp(W);
    return sizeof(float) * ((size_t)(kGradTY + 2 * wm1) * (kGradTX + Wp) + (size_t)W * Wp);
}

size_t grad_smem_bytes(int wm1) {
    const int W = 2 * wm1 + 1, K = W * W, L = W + 1, H = kGradTile + 2 * wm1;
    const size_t tmpl = grad_tmpl_smem(wm1);
    const size_t frames = sizeof(float) * ((size_t)H * H + 2 * (size_t)K + (size_t)L * L);
    const size_t fin = sizeof(float) * (size_t)L * L;
    return std::max(tmpl, std::max(frames, fin));
}

cudaError_t launch_grad(const uint16_t* frames, int64_t T, int m, int n, int wm1, const float* G, float scale,
                        const double* inv_area, const int32_t* coff, const void* tmpl, int tmpl_f32, int corr,
                        float* acc, float* Q, float* grad_template, float* grad_frames, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    const int W = 2 * wm1 + 1, K = W * W, L = W + 1, H = kGradTile + 2 * wm1;
    cudaError_t e = cudaSuccess;
    if (corr && (e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)m * n, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Q, 0, sizeof(float) * (size_t)K, st)) != cudaSuccess) return e;
    k_grad_qsum<<<dim3((K + 255) / 256, (unsigned)((T + kQsumFrames - 1) / kQsumFrames)), 256, 0, st>>>(
        G, T, K, inv_area, scale, Q);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 tiles((n + kGradTile - 1) / kGradTile, (m + kGradTile - 1) / kGradTile);
    if (corr) {
        const size_t sm_t = grad_tmpl_smem(wm1);
        if ((e = ensure_smem((const void*)k_grad_tmpl, sm_t)) != cudaSuccess) return e;
        const dim3 g1((n + kGradTX - 1) / kGradTX, (m + kGradTY - 1) / kGradTY,
                      (unsigned)((T + kGradTmplFrames - 1) / kGradTmplFrames));
        k_grad_tmpl<<<g1, kGradThreads, sm_t, st>>>(frames, T, m, n, wm1, G, inv_area, scale, coff, acc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t sm_f = sizeof(float) * (size_t)L * L;
    if ((e = ensure_smem((const void*)k_grad_tmpl_finish, sm_f)) != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>(1024, ((int64_t)m * n + 255) / 256);
    k_grad_tmpl_finish<<<(unsigned)blocks, 256, sm_f, st>>>(acc, Q, m, n, wm1, tmpl, tmpl_f32, coff, grad_template);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (grad_frames) {
        const size_t sm_g = sizeof(float) * ((size_t)H * H + 2 * (size_t)K + (size_t)L * L);
        if ((e = ensure_smem((const void*)k_grad_frames, sm_g)) != cudaSuccess) return e;
        for (int64_t f0 = 0; f0 < T; f0 += 65535) {
            const int64_t cnt = std::min<int64_t>(65535, T - f0);
            const dim3 g2(tiles.x, tiles.y, (unsigned)cnt);
            k_grad_frames<<<g2, kGradThreads, sm_g, st>>>(frames + f0 * (int64_t)m * n, m, n, wm1, G + f0 * K,
                                                           inv_area, scale, tmpl, tmpl_f32, coff,
                                                           grad_frames + f0 * (int64_t)m * n);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace moco
