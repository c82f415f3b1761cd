// The C ABI of include/moco.h: plans, workspace, validation and the launch
// sequence of the translation search (Section 2 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "moco.h"
#include "plan.h"

namespace moco {

const char* const kKernelNames[K_COUNT] = {"k_frame_rows", "k_energy", "k_cols", "k_rows_inv", "k_jitter",
                                           "k_copy_shifts", "k_softmin", "k_backward", "k_direct", "k_apply",
                                           "k_jitter_level", "k_adj_rows", "k_adj_cols", "k_adj_inverse"};

thread_local std::string g_last_error;

moco_status fail(moco_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

moco_status cuda_fail(cudaError_t e, const char* what) {
    return fail(MOCO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

DeviceGuard::DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != prev_) cudaSetDevice(prev_);
}

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves one device allocation into 256-byte aligned pieces.
struct Carver {
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> items;
    template <typename T>
    void add(T** p, size_t bytes) {
        items.push_back({reinterpret_cast<void**>(p), off});
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
    }
    void bind(void* base) {
        for (auto& it : items) *it.first = static_cast<char*>(base) + it.second;
    }
};

// The four-step twiddles omega_N^(n2*k1) = exp(-2 pi i n2 k1 / N), each in
// FP64 and rounded once to FP32, in two orders: [k1*N2 + n2] for the forward
// transform, then [n2*N1 + k1] for the inverse (2N entries).
void host_roots(int N, std::vector<float2>& out) {
    int N1 = 0, N2 = 0;
    fft_split(N, &N1, &N2);
    out.resize(2 * (size_t)N);
    for (int k1 = 0; k1 < N1; ++k1)
        for (int n2 = 0; n2 < N2; ++n2) {
            const double a = 2.0 * M_PI * (double)(n2 * k1) / (double)N;
            const float2 z = make_float2((float)std::cos(a), (float)-std::sin(a));
            out[(size_t)k1 * N2 + n2] = z;
            out[(size_t)N + (size_t)n2 * N1 + k1] = z;
        }
}

}  // namespace

int64_t per_frame_scratch_bytes(const ShapePlan& sp) {
    const int64_t W = sp.W, wm1 = sp.wm1;
    int64_t b = 0;
    // The two forms' cross-term scratch is never live at once: one region.
    const int64_t fft = sp.has_fft ? (int64_t)sp.ncv * sp.ldx * 8 + W * sp.ncv * 8 : 0;  // X, Y
    const int64_t dir = sp.has_direct ? (int64_t)sp.mc * sp.ncp * 4 + W * W * 4 * kDirSplits : 0;  // planes, h slabs
    b += std::max(fft, dir);
    b += ((int64_t)sp.mc + sp.nc + 1) * 8;     // rowE, colE, tot
    b += 4 * wm1 * wm1 * 4;                    // corners
    b += W * W * 8;                            // Sa
    b += 8 + 8 + 4;                            // coarse, fbest, margin
    if (sp.levels > 1) b += 8;                 // the refinement's second shift buffer
    b += 9 * 8 + 4;                            // jitter sums and tickets
    return b;
}

moco_status resolve_shape(const moco_shape& d, ShapePlan& sp) {
    if (d.reserved != 0) return fail(MOCO_ERR_INVALID_ARG, "moco_shape.reserved must be 0");
    if (d.m < 1 || d.n < 8 || d.n % 8 != 0 || d.m > 4096 || d.n > 4096)
        return fail(MOCO_ERR_INVALID_ARG, "need 1 <= m <= 4096, 8 <= n <= 4096 and n % 8 == 0");
    if (d.levels < -1 || d.levels > 4) return fail(MOCO_ERR_INVALID_ARG, "levels must be -1 or 0 .. 4");
    if (d.template_dtype != MOCO_TEMPLATE_U16 && d.template_dtype != MOCO_TEMPLATE_F32)
        return fail(MOCO_ERR_INVALID_ARG, "bad template_dtype");
    if (d.xcorr < MOCO_XCORR_AUTO || d.xcorr > MOCO_XCORR_DIRECT_BF16X3)
        return fail(MOCO_ERR_INVALID_ARG, "bad xcorr");
    if (d.group_frames < 0) return fail(MOCO_ERR_INVALID_ARG, "group_frames must be >= 0");
    sp.desc = d;
    sp.levels = d.levels < 0 ? ((d.m > 256 || d.n > 256) ? 1 : 0) : d.levels;
    sp.f32 = d.template_dtype == MOCO_TEMPLATE_F32;
    if (sp.f32 && sp.levels != 0)
        return fail(MOCO_ERR_UNSUPPORTED, "a float template needs levels == 0");
    sp.mc = d.m >> sp.levels;
    sp.nc = d.n >> sp.levels;
    if (sp.mc < 1 || sp.nc < 1) return fail(MOCO_ERR_INVALID_ARG, "image too small for its levels");
    sp.w = d.w;
    if (d.w < 1 || 2 * d.w - 1 > sp.mc || 2 * d.w - 1 > sp.nc)
        return fail(MOCO_ERR_INVALID_ARG, "need w >= 1 and 2w-1 <= min(mc, nc)");
    sp.wm1 = d.w - 1;
    sp.W = 2 * d.w - 1;
    sp.Nr = fft_size_for(sp.mc + d.w - 1);
    sp.Nc = fft_size_for(sp.nc + d.w - 1);
    // (k_rows_inv keeps h, W x W floats, next to a transform buffer)
    // (and its energy sweep holds at most four columns per lane: w <= 128)
    const bool fft_ok = sp.Nr && sp.Nc && rows_inv_smem_bytes(sp.Nc, sp.wm1) <= 227 * 1024 && d.w <= 128;
    // (the direct form reads 2x2 sums: at most one level)
    const bool direct_ok = direct_smem(sp.W) <= 227 * 1024 && sp.W <= 256 && sp.levels <= 1;
    sp.nqc = (sp.nc + 63) / 64;
    sp.ncp = sp.nqc * 64;
    if (d.xcorr == MOCO_XCORR_FFT_FP32 && !fft_ok)
        return fail(MOCO_ERR_UNSUPPORTED,
                    "searched grid + window exceeds the largest FFT length (576), or the window its shared memory");
    if (d.xcorr == MOCO_XCORR_DIRECT_BF16X3 && !direct_ok)
        return fail(MOCO_ERR_UNSUPPORTED, "window too large for the direct form");
    if (!fft_ok && !direct_ok) return fail(MOCO_ERR_UNSUPPORTED, "no cross-term form supports this shape");
    sp.has_fft = fft_ok && d.xcorr != MOCO_XCORR_DIRECT_BF16X3;
    sp.has_direct = direct_ok && d.xcorr != MOCO_XCORR_FFT_FP32;
    sp.form = sp.has_fft ? MOCO_XCORR_FFT_FP32 : MOCO_XCORR_DIRECT_BF16X3;
    if (!sp.Nr) sp.Nr = 48;  // placeholders: no FFT buffers are used
    if (!sp.Nc) sp.Nc = 48;
    sp.ncv = sp.Nc / 2 + 1;
    sp.ldx = sp.mc + (sp.mc & 1);
    sp.unit = 1.0;
    for (int l = 0; l < sp.levels; ++l) sp.unit /= 16.0;  // costs per full-resolution pixel
    if (d.group_frames > 0) {
        sp.group = d.group_frames;
    } else {
        // Large batches keep every per-frame kernel several waves deep on the
        // 152 SMs; about 1 GiB of workspace.
        const int64_t target = 1ll << 30;
        sp.group = (int)std::max<int64_t>(1, std::min<int64_t>(2048, target / per_frame_scratch_bytes(sp)));
    }
    // Host staging chunks of ~64 MiB: the copy engine (the bound of the
    // host path) keeps streaming while each chunk is searched, and the last
    // chunk's search after the final copy stays short.
    const int64_t frame_bytes = (int64_t)d.m * d.n * 2;
    sp.stage_frames = (int)std::max<int64_t>(16, std::min<int64_t>(sp.group, (64ll << 20) / frame_bytes));
    // (after every argument check: invalid shapes are rejected without a CUDA call)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sp.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MOCO_ERR_CUDA, "device query");
    }
    return MOCO_OK;
}

// Per-shape data that lives as long as the plan (template-derived tables).
moco_status allocate_shape(ShapePlan& sp) {
    const int64_t W = sp.W, m = sp.desc.m, n = sp.desc.n;
    Carver c;
    c.add(&sp.tmpl, (size_t)m * n * (sp.f32 ? 4 : 2));
    c.add(&sp.coff_i, 4);
    c.add(&sp.coff_f, 4);
    c.add(&sp.twr, (size_t)sp.Nr * 16);
    c.add(&sp.twc, (size_t)sp.Nc * 16);
    c.add(&sp.bspec, sp.has_fft ? (size_t)sp.ncv * sp.Nr * 8 : 0);
    c.add(&sp.dev_err, 4);
    if (sp.has_direct) {
        c.add(&sp.bprime, (size_t)sp.mc * sp.nc * 4);
        c.add(&sp.dtiles, direct_tiles_bytes(sp.mc, sp.ncp, sp.W));
    }
    c.add(&sp.Sb, (size_t)W * W * 8);
    c.add(&sp.inv_area, (size_t)W * W * 8);
    c.add(&sp.Sb2, (size_t)W * W * 8);
    c.add(&sp.ia32, (size_t)W * W * 4);
    c.add(&sp.grad_acc, (size_t)(m * n * 4));
    c.add(&sp.grad_Q, (size_t)(W * W * 4));
    c.add(&sp.grad_spec, sp.has_fft ? (size_t)sp.ncv * sp.Nr * 8 : 0);
    if (sp.levels && !sp.f32) c.add(&sp.bsq, (size_t)(m + 1) * (n + 1) * 8);
    for (int l = 1; l < sp.levels; ++l) c.add(&sp.tlev[l], level_image_elems((int)m, (int)n, l) * 4);
    c.add(&sp.apply_sum, (size_t)m * n * 8);
    c.add(&sp.apply_cnt, (size_t)m * n * 4);
    sp.x_fstride = (int64_t)sp.ncv * sp.ldx;
    sp.y_fstride = W * sp.ncv;
    sp.bytes = c.off;
    cudaError_t e = cudaMalloc(&sp.base, sp.bytes);
    if (e != cudaSuccess) {
        sp.base = nullptr;
        cudaGetLastError();
        return fail(MOCO_ERR_OOM, "cudaMalloc of " + std::to_string(sp.bytes) + " bytes failed");
    }
    c.bind(sp.base);
    e = cudaMemset(sp.dev_err, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    // Host-computed constant tables.
    std::vector<float2> tw;
    host_roots(sp.Nr, tw);
    e = cudaMemcpy(sp.twr, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload of row roots");
    host_roots(sp.Nc, tw);
    e = cudaMemcpy(sp.twc, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload of column roots");
    std::vector<double> ia((size_t)W * W);
    for (int s = -sp.wm1; s <= sp.wm1; ++s)
        for (int t = -sp.wm1; t <= sp.wm1; ++t)
            ia[(size_t)(s + sp.wm1) * W + (t + sp.wm1)] =
                1.0 / ((double)(sp.mc - std::abs(s)) * (double)(sp.nc - std::abs(t)));
    e = cudaMemcpy(sp.inv_area, ia.data(), ia.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload of 1/Area");
    std::vector<float> ia32(ia.size());
    for (size_t k = 0; k < ia.size(); ++k) ia32[k] = (float)(ia[k] * sp.unit);
    e = cudaMemcpy(sp.ia32, ia32.data(), ia32.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload of unit/Area");
    return MOCO_OK;
}

// Per-batch scratch of one shape, carved from `base` (or only sized when
// base is null). Shapes run one after another on the plan's stream, so all
// shapes of a plan share one scratch region sized for the largest.
size_t bind_scratch(ShapePlan& sp, void* base) {
    const int64_t G = sp.group, W = sp.W, m = sp.desc.m, n = sp.desc.n;
    Carver c;
    // Cross-term scratch: the FFT form's X, Y and the direct form's planes, h
    // share one region (a shape runs one form at a time).
    const size_t fft_x = sp.has_fft ? (size_t)(G * sp.x_fstride * 8) : 0;
    const size_t fft_y = sp.has_fft ? (size_t)(G * sp.y_fstride * 8) : 0;
    const size_t dir_p = sp.has_direct ? (size_t)(G * sp.mc * sp.ncp * 2) : 0;
    const size_t dir_h = sp.has_direct ? (size_t)(G * W * W * 4 * kDirSplits) : 0;  // one h slab per K split
    const size_t fft_total = align_up(fft_x, 256) + fft_y;
    const size_t dir_total = 2 * align_up(dir_p, 256) + dir_h;
    void* xregion = nullptr;
    c.add(&xregion, std::max(fft_total, dir_total));
    c.add(&sp.rowE, (size_t)(G * sp.mc * 8));
    c.add(&sp.colE, (size_t)(G * sp.nc * 8));
    c.add(&sp.tot, (size_t)(G * 8));
    c.add(&sp.corners, (size_t)(G * 4 * sp.wm1 * sp.wm1 * 4));
    c.add(&sp.Sa, (size_t)(G * W * W * 8));
    c.add(&sp.coarse, (size_t)(G * 2 * 4));
    if (sp.levels > 1) c.add(&sp.coarse2, (size_t)(G * 2 * 4));
    c.add(&sp.fbest, (size_t)(G * 8));
    c.add(&sp.margin, (size_t)(G * 4));
    c.add(&sp.jit_acc, (size_t)(G * 9 * 8));
    c.add(&sp.jit_ticket, (size_t)(G * 4));
    for (int k = 0; k < 2; ++k) {
        c.add(&sp.stage[k], (size_t)((int64_t)sp.stage_frames * m * n * 2));
        c.add(&sp.stage_shifts[k], (size_t)(sp.stage_frames * 2 * 4));
    }
    if (!base) return c.off;
    c.bind(base);
    char* x = static_cast<char*>(xregion);
    if (sp.has_fft) {
        sp.X = reinterpret_cast<float2*>(x);
        sp.Y = reinterpret_cast<float2*>(x + align_up(fft_x, 256));
    }
    if (sp.has_direct) {
        sp.planes_hi = x;
        sp.planes_lo = x + align_up(dir_p, 256);
        sp.hbuf = reinterpret_cast<float*>(x + 2 * align_up(dir_p, 256));
    }
    return c.off;
}

// Offset, energies and spectrum of the template (run whenever it changes).
moco_status prepare_template(ShapePlan& sp, const void* tmpl_dev, cudaStream_t st) {
    const size_t bytes = (size_t)sp.desc.m * sp.desc.n * (sp.f32 ? 4 : 2);
    cudaError_t e = cudaMemcpyAsync(sp.tmpl, tmpl_dev, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "template copy");
    // (the per-frame totals' scratch, free here, holds the slice sums)
    e = launch_template_offset(sp.f32, sp.tmpl, sp.desc.m, sp.desc.n, sp.levels, sp.coff_i, sp.coff_f, sp.tot,
                               sp.group, st);
    if (e != cudaSuccess) return cuda_fail(e, "template offset");
    if (sp.has_fft)
        e = launch_frame_rows(sp.Nc, sp.f32, sp.tmpl, 0, 1, sp.desc.m, sp.desc.n, sp.levels, sp.mc, sp.nc,
                              sp.coff_i, sp.coff_f, sp.twc, sp.X, sp.x_fstride, sp.ldx, sp.rowE, sp.colE, sp.tot,
                              sp.corners, sp.wm1, sp.dev_err, sp.group, st);
    else
        e = launch_frame_planes(sp.f32, sp.tmpl, 0, 1, sp.desc.m, sp.desc.n, sp.levels, sp.mc, sp.nc, sp.coff_i,
                                sp.coff_f, sp.twc, sp.rowE, sp.colE, sp.tot, sp.corners, sp.wm1, sp.planes_hi,
                                sp.planes_lo, sp.ncp, st);
    if (e != cudaSuccess) return cuda_fail(e, "template rows");
    e = launch_energy(sp.f32, true, sp.rowE, sp.colE, sp.tot, sp.corners, 1, sp.mc, sp.nc, sp.wm1, sp.Sb, 1, st);
    if (e == cudaSuccess) e = launch_pair_from_double(sp.Sb, sp.Sb2, (int64_t)sp.W * sp.W, st);
    if (e != cudaSuccess) return cuda_fail(e, "template energies");
    // Before the autotuner has fixed the form both forms' tables are built;
    // afterwards only the chosen form's.
    if (sp.has_fft && (!sp.tuned || sp.form == MOCO_XCORR_FFT_FP32)) {
        e = launch_cols(sp.Nr, true, sp.X, sp.x_fstride, sp.ldx, sp.mc, sp.ncv, 1, sp.twr, nullptr, sp.bspec, 0,
                        sp.wm1, (float)(1.0 / ((double)sp.Nr * (double)sp.Nc)), sp.dev_err, st);
        if (e != cudaSuccess) return cuda_fail(e, "template spectrum");
    }
    if (sp.has_direct && (!sp.tuned || sp.form == MOCO_XCORR_DIRECT_BF16X3)) {
        e = launch_toeplitz(sp.f32, sp.tmpl, sp.desc.m, sp.desc.n, sp.levels, sp.mc, sp.nc, sp.ncp, sp.wm1, sp.coff_i,
                            sp.coff_f, sp.bprime, sp.dtiles, st);
        if (e != cudaSuccess) return cuda_fail(e, "template Toeplitz tiles");
    }
    if (sp.bsq) {
        e = launch_sq_prefix(static_cast<const uint16_t*>(sp.tmpl), sp.desc.m, sp.desc.n, sp.bsq, st);
        if (e != cudaSuccess) return cuda_fail(e, "template square prefix table");
    }
    for (int l = 1; l < sp.levels; ++l) {
        e = launch_box_level(static_cast<const uint16_t*>(sp.tmpl), sp.desc.m, sp.desc.n, l, sp.tlev[l], st);
        if (e != cudaSuccess) return cuda_fail(e, "template level image");
    }
    return MOCO_OK;
}

// The searched-grid pass over frames [f0, f0+g) staged at `frames`:
// energies, cross term, combine, argmin -> coarse_out, or sp.coarse when
// null (and optional outputs).
moco_status search_group(ShapePlan& sp, const uint16_t* frames, int64_t g, double* cost, double* fbest,
                         float* margin, cudaStream_t st, int32_t* coarse_out = nullptr) {
    const int m = sp.desc.m, n = sp.desc.n;
    int32_t* coarse = coarse_out ? coarse_out : sp.coarse;
    Profiler& P = *sp.prof;
    if (sp.form == MOCO_XCORR_DIRECT_BF16X3) {
        P.begin(K_FRAME_ROWS, st);
        cudaError_t e = launch_frame_planes(false, frames, (int64_t)m * n, g, m, n, sp.levels, sp.mc, sp.nc, sp.coff_i,
                                            nullptr, sp.twc, sp.rowE, sp.colE, sp.tot, sp.corners, sp.wm1,
                                            sp.planes_hi, sp.planes_lo, sp.ncp, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_frame_rows (planes)");
        P.begin(K_ENERGY, st);
        e = launch_energy(false, false, sp.rowE, sp.colE, sp.tot, sp.corners, g, sp.mc, sp.nc, sp.wm1, sp.Sa, 0, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_energy");
        P.begin(K_DIRECT, st);
        const int ksplit = direct_ksplit(sp.W, g, sp.mc, sp.nqc, sp.num_sms);
        e = launch_direct(sp.planes_hi, sp.planes_lo, g, sp.mc, sp.ncp, sp.nqc, sp.wm1, sp.dtiles, sp.hbuf, ksplit, sp.dev_err,
                          st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_direct");
        P.begin(K_ROWS_INV, st);
        e = launch_combine_h(sp.hbuf, ksplit, g, sp.wm1, reinterpret_cast<const float2*>(sp.Sa), sp.Sb2, sp.ia32, cost, coarse,
                             fbest ? fbest : sp.fbest, margin ? margin : sp.margin, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_combine_h");
        return MOCO_OK;
    }
    P.begin(K_FRAME_ROWS, st);
    cudaError_t e = launch_frame_rows(sp.Nc, false, frames, (int64_t)m * n, g, m, n, sp.levels, sp.mc, sp.nc,
                                      sp.coff_i, nullptr, sp.twc, sp.X, sp.x_fstride, sp.ldx, sp.rowE, sp.colE,
                                      sp.tot, sp.corners, sp.wm1, sp.dev_err, sp.group, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "k_frame_rows");
    P.begin(K_COLS, st);
    e = launch_cols(sp.Nr, false, sp.X, sp.x_fstride, sp.ldx, sp.mc, sp.ncv, g, sp.twr, sp.bspec, sp.Y,
                    sp.y_fstride, sp.wm1, 0.f, sp.dev_err, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "k_cols");
    P.begin(K_ROWS_INV, st);
    e = launch_rows_inv(sp.Nc, sp.Y, sp.y_fstride, sp.ncv, sp.wm1, g, sp.twc, sp.rowE, sp.colE, sp.tot, sp.corners,
                        sp.mc, sp.nc, sp.Sb2, sp.ia32, cost, coarse, fbest ? fbest : sp.fbest,
                        margin ? margin : sp.margin, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "k_rows_inv");
    return MOCO_OK;
}

moco_status autotune(ShapePlan& sp, cudaStream_t st);

moco_status align_frames(ShapePlan& sp, const uint16_t* frames, int64_t T, int32_t* shifts, double* best_cost,
                         float* margin, double* final_cost, cudaStream_t st) {
    const int64_t mn = (int64_t)sp.desc.m * sp.desc.n;
    for (int64_t f0 = 0; f0 < T; f0 += sp.group) {
        const int64_t g = std::min<int64_t>(sp.group, T - f0);
        moco_status s = search_group(sp, frames + f0 * mn, g, nullptr, best_cost ? best_cost + f0 : nullptr,
                                     margin ? margin + f0 : nullptr, st);
        if (s != MOCO_OK) return s;
        cudaError_t e;
        // Levels L-1 .. 1: the 3x3 refinement on each level's box sums; the
        // shifts alternate between the two buffers.
        const int32_t* cin = sp.coarse;
        for (int l = sp.levels - 1; l >= 1; --l) {
            int32_t* cout = (cin == sp.coarse) ? sp.coarse2 : sp.coarse;
            sp.prof->begin(K_JITTER_LEVEL, st);
            e = launch_jitter_level(frames + f0 * mn, mn, g, sp.desc.m, sp.desc.n, l, sp.tlev[l], cin, cout,
                                    sp.jit_acc, sp.jit_ticket, st);
            sp.prof->end(st);
            if (e != cudaSuccess) return cuda_fail(e, "k_jitter_level");
            cin = cout;
        }
        sp.prof->begin(sp.levels ? K_JITTER : K_COPY_SHIFTS, st);
        if (sp.levels && sp.bsq) {
            JitSegment seg;
            seg.frames = frames + f0 * mn;
            seg.fstride = mn;
            seg.T = g;
            seg.tmpl = static_cast<const uint16_t*>(sp.tmpl);
            seg.bsq = sp.bsq;
            seg.coarse = cin;
            seg.shifts = shifts + 2 * f0;
            seg.ffinal = final_cost ? final_cost + f0 : nullptr;
            seg.m = sp.desc.m;
            seg.n = sp.desc.n;
            e = launch_jitter_multi(&seg, 1, sp.jit_acc, sp.jit_ticket, g, sp.num_sms, st);
        } else if (sp.levels)
            e = launch_jitter(frames + f0 * mn, mn, g, static_cast<const uint16_t*>(sp.tmpl), sp.desc.m,
                              sp.desc.n, sp.bsq, cin, shifts + 2 * f0, final_cost ? final_cost + f0 : nullptr,
                              sp.jit_acc, sp.jit_ticket, st);
        else
            e = launch_copy_shifts(sp.coarse, shifts + 2 * f0, best_cost ? best_cost + f0 : sp.fbest,
                                   final_cost ? final_cost + f0 : nullptr, g, st);
        sp.prof->end(st);
        if (e != cudaSuccess) return cuda_fail(e, sp.levels ? "k_jitter" : "k_copy_shifts");
    }
    return MOCO_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// MOCO_XCORR_AUTO: time both forms on one batch of zero frames (the work
// does not depend on the values) and keep the faster. The batch is as long
// as the plan's internal batch, up to 512 MiB of frames (a short one would
// time both forms far from their steady state: too few frame tiles for the
// direct form, too few frames per column CTA for the FFT form), in a
// buffer freed before returning; if that allocation fails, the host staging
// buffer's frames.
moco_status autotune(ShapePlan& sp, cudaStream_t st) {
    if (!(sp.has_fft && sp.has_direct)) {
        sp.tuned = true;
        return MOCO_OK;
    }
    const int64_t fbytes = (int64_t)sp.desc.m * sp.desc.n * 2;
    int64_t g = std::min<int64_t>(sp.group, std::max<int64_t>(sp.stage_frames, (512ll << 20) / fbytes));
    void* tune = nullptr;
    if (cudaMalloc(&tune, (size_t)(g * fbytes)) != cudaSuccess) {
        cudaGetLastError();
        tune = nullptr;
        g = std::min<int64_t>(sp.stage_frames, sp.group);
    }
    const uint16_t* frames = tune ? static_cast<const uint16_t*>(tune) : sp.stage[0];
    cudaError_t e = cudaMemsetAsync(const_cast<uint16_t*>(frames), 0, (size_t)(g * fbytes), st);
    if (e != cudaSuccess) {
        if (tune) cudaFree(tune);
        return cuda_fail(e, "autotune clear");
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    Profiler off;
    Profiler* keep = sp.prof;
    sp.prof = &off;
    moco_status r = MOCO_OK;
    float best = 0.f;
    int best_form = MOCO_XCORR_FFT_FP32;
    for (int form : {MOCO_XCORR_FFT_FP32, MOCO_XCORR_DIRECT_BF16X3}) {
        if (form == MOCO_XCORR_DIRECT_BF16X3) {
            // Skip timing the direct form when even the tensor cores' nominal
            // dense BF16 rate (2.25 PFLOP/s) could not beat the FFT form: its
            // three products of the (2w-1)^2-shift contraction alone take longer.
            const double flops = 3.0 * 2.0 * (double)sp.W * sp.W * sp.mc * sp.nc * (double)g;
            if (flops / 2.25e15 * 1e3 >= (double)sp.tuned_ms[MOCO_XCORR_FFT_FP32]) break;
        }
        sp.form = form;
        r = search_group(sp, frames, g, nullptr, nullptr, nullptr, st);  // warm-up
        if (r != MOCO_OK) break;
        cudaEventRecord(a, st);
        for (int it = 0; it < 3 && r == MOCO_OK; ++it) r = search_group(sp, frames, g, nullptr, nullptr, nullptr, st);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) { r = cuda_fail(e, "autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        sp.tuned_ms[form] = ms / 3.f;
        if (form == MOCO_XCORR_FFT_FP32 || ms < best) { best = ms; best_form = form; }
    }
    sp.prof = keep;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (tune) {
        cudaStreamSynchronize(st);
        cudaFree(tune);
    }
    sp.form = best_form;
    sp.tuned = true;
    return r;
}

}  // namespace moco

using namespace moco;

extern "C" {

const char* moco_status_string(moco_status s) {
    switch (s) {
        case MOCO_OK: return "MOCO_OK";
        case MOCO_ERR_INVALID_ARG: return "MOCO_ERR_INVALID_ARG";
        case MOCO_ERR_UNSUPPORTED: return "MOCO_ERR_UNSUPPORTED";
        case MOCO_ERR_OOM: return "MOCO_ERR_OOM";
        case MOCO_ERR_CUDA: return "MOCO_ERR_CUDA";
        case MOCO_ERR_TIMEOUT: return "MOCO_ERR_TIMEOUT";
    }
    return "MOCO_ERR_UNKNOWN";
}

const char* moco_last_error(void) { return g_last_error.c_str(); }

moco_status moco_plan_destroy(moco_plan_t plan) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    DeviceGuard guard(plan->device);
    cudaDeviceSynchronize();
    for (auto& sp : plan->shapes)
        if (sp.base) cudaFree(sp.base);
    if (plan->scratch) cudaFree(plan->scratch);
    if (plan->mj_base) cudaFree(plan->mj_base);
    if (plan->aux) cudaStreamDestroy(plan->aux);
    for (auto& ev : plan->prof.pool) cudaEventDestroy(ev);
    for (auto& ev : plan->ev)
        if (ev) cudaEventDestroy(ev);
    delete plan;
    return MOCO_OK;
}

moco_status moco_plan(const moco_shape* shapes, int32_t nshapes, const void* const* templates_dev, void* stream,
                      moco_plan_t* out) {
    g_last_error.clear();
    if (!out) return fail(MOCO_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!shapes || nshapes < 1 || !templates_dev) return fail(MOCO_ERR_INVALID_ARG, "need shapes and templates");
    for (int k = 0; k < nshapes; ++k)
        if (!templates_dev[k]) return fail(MOCO_ERR_INVALID_ARG, "null template pointer");
    moco_plan_t plan = new moco_plan_s();
    cudaGetDevice(&plan->device);
    plan->shapes.resize(nshapes);
    for (auto& sp : plan->shapes) sp.prof = &plan->prof;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    moco_status s = MOCO_OK;
    for (int k = 0; k < nshapes && s == MOCO_OK; ++k) s = resolve_shape(shapes[k], plan->shapes[k]);
    for (int k = 0; k < nshapes && s == MOCO_OK; ++k) s = allocate_shape(plan->shapes[k]);
    if (s == MOCO_OK) {
        size_t need = 0;
        for (auto& sp : plan->shapes) need = std::max(need, bind_scratch(sp, nullptr));
        cudaError_t e = cudaMalloc(&plan->scratch, need);
        if (e != cudaSuccess) {
            plan->scratch = nullptr;
            cudaGetLastError();
            s = fail(MOCO_ERR_OOM, "cudaMalloc of " + std::to_string(need) + " bytes of batch scratch failed");
        } else {
            plan->scratch_bytes = need;
            for (auto& sp : plan->shapes) bind_scratch(sp, plan->scratch);
        }
    }
    for (int k = 0; k < nshapes && s == MOCO_OK; ++k) s = prepare_template(plan->shapes[k], templates_dev[k], st);
    for (int k = 0; k < nshapes && s == MOCO_OK; ++k) s = autotune(plan->shapes[k], st);
    if (s == MOCO_OK) {
        // Scratch of the several-stack refinement (nine sums and a ticket per
        // frame of one launch) and the SM count its persistent launch fills.
        const size_t mj = align_up(sizeof(u64) * 9 * kMultiJitFrames, 256) +
                          align_up(sizeof(unsigned int) * kMultiJitFrames, 256);
        cudaError_t e = cudaMalloc(&plan->mj_base, mj);
        if (e != cudaSuccess) {
            plan->mj_base = nullptr;
            cudaGetLastError();
            s = fail(MOCO_ERR_OOM, "cudaMalloc of the refinement scratch failed");
        } else {
            char* b = static_cast<char*>(plan->mj_base);
            plan->mj_acc = reinterpret_cast<u64*>(b);
            plan->mj_ticket = reinterpret_cast<unsigned int*>(b + align_up(sizeof(u64) * 9 * kMultiJitFrames, 256));
            e = cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device);
            if (e != cudaSuccess) s = cuda_fail(e, "device query");
        }
    }
    if (s == MOCO_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&plan->aux, cudaStreamNonBlocking);
        for (auto& ev : plan->ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "plan set-up");
    }
    if (s != MOCO_OK) {
        std::string msg = g_last_error;
        moco_plan_destroy(plan);
        g_last_error = msg;
        return s;
    }
    *out = plan;
    return MOCO_OK;
}

moco_status moco_set_template(moco_plan_t plan, int32_t shape_idx, const void* template_dev, void* stream) {
    if (!plan || !template_dev) return fail(MOCO_ERR_INVALID_ARG, "null plan or template");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    DeviceGuard guard(plan->device);
    return prepare_template(plan->shapes[shape_idx], template_dev, static_cast<cudaStream_t>(stream));
}

moco_status moco_plan_query(moco_plan_t plan, int32_t shape_idx, moco_shape_info* info) {
    if (!plan || !info) return fail(MOCO_ERR_INVALID_ARG, "null plan or info");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    const ShapePlan& sp = plan->shapes[shape_idx];
    DeviceGuard guard(plan->device);
    int32_t off = 0;
    cudaError_t e = cudaMemcpy(&off, sp.coff_i, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "offset read-back");
    info->levels = sp.levels;
    info->mc = sp.mc;
    info->nc = sp.nc;
    info->fft_rows = sp.Nr;
    info->fft_cols = sp.Nc;
    info->xcorr = sp.form;
    info->group_frames = sp.group;
    info->offset = off;
    info->workspace_bytes = (int64_t)(sp.bytes + plan->scratch_bytes);
    return MOCO_OK;
}

moco_status moco_align_stack(moco_plan_t plan, const moco_stack* stacks, int32_t nstacks, void* stream) {
    if (!plan || (nstacks > 0 && !stacks) || nstacks < 0) return fail(MOCO_ERR_INVALID_ARG, "null plan or stacks");
    for (int k = 0; k < nstacks; ++k) {
        const moco_stack& s = stacks[k];
        if (s.shape_idx < 0 || s.shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
        if (s.reserved != 0 || s.T < 0) return fail(MOCO_ERR_INVALID_ARG, "bad stack");
        if (s.T > 0 && (!s.frames_dev || !s.shifts_dev)) return fail(MOCO_ERR_INVALID_ARG, "null frames or shifts");
        if (s.T > 0 && !aligned16(s.frames_dev)) return fail(MOCO_ERR_INVALID_ARG, "frames must be 16-byte aligned");
        if (plan->shapes[s.shape_idx].f32 && s.T > 0 && plan->shapes[s.shape_idx].levels)
            return fail(MOCO_ERR_UNSUPPORTED, "float template with levels");
    }
    DeviceGuard guard(plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Stacks searched on one 2x2 level and refined at full resolution (the
    // paper's rule above 256x256): with two or more of them, every stack's
    // search runs first, writing its searched-grid optima into the caller's
    // shift buffer, then one refinement launch runs a grid over the (stack,
    // frame, warp item) work items of all of them.
    auto deferred = [&](const moco_stack& s) {
        const ShapePlan& sp = plan->shapes[s.shape_idx];
        return s.T > 0 && sp.levels == 1 && sp.bsq != nullptr;
    };
    int ndef = 0;
    for (int k = 0; k < nstacks; ++k) ndef += deferred(stacks[k]) ? 1 : 0;
    std::vector<JitSegment> segs;
    for (int k = 0; k < nstacks; ++k) {
        const moco_stack& s = stacks[k];
        if (s.T == 0) continue;
        ShapePlan& sp = plan->shapes[s.shape_idx];
        if (ndef < 2 || !deferred(s)) {
            moco_status r = align_frames(sp, s.frames_dev, s.T, s.shifts_dev, s.best_cost_dev, s.margin_dev,
                                         s.final_cost_dev, st);
            if (r != MOCO_OK) return r;
            continue;
        }
        const int64_t mn = (int64_t)sp.desc.m * sp.desc.n;
        for (int64_t f0 = 0; f0 < s.T; f0 += sp.group) {
            const int64_t g = std::min<int64_t>(sp.group, s.T - f0);
            moco_status r = search_group(sp, s.frames_dev + f0 * mn, g, nullptr,
                                         s.best_cost_dev ? s.best_cost_dev + f0 : nullptr,
                                         s.margin_dev ? s.margin_dev + f0 : nullptr, st, s.shifts_dev + 2 * f0);
            if (r != MOCO_OK) return r;
        }
        for (int64_t f0 = 0; f0 < s.T; f0 += kMultiJitFrames) {
            JitSegment g;
            g.frames = s.frames_dev + f0 * mn;
            g.fstride = mn;
            g.T = std::min<int64_t>(kMultiJitFrames, s.T - f0);
            g.tmpl = static_cast<const uint16_t*>(sp.tmpl);
            g.bsq = sp.bsq;
            g.coarse = s.shifts_dev + 2 * f0;  // read before each frame's result overwrites it
            g.shifts = s.shifts_dev + 2 * f0;
            g.ffinal = s.final_cost_dev ? s.final_cost_dev + f0 : nullptr;
            g.m = sp.desc.m;
            g.n = sp.desc.n;
            segs.push_back(g);
        }
    }
    if (!segs.empty()) {
        plan->prof.begin(K_JITTER, st);
        cudaError_t e = launch_jitter_multi(segs.data(), (int)segs.size(), plan->mj_acc, plan->mj_ticket,
                                            kMultiJitFrames, plan->num_sms, st);
        plan->prof.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_jitter_multi");
    }
    return MOCO_OK;
}

moco_status moco_apply_shifts(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              const int32_t* shifts_dev, uint16_t fill, uint16_t* corrected_dev, double* mean_dev,
                              void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0) return fail(MOCO_ERR_INVALID_ARG, "T < 0");
    ShapePlan& sp = plan->shapes[shape_idx];
    const int m = sp.desc.m, n = sp.desc.n;
    if (n % 8 != 0) return fail(MOCO_ERR_UNSUPPORTED, "moco_apply_shifts needs n % 8 == 0");
    if (T == 0 && mean_dev == nullptr) return MOCO_OK;
    if (T > 0 && (!frames_dev || !shifts_dev)) return fail(MOCO_ERR_INVALID_ARG, "null frames or shifts");
    if (T > 0 && !aligned16(frames_dev)) return fail(MOCO_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    if (corrected_dev && !aligned16(corrected_dev))
        return fail(MOCO_ERR_INVALID_ARG, "corrected frames must be 16-byte aligned");
    DeviceGuard guard(plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    sp.prof->begin(K_APPLY, st);
    e = launch_apply(frames_dev, (int64_t)m * n, T, m, n, shifts_dev, fill, corrected_dev, mean_dev, sp.apply_sum,
                     sp.apply_cnt, sms, st);
    sp.prof->end(st);
    if (e != cudaSuccess) return cuda_fail(e, "k_apply");
    return MOCO_OK;
}

moco_status moco_cost_surface(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              double* cost_dev, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0) return fail(MOCO_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return MOCO_OK;
    if (!frames_dev || !cost_dev) return fail(MOCO_ERR_INVALID_ARG, "null frames or cost");
    if (!aligned16(frames_dev)) return fail(MOCO_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    DeviceGuard guard(plan->device);
    ShapePlan& sp = plan->shapes[shape_idx];
    const int64_t mn = (int64_t)sp.desc.m * sp.desc.n, WW = (int64_t)sp.W * sp.W;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t f0 = 0; f0 < T; f0 += sp.group) {
        const int64_t g = std::min<int64_t>(sp.group, T - f0);
        moco_status s = search_group(sp, frames_dev + f0 * mn, g, cost_dev + f0 * WW, nullptr, nullptr, st);
        if (s != MOCO_OK) return s;
    }
    return MOCO_OK;
}

moco_status moco_softmin(moco_plan_t plan, int32_t shape_idx, const double* cost_dev, int64_t T, double tau_scale,
                         double* loss_dev, float* weights_dev, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0 || !(tau_scale >= 0.0)) return fail(MOCO_ERR_INVALID_ARG, "T < 0 or bad tau_scale");
    if (T == 0) return MOCO_OK;
    if (!cost_dev || !loss_dev || !weights_dev) return fail(MOCO_ERR_INVALID_ARG, "null cost, loss or weights");
    DeviceGuard guard(plan->device);
    ShapePlan& sp = plan->shapes[shape_idx];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    plan->prof.begin(K_SOFTMIN, st);
    cudaError_t e = launch_softmin(cost_dev, T, sp.W * sp.W, tau_scale, loss_dev, weights_dev, st);
    plan->prof.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "k_softmin");
    return MOCO_OK;
}

moco_status moco_cost_backward(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                               const float* grad_cost_dev, float grad_scale, float* grad_template_dev,
                               float* grad_frames_dev, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0) return fail(MOCO_ERR_INVALID_ARG, "T < 0");
    ShapePlan& sp = plan->shapes[shape_idx];
    if (sp.levels != 0) return fail(MOCO_ERR_UNSUPPORTED, "the adjoint needs levels == 0");
    if (grad_smem_bytes(sp.wm1) > 227 * 1024) return fail(MOCO_ERR_UNSUPPORTED, "window too large for the adjoint");
    if (T == 0) return MOCO_OK;
    if (!frames_dev || !grad_cost_dev || !grad_template_dev)
        return fail(MOCO_ERR_INVALID_ARG, "null frames, grad_cost or grad_template");
    DeviceGuard guard(plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Profiler& P = plan->prof;
    cudaError_t e = cudaSuccess;
    if (sp.has_fft) {
        // sum_f a'_f (correlated with) q_f = IDFT2(sum_f A_f conj(Q_f)), group by group
        // through the search's own row spectra X; QX takes Y's place.
        const int64_t mn = (int64_t)sp.desc.m * sp.desc.n, K = (int64_t)sp.W * sp.W;
        e = cudaMemsetAsync(sp.grad_spec, 0, (size_t)sp.ncv * sp.Nr * 8, st);
        for (int64_t f0 = 0; f0 < T && e == cudaSuccess; f0 += sp.group) {
            const int64_t g = std::min<int64_t>(sp.group, T - f0);
            P.begin(K_ADJ_ROWS, st);
            e = launch_frame_rows(sp.Nc, false, frames_dev + f0 * mn, mn, g, sp.desc.m, sp.desc.n, 0, sp.mc, sp.nc,
                                  sp.coff_i, nullptr, sp.twc, sp.X, sp.x_fstride, sp.ldx, sp.rowE, sp.colE, sp.tot,
                                  sp.corners, sp.wm1, sp.dev_err, sp.group, st);
            if (e == cudaSuccess)
                e = launch_q_rows(sp.Nc, grad_cost_dev + f0 * K, sp.inv_area, grad_scale, sp.wm1, g, sp.twc, sp.Y, st);
            P.end(st);
            P.begin(K_ADJ_COLS, st);
            if (e == cudaSuccess)
                e = launch_adj_cols(sp.Nr, sp.X, sp.x_fstride, sp.ldx, sp.mc, sp.ncv, sp.Y, sp.wm1, g, sp.twr,
                                    sp.grad_spec, sp.dev_err, st);
            P.end(st);
        }
        P.begin(K_ADJ_INV, st);
        if (e == cudaSuccess)
            e = launch_adj_inverse(sp.Nr, sp.Nc, sp.grad_spec, sp.ncv, sp.mc, sp.nc, sp.twr, sp.twc, sp.X,
                                   sp.grad_acc, st);
        P.end(st);
    }
    P.begin(K_BACKWARD, st);
    if (e == cudaSuccess)
        e = launch_grad(frames_dev, T, sp.desc.m, sp.desc.n, sp.wm1, grad_cost_dev, grad_scale, sp.inv_area,
                        sp.coff_i, sp.tmpl, sp.f32 ? 1 : 0, sp.has_fft ? 0 : 1, sp.grad_acc, sp.grad_Q,
                        grad_template_dev, grad_frames_dev, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernels");
    return MOCO_OK;
}

moco_status moco_softmin_grad(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_dev, int64_t T,
                              double tau_scale, float grad_scale, double* cost_dev, double* loss_dev,
                              float* weights_dev, float* grad_template_dev, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0 || !(tau_scale >= 0.0)) return fail(MOCO_ERR_INVALID_ARG, "T < 0 or bad tau_scale");
    ShapePlan& sp = plan->shapes[shape_idx];
    if (sp.levels != 0) return fail(MOCO_ERR_UNSUPPORTED, "the adjoint needs levels == 0");
    if (T == 0) return MOCO_OK;
    if (!frames_dev || !cost_dev || !loss_dev || !weights_dev || !grad_template_dev)
        return fail(MOCO_ERR_INVALID_ARG, "null frames, cost, loss, weights or grad_template");
    if (!aligned16(frames_dev)) return fail(MOCO_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    if (sp.form != MOCO_XCORR_FFT_FP32 || !sp.has_fft) {
        moco_status s = moco_cost_surface(plan, shape_idx, frames_dev, T, cost_dev, stream);
        if (s == MOCO_OK) s = moco_softmin(plan, shape_idx, cost_dev, T, tau_scale, loss_dev, weights_dev, stream);
        if (s == MOCO_OK)
            s = moco_cost_backward(plan, shape_idx, frames_dev, T, weights_dev, grad_scale, grad_template_dev, nullptr,
                                   stream);
        return s;
    }
    DeviceGuard guard(plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Profiler& P = plan->prof;
    const int64_t mn = (int64_t)sp.desc.m * sp.desc.n, WW = (int64_t)sp.W * sp.W;
    cudaError_t e = cudaMemsetAsync(sp.grad_spec, 0, (size_t)sp.ncv * sp.Nr * 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint spectrum clear");
    for (int64_t f0 = 0; f0 < T; f0 += sp.group) {
        const int64_t g = std::min<int64_t>(sp.group, T - f0);
        // the search leaves this batch's row spectra in X and frees Y
        moco_status s = search_group(sp, frames_dev + f0 * mn, g, cost_dev + f0 * WW, nullptr, nullptr, st);
        if (s != MOCO_OK) return s;
        P.begin(K_SOFTMIN, st);
        e = launch_softmin(cost_dev + f0 * WW, g, (int)WW, tau_scale, loss_dev + f0, weights_dev + f0 * WW, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_softmin");
        P.begin(K_ADJ_ROWS, st);
        e = launch_q_rows(sp.Nc, weights_dev + f0 * WW, sp.inv_area, grad_scale, sp.wm1, g, sp.twc, sp.Y, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_q_rows");
        P.begin(K_ADJ_COLS, st);
        e = launch_adj_cols(sp.Nr, sp.X, sp.x_fstride, sp.ldx, sp.mc, sp.ncv, sp.Y, sp.wm1, g, sp.twr, sp.grad_spec,
                            sp.dev_err, st);
        P.end(st);
        if (e != cudaSuccess) return cuda_fail(e, "k_adj_cols");
    }
    P.begin(K_ADJ_INV, st);
    e = launch_adj_inverse(sp.Nr, sp.Nc, sp.grad_spec, sp.ncv, sp.mc, sp.nc, sp.twr, sp.twc, sp.X, sp.grad_acc, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint inverse");
    P.begin(K_BACKWARD, st);
    e = launch_grad(frames_dev, T, sp.desc.m, sp.desc.n, sp.wm1, weights_dev, grad_scale, sp.inv_area, sp.coff_i,
                    sp.tmpl, sp.f32 ? 1 : 0, 0, sp.grad_acc, sp.grad_Q, grad_template_dev, nullptr, st);
    P.end(st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernels");
    return MOCO_OK;
}

moco_status moco_selftest_wait(moco_plan_t plan, int32_t shape_idx, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    DeviceGuard guard(plan->device);
    cudaError_t e = launch_wait_selftest(plan->shapes[shape_idx].dev_err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "moco_selftest_wait");
    return MOCO_OK;
}

moco_status moco_plan_status(moco_plan_t plan) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    DeviceGuard guard(plan->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "moco_plan_status");
    moco_status r = MOCO_OK;
    for (auto& sp : plan->shapes) {
        unsigned int flag = 0;
        e = cudaMemcpy(&flag, sp.dev_err, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "status read-back");
        if (flag) {
            cudaMemset(sp.dev_err, 0, 4);
            r = fail(MOCO_ERR_TIMEOUT, "a bounded device-side wait gave up");
        }
    }
    return r;
}

moco_status moco_profile_enable(moco_plan_t plan, int32_t max_launches) {
    if (!plan || max_launches < 0) return fail(MOCO_ERR_INVALID_ARG, "null plan or negative size");
    DeviceGuard guard(plan->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "moco_profile_enable");
    Profiler& P = plan->prof;
    for (auto& ev : P.pool) cudaEventDestroy(ev);
    P.pool.clear();
    P.marks.clear();
    P.used = 0;
    P.truncated = false;
    P.on = max_launches > 0;
    for (int32_t k = 0; k < 2 * max_launches; ++k) {
        cudaEvent_t ev;
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            P.on = false;
            return cuda_fail(e, "event pool");
        }
        P.pool.push_back(ev);
    }
    return MOCO_OK;
}

moco_status moco_profile_read(moco_plan_t plan, moco_kernel_stat* stats, int32_t capacity, int32_t* count,
                              int32_t reset) {
    if (!plan || !count || capacity < 0 || (capacity > 0 && !stats)) return fail(MOCO_ERR_INVALID_ARG, "bad arguments");
    Profiler& P = plan->prof;
    if (!P.on) return fail(MOCO_ERR_INVALID_ARG, "profiling is not enabled");
    DeviceGuard guard(plan->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "moco_profile_read");
    int64_t launches[K_COUNT] = {0};
    double ms[K_COUNT] = {0};
    for (auto& mk : P.marks) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, P.pool[mk.second], P.pool[mk.second + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        launches[mk.first] += 1;
        ms[mk.first] += t;
    }
    int32_t c = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        if (!launches[k]) continue;
        if (c < capacity) {
            std::memset(stats[c].name, 0, sizeof(stats[c].name));
            std::strncpy(stats[c].name, kKernelNames[k], sizeof(stats[c].name) - 1);
            stats[c].launches = launches[k];
            stats[c].total_ms = ms[k];
        }
        ++c;
    }
    *count = c;
    if (reset) {
        P.marks.clear();
        P.used = 0;
        P.truncated = false;
    }
    return MOCO_OK;
}

moco_status moco_align_host(moco_plan_t plan, int32_t shape_idx, const uint16_t* frames_host, int64_t T,
                            int32_t* shifts_host, void* stream) {
    if (!plan) return fail(MOCO_ERR_INVALID_ARG, "null plan");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    if (T < 0) return fail(MOCO_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return MOCO_OK;
    if (!frames_host || !shifts_host) return fail(MOCO_ERR_INVALID_ARG, "null frames or shifts");
    DeviceGuard guard(plan->device);
    ShapePlan& sp = plan->shapes[shape_idx];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t cp = plan->aux;
    cudaEvent_t copied[2] = {plan->ev[0], plan->ev[1]}, done[2] = {plan->ev[2], plan->ev[3]};
    const int64_t mn = (int64_t)sp.desc.m * sp.desc.n;
    cudaError_t e = cudaEventRecord(done[0], st);
    if (e == cudaSuccess) e = cudaEventRecord(done[1], st);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    int k = 0;
    for (int64_t f0 = 0; f0 < T; f0 += sp.stage_frames, k ^= 1) {
        const int64_t g = std::min<int64_t>(sp.stage_frames, T - f0);
        // The copy into staging buffer k waits for the compute that last used it.
        e = cudaStreamWaitEvent(cp, done[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sp.stage[k], frames_host + f0 * mn, (size_t)(g * mn * 2), cudaMemcpyHostToDevice, cp);
        if (e == cudaSuccess) e = cudaEventRecord(copied[k], cp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, copied[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device staging");
        moco_status s = align_frames(sp, sp.stage[k], g, sp.stage_shifts[k], nullptr, nullptr, nullptr, st);
        if (s != MOCO_OK) return s;
        e = cudaMemcpyAsync(shifts_host + 2 * f0, sp.stage_shifts[k], (size_t)(g * 8), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(done[k], st);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host shifts");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "moco_align_host");
    return MOCO_OK;
}

}  // extern "C"
