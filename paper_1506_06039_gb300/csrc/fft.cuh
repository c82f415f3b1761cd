// Hand-written FP32 complex FFT building blocks for the cross-correlation
// term h_{s,t} of Section 2 (computed, as the paper says, through 2-D FFTs of
// the zero-padded images).
//
// Two layers:
//  * Dft<R, INV>: an R-point DFT held entirely in registers (R <= 36), built
//    by Cooley-Tukey from hand-written 2-, 3-, 4- and 5-point kernels. All
//    indices are compile-time constants after unrolling, so twiddles become
//    constant-bank operands.
//  * fft4_fwd / fft4_inv: an N = N1 * N2 point transform of several rows held
//    in shared memory, done as the classic "four-step": N2 tasks per row each
//    run an N1-point codelet on a stride-N2 comb, multiply by omega_N^(n2 k1),
//    then N1 tasks per row each run an N2-point codelet on a contiguous block.
//    The forward transform leaves X[k] at position N2*(k mod N1) + k/N1; the
//    inverse takes exactly that layout and returns natural order, so the
//    frequency-domain product in between never needs a reorder. Positions
//    map to shared-memory slots through sk() (a bank-conflict skew).
#pragma once
#include <cuda_runtime.h>
#include "twiddles.cuh"

namespace moco {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// Multiply by -i (forward direction) or +i (inverse direction).
template <bool INV>
__device__ __forceinline__ float2 rot_q(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Multiply by omega_R^e (conjugated for the inverse), e a compile-time constant
// after unrolling; quarter turns are exact sign/swap operations.
template <int R, bool INV>
__device__ __forceinline__ float2 twiddle_R(float2 a, int e) {
    if (e == 0) return a;
    if (4 * e == R) return rot_q<INV>(a);
    if (2 * e == R) return cneg(a);
    if (4 * e == 3 * R) return rot_q<!INV>(a);
    float2 w = Tw<R>::get(e);
    if (INV) w.y = -w.y;
    return cmul(a, w);
}

template <int R>
struct Split;
template <> struct Split<6> { enum { A = 2, B = 3 }; };
template <> struct Split<8> { enum { A = 2, B = 4 }; };
template <> struct Split<9> { enum { A = 3, B = 3 }; };
template <> struct Split<10> { enum { A = 2, B = 5 }; };
template <> struct Split<12> { enum { A = 4, B = 3 }; };
template <> struct Split<15> { enum { A = 3, B = 5 }; };
template <> struct Split<16> { enum { A = 4, B = 4 }; };
template <> struct Split<18> { enum { A = 2, B = 9 }; };
template <> struct Split<20> { enum { A = 4, B = 5 }; };
template <> struct Split<24> { enum { A = 8, B = 3 }; };
template <> struct Split<25> { enum { A = 5, B = 5 }; };
template <> struct Split<27> { enum { A = 3, B = 9 }; };
template <> struct Split<30> { enum { A = 2, B = 15 }; };
template <> struct Split<32> { enum { A = 4, B = 8 }; };
template <> struct Split<36> { enum { A = 4, B = 9 }; };

// y_k = sum_j x_j omega^(jk), omega = exp(-2 pi i / R) forward, conjugate inverse.
template <int R, bool INV>
struct Dft {
    __device__ __forceinline__ static void run(float2 (&x)[R]) {
        constexpr int A = Split<R>::A, B = Split<R>::B;
        float2 y[B][A];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            float2 t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = x[b + B * a];
            Dft<A, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) y[b][k1] = twiddle_R<R, INV>(t[k1], (b * k1) % R);
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = y[b][k1];
            Dft<B, INV>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
        }
    }
};

template <bool INV>
struct Dft<1, INV> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[2]) {
        float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<3, INV> {
    // y1 = x0 - (x1+x2)/2 - i*sin(2pi/3)*(x1-x2) (forward), y2 the conjugate rotation.
    __device__ __forceinline__ static void run(float2 (&x)[3]) {
        const float s3 = 0.866025403784438646763723170752936183f;
        float2 t1 = cadd(x[1], x[2]);
        float2 t2 = csub(x[1], x[2]);
        float2 y0 = cadd(x[0], t1);
        float2 m = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
        float2 r = rot_q<INV>(cscale(t2, s3));
        x[0] = y0;
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[4]) {
        float2 a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        float2 c = cadd(x[1], x[3]), d = rot_q<INV>(csub(x[1], x[3]));
        x[0] = cadd(a, c);
        x[2] = csub(a, c);
        x[1] = cadd(b, d);
        x[3] = csub(b, d);
    }
};

template <bool INV>
struct Dft<5, INV> {
    // With c1 = cos(2pi/5), c2 = cos(4pi/5), s1 = sin(2pi/5), s2 = sin(4pi/5):
    //   y1,4 = x0 + c1 (x1+x4) + c2 (x2+x3) -/+ i [s1 (x1-x4) + s2 (x2-x3)]
    //   y2,3 = x0 + c2 (x1+x4) + c1 (x2+x3) -/+ i [s2 (x1-x4) - s1 (x2-x3)]
    __device__ __forceinline__ static void run(float2 (&x)[5]) {
        const float c1 = 0.309016994374947424102293417182819059f;
        const float c2 = -0.809016994374947424102293417182819059f;
        const float s1 = 0.951056516295153572116439333379382143f;
        const float s2 = 0.587785252292473129168705954639072769f;
        float2 p1 = cadd(x[1], x[4]), m1 = csub(x[1], x[4]);
        float2 p2 = cadd(x[2], x[3]), m2 = csub(x[2], x[3]);
        float2 x0 = x[0];
        float2 a1 = make_float2(fmaf(c2, p2.x, fmaf(c1, p1.x, x0.x)), fmaf(c2, p2.y, fmaf(c1, p1.y, x0.y)));
        float2 a2 = make_float2(fmaf(c1, p2.x, fmaf(c2, p1.x, x0.x)), fmaf(c1, p2.y, fmaf(c2, p1.y, x0.y)));
        float2 b1 = make_float2(fmaf(s2, m2.x, s1 * m1.x), fmaf(s2, m2.y, s1 * m1.y));
        float2 b2 = make_float2(fmaf(-s1, m2.x, s2 * m1.x), fmaf(-s1, m2.y, s2 * m1.y));
        b1 = rot_q<INV>(b1);
        b2 = rot_q<INV>(b2);
        x[0] = cadd(x0, cadd(p1, p2));
        x[1] = cadd(a1, b1);
        x[4] = csub(a1, b1);
        x[2] = cadd(a2, b2);
        x[3] = csub(a2, b2);
    }
};

// ---- Four-step transforms of rows in shared memory -------------------------

template <int N>
struct Four;
#define MOCO_FOUR(N_, A_, B_) \
    template <> struct Four<N_> { enum { N1 = A_, N2 = B_ }; };
MOCO_FOUR(48, 8, 6)
MOCO_FOUR(64, 8, 8)
MOCO_FOUR(96, 8, 12)
MOCO_FOUR(128, 8, 16)
MOCO_FOUR(144, 16, 9)
MOCO_FOUR(160, 16, 10)
MOCO_FOUR(192, 16, 12)
MOCO_FOUR(256, 16, 16)
MOCO_FOUR(288, 16, 18)
MOCO_FOUR(320, 16, 20)
MOCO_FOUR(384, 16, 24)
MOCO_FOUR(512, 16, 32)
MOCO_FOUR(576, 16, 36)
#undef MOCO_FOUR

// Shared-memory slot of logical position p in a row: with an even N2 one
// spare slot follows every N2 positions, so that the second stage's
// contiguous N2-blocks (one per thread) start on different banks.
// Row stride ROW: the first forward and second inverse stages run N2 tasks
// per row along the row, so a half-warp (16 complex values, 128 bytes)
// straddles two rows; a stride congruent to N2 modulo 16 complex values
// makes consecutive tasks land on consecutive bank pairs across the row
// boundary (N1 = 16 sizes whose N2 is not a multiple of 16). Otherwise one
// more than the skewed length (odd: row-strided reads stay conflict-free).
template <int N>
struct Skew {
    enum {
        S = (Four<N>::N2 % 2 == 0) ? 1 : 0,
        BASE = N + S * Four<N>::N1,
        ROW = (Four<N>::N1 == 16 && Four<N>::N2 % 16 != 0) ? BASE + ((Four<N>::N2 - BASE) % 16 + 16) % 16
                                                           : BASE + 1
    };
};
template <int N>
__device__ __forceinline__ int sk(int p) {
    return Skew<N>::S ? p + p / Four<N>::N2 : p;
}
// Row stride (in complex elements) of a transform buffer: skewed length + 1.
template <int N>
constexpr int fft_ld() { return Skew<N>::ROW; }

// Position of spectral index k in the forward output layout.
template <int N>
__device__ __forceinline__ int spec_pos(int k) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2;
    return N2 * (k % N1) + k / N1;
}

// Twiddle tables (in shared memory), both holding omega_N^(n2*k1) =
// exp(-2 pi i n2 k1 / N) for n2 < N2, k1 < N1, in the order the lanes of a
// warp read them so that the reads are conflict-free:
//   forward: twf[k1*N2 + n2] (lanes run over n2),
//   inverse: twi[n2*N1 + k1] (lanes run over k1).
// The global copy is [twf | twi], 2N entries.

// Second stage of the forward transform (after a barrier that follows the
// first): N1 tasks per row, one N2-point codelet each; ends with a barrier.
template <int N>
__device__ void fft4_fwd_stage2(float2* buf, int ld, int rows, int tid, int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;
    for (int task = tid; task < rows * N1; task += nthr) {
        int r = task / N1, k1 = task - r * N1;
        float2* p = buf + r * ld + B * k1;
        float2 x[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) x[n2] = p[n2];
        Dft<N2, false>::run(x);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) p[k2] = x[k2];
    }
    __syncthreads();
}

// First stage of the forward transform with row r's natural-order input
// x[n] = fetch(r, n) taken from anywhere; the stage's output goes to buf
// (rows at buf + r * ld) in the layout fft4_fwd_stage2 continues from. No
// barrier.
template <int N, typename Fetch>
__device__ void fft4_fwd_stage1_gen(Fetch fetch, float2* buf, int ld, int rows, const float2* twf, int tid,
                                    int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;
    for (int task = tid; task < rows * N2; task += nthr) {
        int r = task / N2, n2 = task - r * N2;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = fetch(r, n1 * N2 + n2);
        Dft<N1, false>::run(x);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) x[k1] = cmul(x[k1], twf[k1 * N2 + n2]);
        float2* p = buf + r * ld + n2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) p[B * k1] = x[k1];
    }
}

// The same with the input read from a plain (unskewed) array: row r's
// x[n] = src[r * lds + n] for n < valid, zero beyond.
template <int N>
__device__ void fft4_fwd_stage1_from(const float2* src, int lds, int valid, float2* buf, int ld, int rows,
                                     const float2* twf, int tid, int nthr) {
    fft4_fwd_stage1_gen<N>(
        [&](int r, int n) { return n < valid ? src[r * lds + n] : make_float2(0.f, 0.f); }, buf, ld, rows, twf, tid,
        nthr);
}

// Forward transform of `rows` rows at buf + r*ld (natural-order input).
// Every thread of the block must call this (it synchronises).
template <int N>
__device__ void fft4_fwd(float2* buf, int ld, int rows, const float2* twf, int tid, int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;  // B: skewed block stride
    for (int task = tid; task < rows * N2; task += nthr) {
        int r = task / N2, n2 = task - r * N2;
        float2* p = buf + r * ld + n2;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = p[B * n1];
        Dft<N1, false>::run(x);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) x[k1] = cmul(x[k1], twf[k1 * N2 + n2]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) p[B * k1] = x[k1];
    }
    __syncthreads();
    fft4_fwd_stage2<N>(buf, ld, rows, tid, nthr);
}

// The middle of a forward transform, a pointwise product and the inverse, in
// one pass over registers: after the forward transform's first stage (and a
// barrier), each task's contiguous N2-block is the same block that the
// forward second stage writes, the product reads (the spectrum's forward
// output layout keeps block k1 together) and the inverse first stage reads.
// So task (r, k1) runs the forward N2-point codelet, multiplies by
// spec[r * spec_ld + N2 * k1 + k2], runs the inverse N2-point codelet and
// its twiddles, and writes the block back once. Ends with a barrier; the
// inverse's second stage (fft4_inv_stage2) completes the inverse.
template <int N>
__device__ void fft4_fwd2_mul_inv1(float2* buf, int ld, int rows, const float2* spec, int spec_ld,
                                   const float2* twi, int tid, int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;
    for (int task = tid; task < rows * N1; task += nthr) {
        int r = task / N1, k1 = task - r * N1;
        float2* p = buf + r * ld + B * k1;
        const float2* q = spec + r * spec_ld + N2 * k1;
        float2 x[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) x[n2] = p[n2];
        Dft<N2, false>::run(x);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) x[k2] = cmul(x[k2], q[k2]);
        Dft<N2, true>::run(x);
#pragma unroll
        for (int n2 = 1; n2 < N2; ++n2) x[n2] = cmulc(x[n2], twi[n2 * N1 + k1]);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) p[n2] = x[n2];
    }
    __syncthreads();
}

// Second stage of the inverse transform (after its first stage and a
// barrier): N2 tasks per row, one N1-point codelet each; ends with a barrier.
template <int N>
__device__ void fft4_inv_stage2(float2* buf, int ld, int rows, int tid, int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;
    for (int task = tid; task < rows * N2; task += nthr) {
        int r = task / N2, n2 = task - r * N2;
        float2* p = buf + r * ld + n2;
        float2 x[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) x[k1] = p[B * k1];
        Dft<N1, true>::run(x);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) p[B * n1] = x[n1];
    }
    __syncthreads();
}

// Inverse (unnormalised, omega^+) transform: input in the forward output
// layout, output in natural order.
template <int N>
__device__ void fft4_inv(float2* buf, int ld, int rows, const float2* twi, int tid, int nthr) {
    constexpr int N1 = Four<N>::N1, N2 = Four<N>::N2, B = N2 + Skew<N>::S;  // B: skewed block stride
    for (int task = tid; task < rows * N1; task += nthr) {
        int r = task / N1, k1 = task - r * N1;
        float2* p = buf + r * ld + B * k1;
        float2 x[N2];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) x[k2] = p[k2];
        Dft<N2, true>::run(x);
#pragma unroll
        for (int n2 = 1; n2 < N2; ++n2) x[n2] = cmulc(x[n2], twi[n2 * N1 + k1]);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) p[n2] = x[n2];
    }
    __syncthreads();
    for (int task = tid; task < rows * N2; task += nthr) {
        int r = task / N2, n2 = task - r * N2;
        float2* p = buf + r * ld + n2;
        float2 x[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) x[k1] = p[B * k1];
        Dft<N1, true>::run(x);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) p[B * n1] = x[n1];
    }
    __syncthreads();
}

}  // namespace moco
