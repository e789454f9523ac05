// Two-pass FFT of lines held in shared memory (FP32 or FP64), L = A * B with A, B in {2, 4, 8, 16, 32}.
//
// With l = b + B a (input index) and k = k1 + A k2 (output index), the DFT factors as
//   X[k1 + A k2] = sum_b wB^(b k2) [ w^(b k1) sum_a wA^(a k1) x[b + B a] ],   w = exp(-2 pi i / L),
// so a forward transform is
//   pass 1: for every b, an A-point DFT over a, times w^(b k1), written back to the
//           positions it was read from (b + B k1);
//   pass 2: for every k1, a B-point DFT over b, written back to the positions b + B k1
//           it was read from, which then hold X[k1 + A k2] at position k2 + B k1.
// Each thread owns the positions it reads, so a pass needs no barrier inside it and every
// element makes two round trips through shared memory (a radix-4 Stockham FFT makes
// log4 L).  The spectrum is left in this "transposed" order: kz sits at position
// tpos(kz) = kz / A + B (kz % A).  The inverse transform runs the passes in the
// opposite order with conjugate twiddles and takes the transposed order to natural order:
//   pass 1: for every k1, a B-point inverse DFT over k2 (positions k2 + B k1), times
//           w^-(b k1), written to positions b + B k1;
//   pass 2: for every b, an A-point inverse DFT over k1, giving x[b + B a] at b + B a.
// Small DFTs run in registers (decimation in time down to 4-point butterflies) with the
// twiddles of 8 and 16 points written as exact constants (cos and sin of multiples of pi/8).
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace fft2 {

constexpr double kC1 = 0.92387953251128674;  // cos(pi/8)
constexpr double kS1 = 0.38268343236508978;  // sin(pi/8)
constexpr double kC2 = 0.70710678118654752;  // cos(pi/4)
constexpr double kC16 = 0.98078528040323044913;  // cos(pi/16)
constexpr double kS16 = 0.19509032201612826785;  // sin(pi/16)
constexpr double kC316 = 0.83146961230254523708;  // cos(3 pi/16)
constexpr double kS316 = 0.55557023301960222474;  // sin(3 pi/16)

template <typename C>
__device__ __forceinline__ C rot(C a, double c, double s) {  // a * (c + i s), in the precision of C
    using R = decltype(a.x);
    const R cr = (R)c, sr = (R)s;
    return mk(a.x * cr - a.y * sr, a.x * sr + a.y * cr);
}

template <int N, typename C = float2>
struct DFT;
template <typename C>
struct DFT<2, C> {
    static __device__ __forceinline__ void run(C* v, int) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <typename C>
struct DFT<4, C> {
    static __device__ __forceinline__ void run(C* v, int dir) { dft4(v[0], v[1], v[2], v[3], dir); }
};
template <typename C>
struct DFT<8, C> {
    static __device__ __forceinline__ void run(C* v, int dir) {
        C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        dft4(e[0], e[1], e[2], e[3], dir);
        dft4(o[0], o[1], o[2], o[3], dir);
        const double d = (double)dir;
        o[1] = rot(o[1], kC2, d * kC2);
        o[2] = cmul_i(o[2], dir);
        o[3] = rot(o[3], -kC2, d * kC2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};
template <typename C>
struct DFT<16, C> {
    static __device__ __forceinline__ void run(C* v, int dir) {
        C e[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        DFT<8, C>::run(e, dir);
        DFT<8, C>::run(o, dir);
        const double d = (double)dir;
        o[1] = rot(o[1], kC1, d * kS1);
        o[2] = rot(o[2], kC2, d * kC2);
        o[3] = rot(o[3], kS1, d * kC1);
        o[4] = cmul_i(o[4], dir);
        o[5] = rot(o[5], -kS1, d * kC1);
        o[6] = rot(o[6], -kC2, d * kC2);
        o[7] = rot(o[7], -kC1, d * kS1);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 8] = csub(e[k], o[k]);
        }
    }
};

// a * exp(dir i pi k / 16), k in 0..15 a compile-time constant after unrolling
template <typename C>
__device__ __forceinline__ C twist32(C a, int k, int dir) {
    const double d = (double)dir;
    switch (k) {
        case 0: return a;
        case 1: return rot(a, kC16, d * kS16);
        case 2: return rot(a, kC1, d * kS1);
        case 3: return rot(a, kC316, d * kS316);
        case 4: return rot(a, kC2, d * kC2);
        case 5: return rot(a, kS316, d * kC316);
        case 6: return rot(a, kS1, d * kC1);
        case 7: return rot(a, kS16, d * kC16);
        case 8: return cmul_i(a, dir);
        case 9: return rot(a, -kS16, d * kC16);
        case 10: return rot(a, -kS1, d * kC1);
        case 11: return rot(a, -kS316, d * kC316);
        case 12: return rot(a, -kC2, d * kC2);
        case 13: return rot(a, -kC316, d * kS316);
        case 14: return rot(a, -kC1, d * kS1);
        default: return rot(a, -kC16, d * kS16);
    }
}

template <typename C>
struct DFT<32, C> {
    static __device__ __forceinline__ void run(C* v, int dir) {
        C e[16], o[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        DFT<16, C>::run(e, dir);
        DFT<16, C>::run(o, dir);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const C t = twist32(o[k], k, dir);
            v[k] = cadd(e[k], t);
            v[k + 16] = csub(e[k], t);
        }
    }
};

// a * w^n, w = exp(dir 2 pi i / N), N in {4, 8, 16, 32}, n < N/2 a compile-time constant after unrolling
template <int N, typename C>
__device__ __forceinline__ C twist(C a, int n, int dir) {
    if constexpr (N == 32) return twist32(a, n, dir);
    const double d = (double)dir;
    switch (n * (16 / N)) {  // the same angle in sixteenths of a turn
        case 0: return a;
        case 1: return rot(a, kC1, d * kS1);
        case 2: return rot(a, kC2, d * kC2);
        case 3: return rot(a, kS1, d * kC1);
        case 4: return cmul_i(a, dir);
        case 5: return rot(a, -kS1, d * kC1);
        case 6: return rot(a, -kC2, d * kC2);
        default: return rot(a, -kC1, d * kS1);
    }
}

// N-point DFT of v[0..N/2) with v[N/2..N) taken as zero (not read): split in frequency,
// X[2k] = DFT_{N/2}(x)[k], X[2k+1] = DFT_{N/2}(x w^n)[k]; all N outputs written to v.
template <int N, typename C>
__device__ __forceinline__ void dft_half_in(C* v, int dir) {
    C e[N / 2], o[N / 2];
#pragma unroll
    for (int n = 0; n < N / 2; ++n) {
        e[n] = v[n];
        o[n] = twist<N>(v[n], n, dir);
    }
    DFT<N / 2, C>::run(e, dir);
    DFT<N / 2, C>::run(o, dir);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        v[2 * k] = e[k];
        v[2 * k + 1] = o[k];
    }
}

// first N/2 outputs of the N-point DFT of v (split in time): X[k] = E[k] + w^k O[k], k < N/2
template <int N, typename C>
__device__ __forceinline__ void dft_half_out(C* v, int dir) {
    C e[N / 2], o[N / 2];
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        e[k] = v[2 * k];
        o[k] = v[2 * k + 1];
    }
    DFT<N / 2, C>::run(e, dir);
    DFT<N / 2, C>::run(o, dir);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) v[k] = cadd(e[k], twist<N>(o[k], k, dir));
}

// factorisation L = A * B used for each length (8 <= L <= 512)
__host__ __device__ constexpr int split_a(int L) { return L <= 16 ? 4 : (L <= 64 ? 8 : (L <= 256 ? 16 : 32)); }
template <int L>
struct Split {
    static_assert(L >= 8 && L <= 512 && (L & (L - 1)) == 0, "two-pass FFT lengths are 8..512");
    static constexpr int A = split_a(L), B = L / A;
};

// position of frequency k in the transposed order left by the forward transform, and back
__host__ __device__ constexpr int tpos(int L, int k) { return k / split_a(L) + (L / split_a(L)) * (k % split_a(L)); }
__host__ __device__ constexpr int freq_at(int L, int p) { return p / (L / split_a(L)) + split_a(L) * (p % (L / split_a(L))); }

// Forward transform of NL lines, natural order in (elements l >= nin taken as zero and
// not read; nin <= L/2, so the upper half of every pass-1 input is zero at compile time),
// transposed order out.  Line n starts at s + off(n); elements at stride ES.
// tw[m] = exp(-2 pi i m / L).  Called by all NT threads; ends with a barrier.
// forward_g: the same, run by NT threads with index tid, sync() as the barrier between passes.
template <int L, int NT, class Off, typename C, class Sync>
__device__ __forceinline__ void forward_g(C* s, int NL, Off off, int ES, const C* tw, int nin, int tid, Sync sync) {
    constexpr int A = Split<L>::A, B = Split<L>::B;
    for (int t = tid; t < NL * B; t += NT) {
        const int n = t % NL, b = t / NL;
        C* ln = s + off(n);
        C v[A];
#pragma unroll
        for (int a = 0; a < A / 2; ++a) {
            const int l = b + B * a;
            v[a] = l < nin ? ln[l * ES] : C{};
        }
        dft_half_in<A>(v, -1);
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) ln[(b + B * k1) * ES] = v[k1];
    }
    sync();
    for (int t = tid; t < NL * A; t += NT) {
        const int n = t % NL, k1 = t / NL;
        C* ln = s + off(n) + B * k1 * ES;
        C v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) v[b] = ln[b * ES];
        DFT<B, C>::run(v, -1);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) ln[k2 * ES] = v[k2];
    }
    sync();
}
template <int L, int NT, class Off, typename C>
__device__ __forceinline__ void forward(C* s, int NL, Off off, int ES, const C* tw, int nin) {
    forward_g<L, NT>(s, NL, off, ES, tw, nin, (int)threadIdx.x, [] { __syncthreads(); });
}

// Inverse (unnormalised) transform of NL lines, transposed order in, natural order out;
// only outputs l < nout (<= L/2) are written.  Called by all NT threads; ends with a barrier.
// inverse_g: the same, run by NT threads with index tid, sync() as the barrier between passes.
template <int L, int NT, class Off, typename C, class Sync>
__device__ __forceinline__ void inverse_g(C* s, int NL, Off off, int ES, const C* tw, int nout, int tid, Sync sync) {
    constexpr int A = Split<L>::A, B = Split<L>::B;
    for (int t = tid; t < NL * A; t += NT) {
        const int n = t % NL, k1 = t / NL;
        C* ln = s + off(n) + B * k1 * ES;
        C v[B];
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) v[k2] = ln[k2 * ES];
        DFT<B, C>::run(v, +1);
#pragma unroll
        for (int b = 1; b < B; ++b) v[b] = cmul(v[b], cconj(tw[b * k1]));
#pragma unroll
        for (int b = 0; b < B; ++b) ln[b * ES] = v[b];
    }
    sync();
    for (int t = tid; t < NL * B; t += NT) {
        const int n = t % NL, b = t / NL;
        C* ln = s + off(n);
        C v[A];
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) v[k1] = ln[(b + B * k1) * ES];
        dft_half_out<A>(v, +1);
#pragma unroll
        for (int a = 0; a < A / 2; ++a) {
            const int l = b + B * a;
            if (l < nout) ln[l * ES] = v[a];
        }
    }
    sync();
}
template <int L, int NT, class Off, typename C>
__device__ __forceinline__ void inverse(C* s, int NL, Off off, int ES, const C* tw, int nout) {
    inverse_g<L, NT>(s, NL, off, ES, tw, nout, (int)threadIdx.x, [] { __syncthreads(); });
}

}  // namespace fft2
