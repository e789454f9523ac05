// Line transforms of the matvec's line path (Section IV-A on grids whose xy circulant is not
// square or is longer than 128): the forward FFTs along x and along y and the inverse FFT along
// y, TB lines to a CTA, each line in shared memory with the two-pass register FFT of fft2.cuh
// (two passes through shared memory per transform instead of one per radix-4 stage).
//
// Orders.  The forward transform leaves a line's spectrum in fft2's transposed order (position p
// holds frequency freq_at(L, p)).  The x transform stores it in the matvec's stored column order
// (column q holds kx = colkx[q], mirror pairs side by side, as the z passes expect); the y
// transform stores rows in the transposed order itself (row p holds ky = freq_at(Ly, p), the
// split the z passes take as (ay, by) = (A, B)).  The inverse transform reads that order back
// and writes natural order, cropped.  The inverse loads, all L elements of each line, are issued
// at once by cp.async; the forward ones (at most L/2 per line) are plain loads.  (The inverse x
// transform with the voxel-wise terms stays on the radix-4 line kernel, which measured faster
// with its epilogue: 5.6 ms against 6.1 ms for 8 right-hand sides on a 128 x 128 x 256 grid.)
#include "block.cuh"
#include "fft.cuh"
#include "fft2.cuh"
#include "line2.cuh"

namespace {

template <int L>
struct Line2Cfg {
    static constexpr int B = fft2::Split<L>::B;
    static constexpr int TB0 = 4096 / L;
    static constexpr int TB = TB0 > 32 ? 32 : TB0;  // lines per CTA
    static constexpr int LS = L + 1;                 // odd line stride: lanes on different lines stay apart
    static constexpr int NT0 = TB * B;
    static constexpr int NT = NT0 < 64 ? 64 : NT0;
    // shared memory: TB lines and the twiddles
    template <typename C>
    static constexpr size_t smem() {
        return sizeof(C) * (size_t)(TB * LS + L);
    }
};

// KIND 0: forward (natural in, spectrum out in the stored order); 1: inverse (stored order in,
// natural out, cropped).
// colkx: stored position q holds frequency colkx[q] (the x transforms), or NULL: position q
// holds transposed position q (the y transforms).
template <typename T, int L, int KIND>
__global__ void __launch_bounds__(Line2Cfg<L>::NT)
    line2_kernel(LineArgs a, const int* __restrict__ colkx, const typename CT<T>::C* __restrict__ twg) {
    using C = typename CT<T>::C;
    using Cfg = Line2Cfg<L>;
    constexpr int TB = Cfg::TB, LS = Cfg::LS, NT = Cfg::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* tw = s + TB * LS;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += NT) tw[m] = twg[m];
    const int ntile = (a.nb + TB - 1) / TB;
    const long long ai = blockIdx.x / ntile;
    const int b0 = (blockIdx.x % ntile) * TB;
    const C* in = reinterpret_cast<const C*>(a.in);
    C* out = reinterpret_cast<C*>(a.out);
    auto off = [](int n) { return n * LS; };
    // positions along the line axis: contiguous lines (il or ol == 1) put one line's elements on
    // consecutive threads, strided lines put the TB lines' element l on consecutive threads
    if constexpr (KIND == 0) {
        const bool cin = a.il == 1;
        for (int idx = tid; idx < TB * a.n_in; idx += NT) {
            const int n = cin ? idx / a.n_in : idx % TB, l = cin ? idx % a.n_in : idx / TB;
            const int b = b0 + n;
            s[off(n) + l] = b < a.nb ? in[ai * a.ia + (long long)l * a.il + (long long)b * a.ib] : mk(T(0), T(0));
        }
        __syncthreads();
        fft2::forward<L, NT>(s, TB, off, 1, tw, a.n_in);
        const bool outc = a.ol == 1;
        for (int idx = tid; idx < TB * L; idx += NT) {
            const int n = outc ? idx / L : idx % TB, q = outc ? idx % L : idx / TB;
            const int b = b0 + n;
            if (b >= a.nb) continue;
            const int p = colkx ? fft2::tpos(L, colkx[q]) : q;
            out[ai * a.oa + (long long)q * a.ol + (long long)b * a.ob] = s[off(n) + p];
        }
    } else {
        const bool cin = a.il == 1;
        for (int idx = tid; idx < TB * L; idx += NT) {
            const int n = cin ? idx / L : idx % TB, q = cin ? idx % L : idx / TB;
            const int b = b0 + n;
            const int p = colkx ? fft2::tpos(L, colkx[q]) : q;
            const bool ok = b < a.nb;
            cp_async_elem(s + off(n) + p, ok ? in + ai * a.ia + (long long)q * a.il + (long long)b * a.ib : in, ok);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        fft2::inverse<L, NT>(s, TB, off, 1, tw, a.n_out);
        const bool outc = a.ol == 1;
        for (int idx = tid; idx < TB * a.n_out; idx += NT) {
            const int n = outc ? idx / a.n_out : idx % TB, l = outc ? idx % a.n_out : idx / TB;
            const int b = b0 + n;
            if (b >= a.nb) continue;
            out[ai * a.oa + (long long)l * a.ol + (long long)b * a.ob] = s[off(n) + l];
        }
    }
}

template <typename T>
const typename CT<T>::C* twiddles(const vie_handle* h, int L);
template <>
const float2* twiddles<float>(const vie_handle* h, int L) {
    return h->tw32 + L;
}
template <>
const double2* twiddles<double>(const vie_handle* h, int L) {
    return h->tw64 + L;
}

template <typename T, int L, int KIND>
int launch_L(const char* name, const vie_handle* h, const LineArgs& a, const int* colkx, cudaStream_t s) {
    using C = typename CT<T>::C;
    using Cfg = Line2Cfg<L>;
    // the two-pass transforms take at most L/2 non-zero inputs (forward) or outputs (inverse)
    if ((KIND == 0 ? a.n_in : a.n_out) > L / 2 || (KIND == 0 ? a.n_out : a.n_in) != L) {
        set_error("line transform: a line needs at most L/2 inputs and L outputs (forward), or the reverse");
        return VIE_EINVAL;
    }
    constexpr size_t smem = Cfg::template smem<C>();
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(line2_kernel<T, L, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long blocks = (long long)a.na * ((a.nb + Cfg::TB - 1) / Cfg::TB);
    if (blocks <= 0) return VIE_OK;
    if (blocks > 0x7fffffffLL) {
        set_error("line FFT grid too large");
        return VIE_EINVAL;
    }
    // algorithmic bytes: inputs read once, outputs written once
    const double bytes = (double)sizeof(C) * (double)a.na * a.nb * (a.n_in + a.n_out);
    VIE_KLAUNCH_B(name, s, bytes,
                  line2_kernel<T, L, KIND><<<(unsigned)blocks, Cfg::NT, smem, s>>>(a, colkx, twiddles<T>(h, L)));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename T, int KIND>
int launch(const char* name, const vie_handle* h, int L, const LineArgs& a, const int* colkx, cudaStream_t s) {
    switch (L) {
        case 8: return launch_L<T, 8, KIND>(name, h, a, colkx, s);
        case 16: return launch_L<T, 16, KIND>(name, h, a, colkx, s);
        case 32: return launch_L<T, 32, KIND>(name, h, a, colkx, s);
        case 64: return launch_L<T, 64, KIND>(name, h, a, colkx, s);
        case 128: return launch_L<T, 128, KIND>(name, h, a, colkx, s);
        case 256: return launch_L<T, 256, KIND>(name, h, a, colkx, s);
        case 512: return launch_L<T, 512, KIND>(name, h, a, colkx, s);
    }
    set_error("line transform: unsupported length " + std::to_string(L));
    return VIE_EINVAL;
}

}  // namespace

bool line2_ok(int L) { return L >= 8 && L <= 512 && (L & (L - 1)) == 0; }

int line2_forward(const char* name, const vie_handle* h, int L, bool fp64, const LineArgs& a, const int* colkx,
                  cudaStream_t s) {
    return fp64 ? launch<double, 0>(name, h, L, a, colkx, s) : launch<float, 0>(name, h, L, a, colkx, s);
}

int line2_inverse(const char* name, const vie_handle* h, int L, bool fp64, const LineArgs& a, const int* colkx,
                  cudaStream_t s) {
    return fp64 ? launch<double, 1>(name, h, L, a, colkx, s) : launch<float, 1>(name, h, L, a, colkx, s);
}
