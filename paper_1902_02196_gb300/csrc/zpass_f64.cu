// FP64 z pass of the matvec (Section IV-A) with the 12 x 12 Green block product fused
// between the forward and inverse z transforms: the FP64 counterpart of zpass_f32.cu, for
// the refinement residuals, the post-processing and the plain FP64 solver; the N block from
// its 60 tensors, or (KOP) the K block (Eq. 8, 25) from its 30.
//
// Same tiling, item decoding and transposed z spectrum as the FP32 kernel.  FP64 values
// take twice the registers, so a thread cannot keep an octant point's 60 Green values
// resident: each frequency point streams them from the [..][60] layout in four groups of
// 15 tensors (960 contiguous bytes per point, served by L1/L2 for the four points of an
// item), and applies each group to the entries it feeds, one column at a time.  The
// kernel is bound by the FP64 pipe, so one shared-memory buffer per CTA suffices: two
// CTAs per SM overlap one's loads and stores with the other's arithmetic.
#include "block.cuh"
#include "fft2.cuh"
#include "zpass_f64.cuh"

namespace {

template <int LZ>
struct ZDCfg {
    static constexpr int TB = LZ <= 128 ? 4 : 2;
    static constexpr int NPAIR = TB / 2;
    static constexpr int NT0 = NPAIR * LZ / 2;
    static constexpr int NT = NT0 < 128 ? 128 : NT0;
    static constexpr int GS = LZ * TB + TB;  // 16-byte elements: quarter-warps of 8 lines stay apart
    static constexpr int BUF = 12 * GS;
    static constexpr size_t smem = sizeof(double2) * (size_t)(BUF + LZ);
};

__device__ __forceinline__ double2 xflip64(double2 v, unsigned m, int a) { return ((m >> a) & 1u) ? cneg(v) : v; }

// entries [start(t), start(t + 1)) of the N table (60 tensors) or of the K table (30)
template <bool KOP>
__device__ __forceinline__ int entry_start(int t) {
    if constexpr (KOP)
        return kKBlock.start[t];
    else
        return kBlock.start[t];
}
template <bool KOP>
__device__ __forceinline__ BlockEntry entry_at(int i) {
    if constexpr (KOP)
        return kKBlock.e[i];
    else
        return kBlock.e[i];
}

// y = B x at one column of one z position, the Green values streamed from gp (NG = 60 values of
// N, or 30 of K); input signs m, output signs mo
template <bool KOP>
__device__ __forceinline__ void point_product64(const double2* __restrict__ gp, double2* s, int gs, int off,
                                                unsigned m, unsigned mo) {
    constexpr int NGRP = KOP ? 2 : 4;  // groups of 15 tensors
    double2 xv[12], acc[12];
#pragma unroll
    for (int b = 0; b < 12; ++b) xv[b] = xflip64(s[b * gs + off], m, b);
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = make_double2(0.0, 0.0);
#pragma unroll
    for (int g = 0; g < NGRP; ++g) {
        double2 u[15];
#pragma unroll
        for (int q = 0; q < 15; ++q) u[q] = __ldg(gp + 15 * g + q);
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            const int t = 15 * g + q;
#pragma unroll
            for (int i = entry_start<KOP>(t); i < entry_start<KOP>(t + 1); ++i) {
                const BlockEntry en = entry_at<KOP>(i);
                cfma(acc[en.a], en.s > 0 ? u[q] : cneg(u[q]), xv[en.b]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) s[a * gs + off] = xflip64(acc[a], mo, a);
}

template <int LZ, bool KOP>
__global__ void __launch_bounds__(ZDCfg<LZ>::NT) zfused64_kernel(ZDArgs z, const double2* __restrict__ twg) {
    using Cfg = ZDCfg<LZ>;
    constexpr int NG = KOP ? 30 : 60;  // Green values per octant point
    constexpr int A = fft2::Split<LZ>::A, B = fft2::Split<LZ>::B, NT = Cfg::NT, TB = Cfg::TB;
    constexpr int NPAIR = Cfg::NPAIR, GS = Cfg::GS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* s = reinterpret_cast<double2*>(smem_raw);
    double2* tw = s + Cfg::BUF;
    const int tid = threadIdx.x;
    const int R = z.nact ? min(*z.nact, z.R) : z.R;
    dev_bytes_add(z.bctr, 16.0 * (2.0 * R * 12 * z.nz * z.Ly * z.Lx + (double)NG * z.Ox * z.Oy * z.Oz), R > 0);
    if (R <= 0) return;
    for (int m = tid; m < LZ; m += NT) tw[m] = twg[m];
    const int ntile = z.Lx / TB;
    const int py = blockIdx.x / ntile, ct = blockIdx.x % ntile, sc0 = ct * TB;
    const long long plane = (long long)z.Ly * z.Lx;
    const int ky = py / z.by + z.ay * (py % z.by);
    const int kyo = ky <= z.Ly / 2 ? ky : z.Ly - ky;
    const unsigned fy = ky > z.Ly / 2 ? z.my : 0u;
    const int nz = z.nz;
    auto line = [](int n) { return (n / TB) * GS + n % TB; };
    // K: the block's overall sign flips at points reflected along an odd number of axes
    const unsigned ko = KOP ? 0xFFFu : 0u;
    const bool ry = ky > z.Ly / 2;

    // block-product item of this thread (as in the FP32 kernel)
    const int ci = tid % NPAIR, j = tid / NPAIR;
    const bool single = ct == ntile - 1 && ci == NPAIR - 1;
    const int kx0 = z.colkx[sc0 + 2 * ci], kx1 = z.colkx[sc0 + 2 * ci + 1];
    const unsigned fx0 = kx0 > z.Lx / 2 ? z.mx : 0u, fx1 = kx1 > z.Lx / 2 ? z.mx : 0u;
    constexpr int NREG = (A / 2 - 1) * B;
    int pa = -1, pb = -1, pc = -1;
    if (j < NREG) {
        const int k1 = 1 + j / B, k2 = j % B;
        pa = k2 + B * k1;
        pb = (B - 1 - k2) + B * (A - k1);
    } else if (j < NREG + B / 2) {
        const int k2 = j - NREG;
        pa = k2 + B * (A / 2);
        pb = (B - 1 - k2) + B * (A / 2);
    } else if (j < LZ / 2) {
        const int k2 = j - NREG - B / 2;
        pa = k2;
        if (k2 == 0)
            pc = B / 2;
        else
            pb = B - k2;
    }
    const int kxo0 = kx0 <= z.Lx / 2 ? kx0 : z.Lx - kx0, kxo1 = kx1 <= z.Lx / 2 ? kx1 : z.Lx - kx1;
    const double2* gcol0 = z.green_t + ((long long)kyo * z.Ox + kxo0) * z.Oz * NG;
    const double2* gcol1 = z.green_t + ((long long)kyo * z.Ox + kxo1) * z.Oz * NG;

#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const double2* base = z.w + (long long)r * 12 * nz * plane + (long long)py * z.Lx + sc0;
        for (int idx = tid; idx < 12 * nz * TB; idx += NT) {
            const int c = idx % TB, l = (idx / TB) % nz, a = idx / (TB * nz);
            cp_async16(s + a * GS + l * TB + c, base + ((long long)a * nz + l) * plane + c);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        fft2::forward<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
        if (pa >= 0) {
            // points (pa, pb: one octant point; pc: kz = LZ/2), each column with its octant point
#pragma unroll 1
            for (int q = 0; q < 6; ++q) {
                const int e = q % 3, col = q / 3;
                const int pp = e == 0 ? pa : (e == 1 ? pb : pc);
                if (pp < 0) continue;
                const int kz = fft2::freq_at(LZ, pp);
                const int kzo = kz <= LZ / 2 ? kz : LZ - kz;
                const bool rz = kz > LZ / 2;
                const unsigned fz = rz ? z.mz : 0u;
                const double2* gp = ((single && col) ? gcol1 : gcol0) + (long long)kzo * NG;
                const unsigned mi = fy ^ fz ^ (col ? fx1 : fx0);
                const bool odd = ry ^ rz ^ (col ? kx1 > z.Lx / 2 : kx0 > z.Lx / 2);
                point_product64<KOP>(gp, s, GS, pp * TB + 2 * ci + col, mi, odd ? mi ^ ko : mi);
            }
        }
        __syncthreads();
        fft2::inverse<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
        double2* out = z.w + (long long)r * 12 * nz * plane + (long long)py * z.Lx + sc0;
        for (int idx = tid; idx < 12 * nz * TB; idx += NT) {
            const int c = idx % TB, l = (idx / TB) % nz, a = idx / (TB * nz);
            out[((long long)a * nz + l) * plane + c] = s[a * GS + l * TB + c];
        }
        __syncthreads();
    }
}

template <int LZ, bool KOP>
int launch_zd_L(const vie_handle* h, const ZDArgs& z, cudaStream_t s) {
    constexpr size_t smem = ZDCfg<LZ>::smem;
    constexpr double NG = KOP ? 30.0 : 60.0;
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(zfused64_kernel<LZ, KOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long blocks = (long long)z.Ly * (z.Lx / ZDCfg<LZ>::TB);
    const double bytes = z.nact ? kDevCounted : 16.0 * (2.0 * z.R * 12 * z.nz * z.Ly * z.Lx + NG * z.Ox * z.Oy * z.Oz);
    VIE_KLAUNCH_B(KOP ? "zpass_block_k_f64" : "zpass_block_f64", s, bytes,
                  zfused64_kernel<LZ, KOP><<<(unsigned)blocks, ZDCfg<LZ>::NT, smem, s>>>(z, h->tw64 + LZ));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <bool KOP>
int launch_zd(const vie_handle* h, const ZDArgs& z, cudaStream_t s) {
    switch (h->L[2]) {
        case 8: return launch_zd_L<8, KOP>(h, z, s);
        case 16: return launch_zd_L<16, KOP>(h, z, s);
        case 32: return launch_zd_L<32, KOP>(h, z, s);
        case 64: return launch_zd_L<64, KOP>(h, z, s);
        case 128: return launch_zd_L<128, KOP>(h, z, s);
        case 256: return launch_zd_L<256, KOP>(h, z, s);
        case 512: return launch_zd_L<512, KOP>(h, z, s);
    }
    set_error("FP64 z pass: unsupported length");
    return VIE_EINVAL;
}

}  // namespace

int zpass_f64_fused(const vie_handle* h, const ZDArgs& z, cudaStream_t s) { return launch_zd<false>(h, z, s); }

int zpass_f64_fused_k(const vie_handle* h, const ZDArgs& z, cudaStream_t s) { return launch_zd<true>(h, z, s); }
