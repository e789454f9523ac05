// FP32 z pass of the matvec (Section IV-A) with the 12 x 12 Green block product fused
// between the forward and inverse z transforms, on the spectrum left by xy_fwd_kernel: the
// N block from its 60 tensors, or (KOP) the K block (Eq. 8, 25) from its 30.
#include "block.cuh"
#include "fft2.cuh"
#include "autotune.h"
#include "zpass_f32.cuh"

// ---------------------------------------------------------------------------
// z pass (FP32, on the spectrum of xy_fwd_kernel): a CTA of 128 threads per (row py,
// tile of 4 stored columns = 2 mirror pairs) loops over the right-hand sides, two CTAs
// to an SM so that one's loads and stores overlap the other's arithmetic; the next
// right-hand side's columns arrive by cp.async while the current one is transformed.
// The z spectrum stays in transposed order between the forward and inverse transforms.
// A thread of the block product owns one (column pair, kz mirror pair) item for the
// whole launch: the 60 Green values of its octant point stay in registers and serve
// the four frequency points (+-kx, +-kz) of every right-hand side, one column at a time
// with packed FP32 pair FMAs.  The item that pairs
// kz = 0 with kz = Lz/2 keeps the second point's values in shared memory; the last
// tile's self-mirrored columns 0 and Lx/2 reload theirs for each right-hand side.
// ---------------------------------------------------------------------------
// Tiles of TB stored columns (TB / 2 mirror pairs): 4 or 8 for Lz <= 128, 2 or 4 for Lz = 256,
// 2 for Lz = 512 (the autotuner below picks one per grid).  One thread per (pair, kz item):
// NT = max(TB/2 * Lz/2, 128); two CTAs per SM when NT = 128 and the two buffers fit twice.
template <int LZ, int TB_>
struct ZFCfg {
    static constexpr int TB = TB_;
    static constexpr int NPAIR = TB / 2;
    static constexpr int NT0 = NPAIR * LZ / 2;
    static constexpr int NT = NT0 < 128 ? 128 : NT0;
    static constexpr int GS = LZ * TB + TB;  // component stride: TB float2 of padding keep half-warps apart
    static constexpr int BUF = 12 * GS;
    static constexpr size_t smem = sizeof(float2) * (size_t)(2 * BUF + LZ + 2 * NPAIR * 60);
    static constexpr int MINB = (NT == 128 && smem <= 113 * 1024) ? 2 : 1;
};

// the NG Green values of one octant point, streamed from the [..][NG] layout
template <int NG>
__device__ __forceinline__ void load_green(float2* u, const float2* __restrict__ gp) {
    const float4* g4 = reinterpret_cast<const float4*>(gp);
#pragma unroll
    for (int q = 0; q < NG / 2; ++q) {
        const float4 v = __ldg(g4 + q);
        u[2 * q] = make_float2(v.x, v.y);
        u[2 * q + 1] = make_float2(v.z, v.w);
    }
}

// sign flip of a complex value by XOR of the sign bits: sbit is 0 or 0x80000000
__device__ __forceinline__ float2 xflip(float2 v, unsigned sbit) {
    return make_float2(__uint_as_float(__float_as_uint(v.x) ^ sbit), __uint_as_float(__float_as_uint(v.y) ^ sbit));
}
__device__ __forceinline__ unsigned sign_bit(unsigned mask, int a) { return (mask << (31 - a)) & 0x80000000u; }

// y = B x at one column of one z position with packed FP32 pairs (__ffma2_rn, two FMAs per
// instruction): for each input b, acc1[a] += (x_b.re, x_b.re) u and acc2[a] += (x_b.im, x_b.im) u,
// so that (B x)_a = (acc1.re - acc2.im, acc1.im + acc2.re); the Green values stay in their
// natural (re, im) pairs.  m: components whose sign flips at this reflected frequency point on
// input, mo on output (m for N; for K also all twelve when an odd number of axes is reflected).
// KOP: the 96 non-zero entries of the K block on its 30 values instead of the 144 of N on 60.
template <bool KOP>
__device__ __forceinline__ BlockEntryT block_entry(int i) {
    if constexpr (KOP)
        return kKBlockB.e[i];
    else
        return kBlockB.e[i];
}

template <bool KOP>
__device__ __forceinline__ void col_point2(const float2* u, float2* s, int gs, int off, unsigned m, unsigned mo) {
    float2 xr[12], xi[12], a1[12], a2[12];
#pragma unroll
    for (int b = 0; b < 12; ++b) {
        const float2 v = xflip(s[b * gs + off], sign_bit(m, b));
        xr[b] = make_float2(v.x, v.x);
        xi[b] = make_float2(v.y, v.y);
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) a1[a] = a2[a] = make_float2(0.f, 0.f);
    constexpr int NE = KOP ? 96 : 144;
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        const BlockEntryT en = block_entry<KOP>(i);
        const int a = en.a, b = en.b, t = en.t;
        if (en.s > 0) {
            a1[a] = __ffma2_rn(xr[b], u[t], a1[a]);
            a2[a] = __ffma2_rn(xi[b], u[t], a2[a]);
        } else {
            a1[a] = __ffma2_rn(make_float2(-xr[b].x, -xr[b].y), u[t], a1[a]);
            a2[a] = __ffma2_rn(make_float2(-xi[b].x, -xi[b].y), u[t], a2[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 12; ++a)
        s[a * gs + off] = xflip(make_float2(a1[a].x - a2[a].y, a1[a].y + a2[a].x), sign_bit(mo, a));
}

template <int LZ, int TB_, bool KOP>
__global__ void __launch_bounds__(ZFCfg<LZ, TB_>::NT, ZFCfg<LZ, TB_>::MINB)
    zfused_kernel(ZFArgs z, const float2* __restrict__ twg) {
    using Cfg = ZFCfg<LZ, TB_>;
    constexpr int NG = KOP ? 30 : 60;  // Green values per octant point
    constexpr int A = fft2::Split<LZ>::A, B = fft2::Split<LZ>::B, NT = Cfg::NT, TB = Cfg::TB;
    constexpr int NPAIR = Cfg::NPAIR, GS = Cfg::GS, BUF = Cfg::BUF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sb = reinterpret_cast<float2*>(smem_raw);
    float2* tw = sb + 2 * BUF;
    float2* gsec = tw + LZ;  // [NPAIR pairs][2 sets][NG] Green values of the item that holds kz = LZ/2
    const int tid = threadIdx.x;
    const int R = z.nact ? min(*z.nact, z.R) : z.R;
    dev_bytes_add(z.bctr, 8.0 * (2.0 * R * 12 * z.nz * z.Ly * z.Lx + (double)NG * z.Ox * z.Oy * z.Oz), R > 0);
    if (R <= 0) return;
    for (int m = tid; m < LZ; m += NT) tw[m] = twg[m];
    const int ntile = z.Lx / TB;
    const int py = blockIdx.x / ntile, ct = blockIdx.x % ntile, sc0 = ct * TB;
    const long long plane = (long long)z.Ly * z.Lx;
    const int ky = py / z.by + z.ay * (py % z.by);
    const int kyo = ky <= z.Ly / 2 ? ky : z.Ly - ky;
    const unsigned fy = ky > z.Ly / 2 ? z.my : 0u;
    const int nz = z.nz;
    // K: the block's overall sign flips at points reflected along an odd number of axes
    const unsigned ko = KOP ? 0xFFFu : 0u;
    const bool ry = ky > z.Ly / 2;

    auto issue = [&](int r, float2* buf) {
        const float2* base = z.w + (long long)r * 12 * nz * plane + (long long)py * z.Lx + sc0;
        for (int idx = tid; idx < 12 * nz * (TB / 2); idx += NT) {
            const int q = idx % (TB / 2), l = (idx / (TB / 2)) % nz, a = idx / ((TB / 2) * nz);
            cp_async16(buf + a * GS + l * TB + 2 * q, base + ((long long)a * nz + l) * plane + 2 * q);
        }
        cp_async_commit();
    };
    auto line = [](int n) { return (n / TB) * GS + n % TB; };

    // block-product item of this thread: column pair ci, kz item j
    const int ci = tid % NPAIR, j = tid / NPAIR;
    const bool single = ct == ntile - 1 && ci == NPAIR - 1;  // columns 0 and Lx/2: own octant columns
    const int kx0 = z.colkx[sc0 + 2 * ci], kx1 = z.colkx[sc0 + 2 * ci + 1];
    const unsigned fx0 = kx0 > z.Lx / 2 ? z.mx : 0u, fx1 = kx1 > z.Lx / 2 ? z.mx : 0u;
    const bool rx0 = kx0 > z.Lx / 2, rx1 = kx1 > z.Lx / 2;
    // kz items, in transposed positions p = k2 + B k1 holding kz = k1 + A k2:
    //   rows k1 = 1..A/2-1 with their mirrors in rows A - k1, then row A/2 (its own mirror),
    //   then row 0 (k2 = 0 pairs kz = 0 with kz = LZ/2, each with its own octant point).
    constexpr int NREG = (A / 2 - 1) * B;
    int pa = -1, pb = -1, pc = -1;  // pa, pb share one octant point; pc (kz = LZ/2) has its own
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
    const float2* gcol0 = z.green_t + ((long long)kyo * z.Ox + kxo0) * z.Oz * NG;
    const float2* gcol1 = z.green_t + ((long long)kyo * z.Ox + kxo1) * z.Oz * NG;
    // the item's frequency points: up to two sharing one octant point (pa, pb), and pc
    // (kz = LZ/2) with its own; its Green values go to shared memory, next to a copy of
    // the first set, so that one register array serves all points of every item
    const int kza = pa >= 0 ? fft2::freq_at(LZ, pa) : 0;
    const int kzoa = kza <= LZ / 2 ? kza : LZ - kza;
    float2 u[NG];
    if (pa >= 0 && !single) {
        load_green<NG>(u, gcol0 + (long long)kzoa * NG);
        if (pc >= 0)
#pragma unroll
            for (int t = 0; t < NG; ++t) {
                gsec[(2 * ci) * NG + t] = u[t];
                gsec[(2 * ci + 1) * NG + t] = gcol0[(long long)(LZ / 2) * NG + t];
            }
    }

    issue(0, sb);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        float2* s = sb + (r & 1) * BUF;
        if (r + 1 < R) {
            issue(r + 1, sb + ((r + 1) & 1) * BUF);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        fft2::forward<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
        if (pa >= 0) {
            // points (position, Green set): (pa, 0), (pb, 0), (pc, 1); single columns take
            // each column in turn with its own Green values, loaded from global memory
#pragma unroll 1
            for (int q = 0; q < (single ? 6 : 3); ++q) {
                const int e = single ? q % 3 : q, col = single ? q / 3 : 0;
                const int pp = e == 0 ? pa : (e == 1 ? pb : pc);
                if (pp < 0) continue;
                const int kz = fft2::freq_at(LZ, pp);
                if (single) {
                    const int kzo = kz <= LZ / 2 ? kz : LZ - kz;
                    load_green<NG>(u, (col ? gcol1 : gcol0) + (long long)kzo * NG);
                } else if (e == 2) {
#pragma unroll
                    for (int t = 0; t < NG; ++t) u[t] = gsec[(2 * ci + 1) * NG + t];
                }
                const bool rz = kz > LZ / 2;
                const unsigned fz = rz ? z.mz : 0u;
                const unsigned m0 = fy ^ fz ^ fx0, m1 = fy ^ fz ^ fx1;
                if (!single || col == 0)
                    col_point2<KOP>(u, s, GS, pp * TB + 2 * ci, m0, (ry ^ rz ^ rx0) ? m0 ^ ko : m0);
                if (!single || col == 1)
                    col_point2<KOP>(u, s, GS, pp * TB + 2 * ci + 1, m1, (ry ^ rz ^ rx1) ? m1 ^ ko : m1);
            }
            if (pc >= 0 && !single) {
#pragma unroll
                for (int t = 0; t < NG; ++t) u[t] = gsec[(2 * ci) * NG + t];
            }
        }
        __syncthreads();
        fft2::inverse<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
        float2* base = z.w + (long long)r * 12 * nz * plane + (long long)py * z.Lx + sc0;
        for (int idx = tid; idx < 12 * nz * (TB / 2); idx += NT) {
            const int q = idx % (TB / 2), l = (idx / (TB / 2)) % nz, a = idx / ((TB / 2) * nz);
            *reinterpret_cast<float4*>(base + ((long long)a * nz + l) * plane + 2 * q) =
                *reinterpret_cast<const float4*>(s + a * GS + l * TB + 2 * q);
        }
        __syncthreads();
    }
}

template <int LZ, int TB, bool KOP>
static int launch_zf_LT(const vie_handle* h, const ZFArgs& z, cudaStream_t s, const char* name) {
    using Cfg = ZFCfg<LZ, TB>;
    constexpr size_t smem = Cfg::smem;
    constexpr double NG = KOP ? 30.0 : 60.0;
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(zfused_kernel<LZ, TB, KOP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    const long long blocks = (long long)z.Ly * (z.Lx / TB);
    // with a device count the kernel adds its bytes to z.bctr
    const double bytes = z.nact ? kDevCounted : 8.0 * (2.0 * z.R * 12 * z.nz * z.Ly * z.Lx + NG * z.Ox * z.Oy * z.Oz);
    VIE_KLAUNCH_B(name, s, bytes,
                  zfused_kernel<LZ, TB, KOP><<<(unsigned)blocks, Cfg::NT, smem, s>>>(z, h->tw32 + LZ));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

// tile widths the kernel is built for at each Lz (the first is the default)
static int zf_candidates(int Lz, int Lx, int* tb) {
    int n = 0;
    if (Lz <= 128) {
        tb[n++] = 4;
        if (Lx >= 8) tb[n++] = 8;
    } else if (Lz == 256) {
        tb[n++] = 2;
        tb[n++] = 4;
    } else {
        tb[n++] = 2;
    }
    return n;
}

template <int L, bool KOP>
static int launch_zf_L(const vie_handle* h, const ZFArgs& z, cudaStream_t s, int tb, const char* name) {
    if constexpr (L >= 256)
        if (tb == 2) return launch_zf_LT<L, 2, KOP>(h, z, s, name);
    if constexpr (L <= 256)
        if (tb == 4) return launch_zf_LT<L, 4, KOP>(h, z, s, name);
    if constexpr (L <= 128)
        if (tb == 8) return launch_zf_LT<L, 8, KOP>(h, z, s, name);
    set_error("z pass: unsupported tile width");
    return VIE_EINVAL;
}

template <bool KOP>
static int launch_zf(const vie_handle* h, const ZFArgs& z, cudaStream_t s, int tb, const char* name) {
    switch (h->L[2]) {
        case 8: return launch_zf_L<8, KOP>(h, z, s, tb, name);
        case 16: return launch_zf_L<16, KOP>(h, z, s, tb, name);
        case 32: return launch_zf_L<32, KOP>(h, z, s, tb, name);
        case 64: return launch_zf_L<64, KOP>(h, z, s, tb, name);
        case 128: return launch_zf_L<128, KOP>(h, z, s, tb, name);
        case 256: return launch_zf_L<256, KOP>(h, z, s, tb, name);
        case 512: return launch_zf_L<512, KOP>(h, z, s, tb, name);
    }
    set_error("z pass: unsupported length");
    return VIE_EINVAL;
}

// the tile width for this launch (measured on first use of the shape, see autotune.h)
template <bool KOP>
static int zf_pick(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    int tb[4];
    const int n = zf_candidates(h->L[2], z.Lx, tb);
    const int key[5] = {KOP ? 2 : 0, h->L[2], z.Lx, z.Ly, z.nz};
    const int pick = autotune_pick(key, n, s, [&](int c, cudaStream_t ts, const ZFArgs& zt) {
        return launch_zf<KOP>(h, zt, ts, tb[c], KOP ? "autotune_zpass_k_f32" : "autotune_zpass_f32");
    }, z, [&](int c) { return "TB=" + std::to_string(tb[c]); });
    return tb[pick];
}

int zpass_f32_fused(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    return launch_zf<false>(h, z, s, zf_pick<false>(h, z, s), "zpass_block_f32");
}

int zpass_f32_tune(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    zf_pick<false>(h, z, s);
    return VIE_OK;
}

int zpass_f32_fused_k(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    return launch_zf<true>(h, z, s, zf_pick<true>(h, z, s), "zpass_block_k_f32");
}

int zpass_f32_tune_k(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    zf_pick<true>(h, z, s);
    return VIE_OK;
}
