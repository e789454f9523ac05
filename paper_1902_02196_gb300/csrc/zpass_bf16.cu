// BF16x3 z pass of the matvec (Section IV-A): the same fused z transform -> 12 x 12 Green block
// product -> inverse z transform as the FP32 kernel, with the block product on the tensor cores.
//
// Each frequency point multiplies its 12 complex inputs by a 12 x 12 complex block.  Written
// over reals, y^T = x^T B^T with x^T a row of 24 reals (re, im of the 12 inputs) and B^T the
// 24 x 24 real form of the block ([Br -Bi; Bi Br] in the (re, im) interleaving).  Points that
// share one octant Green block (the mirror pair of columns kx, Lx - kx and the kz mirror pair,
// their reflection signs applied to inputs and outputs) and several right-hand sides form the
// 16 rows of an mma.sync m16n8k16 tile: M = 4 points x 4 right-hand sides, K = 24 (padded to
// 32), N = 24.  Operands are split into bf16 pairs, v = v_hi + v_lo (v_hi = bf16(v),
// v_lo = bf16(v - v_hi), together 16 significant bits), and the product keeps three of the four
// partial products, x_lo B_hi + x_hi B_lo + x_hi B_hi, accumulated in FP32 (18 MMAs per tile).
// The dropped x_lo B_lo and the two splits' residuals bound the relative error of each real
// product by 3 * 2^-16.
//
// A CTA owns one ky row and one mirror pair of stored columns, and loops over groups of four
// right-hand sides (two for Lz = 512): 8 column lines per component in shared memory, slot
// 2 rr + c for right-hand side rr of the group and column c.  Tile row r holds slot r % TB at
// the item's first kz position (r < TB) or second (r >= TB).  The component stride is 4 mod 16
// float2, so the fragment loads and stores of a half warp (4 slots x 4 components) hit 32
// distinct banks.  The Green tensor is read as precomputed bf16 hi/lo pairs ([Oy][Ox][Oz][60]
// of (hi, lo), each a bf16 (re, im) pair).
#include <cuda_bf16.h>

#include "block.cuh"
#include "fft2.cuh"
#include "autotune.h"
#include "zpass_f32.cuh"

namespace {

template <int LZ, int TB_>
struct ZBCfg {
    static constexpr int TB = TB_;  // column lines per component: 2 columns x TB/2 right-hand sides (8 or 4)
    static constexpr int RG = TB / 2;             // right-hand sides per group
    static constexpr int NT = 256;
    static constexpr int GS = LZ * TB + 4;  // component stride in float2, 4 mod 16
    static constexpr size_t smem = sizeof(float2) * (size_t)(12 * GS + LZ);
    static constexpr int MINB = smem <= 110 * 1024 ? 2 : 1;
};

__device__ __forceinline__ unsigned sbit(unsigned mask, int a) { return (mask << (31 - a)) & 0x80000000u; }

__device__ __forceinline__ float2 flip2(float2 v, unsigned s) {
    return make_float2(__uint_as_float(__float_as_uint(v.x) ^ s), __uint_as_float(__float_as_uint(v.y) ^ s));
}

// v = hi + lo as bf16 pairs (low half = v.x, high half = v.y)
__device__ __forceinline__ void split2(float2 v, unsigned& hi, unsigned& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    hi = *reinterpret_cast<const unsigned*>(&h);
    lo = *reinterpret_cast<const unsigned*>(&l);
}

// d += a b, m16n8k16, bf16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int LZ, int TB_>
__global__ void __launch_bounds__(256, ZBCfg<LZ, TB_>::MINB)
    zbf16_kernel(ZFArgs z, const uint2* __restrict__ gbf, const float2* __restrict__ twg) {
    using Cfg = ZBCfg<LZ, TB_>;
    constexpr int A = fft2::Split<LZ>::A, B = fft2::Split<LZ>::B, NT = Cfg::NT, TB = Cfg::TB, RG = Cfg::RG;
    constexpr int GS = Cfg::GS;
    constexpr int NWARP = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    float2* tw = s + 12 * GS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = z.nact ? min(*z.nact, z.R) : z.R;
    dev_bytes_add(z.bctr, 8.0 * (2.0 * R * 12 * z.nz * z.Ly * z.Lx + 60.0 * z.Ox * z.Oy * z.Oz), R > 0);
    if (R <= 0) return;
    for (int m = tid; m < LZ; m += NT) tw[m] = twg[m];
    const int npair = z.Lx / 2;
    const int py = blockIdx.x / npair, cp = blockIdx.x % npair, sc0 = 2 * cp;
    const long long plane = (long long)z.Ly * z.Lx;
    const int ky = py / z.by + z.ay * (py % z.by);
    const int kyo = ky <= z.Ly / 2 ? ky : z.Ly - ky;
    const unsigned fy = ky > z.Ly / 2 ? z.my : 0u;
    const int nz = z.nz;
    const int kx0 = z.colkx[sc0], kx1 = z.colkx[sc0 + 1];
    const int kxo0 = kx0 <= z.Lx / 2 ? kx0 : z.Lx - kx0, kxo1 = kx1 <= z.Lx / 2 ? kx1 : z.Lx - kx1;
    const unsigned fx0 = kx0 > z.Lx / 2 ? z.mx : 0u, fx1 = kx1 > z.Lx / 2 ? z.mx : 0u;
    const bool xsplit = kxo0 != kxo1;  // the pair (0, Lx/2): two octant columns

    // this lane's place in the fragments: groupID g (tile rows g, g + 8; B column g), q = lane % 4
    const int q = lane & 3, g = lane >> 2;
    // B^T entries of the lane: for n-tile nt the output (4 nt + g/2, re or im as g is even or odd);
    // inputs b = q, q + 4 (k-tile 0) and 8 + q (k-tile 1).  Tensor index and the bits to flip
    // after the optional (re, im) swap: the table sign on both halves, -Bi for a real output
    int tix[9];
    unsigned flp[9];
    const bool swp = (g & 1) != 0;
#pragma unroll
    for (int nt = 0; nt < 3; ++nt)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = 4 * nt + (g >> 1), b = e == 0 ? q : (e == 1 ? q + 4 : 8 + q);
            tix[3 * nt + e] = tensor_of(a, b);
            flp[3 * nt + e] = (swp ? 0u : 0x80000000u) ^ (sign_of(a, b) < 0 ? 0x80008000u : 0u);
        }
    // tile rows of the lane: r0 = g and r1 = g + 8 (valid when r1 < 2 TB)
    const bool r1ok = g + 8 < 2 * TB;
    const int slot0 = g % TB, slot1 = (g + 8) % TB;
    const bool second0 = g >= TB, second1 = true;  // r1 = g + 8 >= TB for TB <= 8
    const int c0 = slot0 & 1, c1 = slot1 & 1;

    auto line = [](int n) { return (n / TB) * GS + n % TB; };
#pragma unroll 1
    for (int rb = 0; rb < R; rb += RG) {
        // loads: slot pair (2 rr, 2 rr + 1) of component a, plane l = 16 contiguous bytes
        for (int idx = tid; idx < 12 * nz * RG; idx += NT) {
            const int rr = idx % RG, l = (idx / RG) % nz, a = idx / (RG * nz);
            const bool in = rb + rr < R;
            const float2* src = in ? z.w + ((long long)(rb + rr) * 12 * nz + (long long)a * nz + l) * plane +
                                         (long long)py * z.Lx + sc0
                                   : z.w;
            cp_async16z(s + a * GS + l * TB + 2 * rr, src, in ? 16 : 0);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        fft2::forward<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
#pragma unroll 1
        for (int j = warp; j < LZ / 2; j += NWARP) {
            // kz positions of item j (as in the FP32 kernel): pa with its mirror pb, or, for
            // the item of kz = 0, the self-mirrored kz = LZ/2 at pc with its own octant point
            constexpr int NREG = (A / 2 - 1) * B;
            int pa, p1;
            bool zsplit = false;
            if (j < NREG) {
                const int k1 = 1 + j / B, k2 = j % B;
                pa = k2 + B * k1;
                p1 = (B - 1 - k2) + B * (A - k1);
            } else if (j < NREG + B / 2) {
                const int k2 = j - NREG;
                pa = k2 + B * (A / 2);
                p1 = (B - 1 - k2) + B * (A / 2);
            } else {
                const int k2 = j - NREG - B / 2;
                pa = k2;
                p1 = k2 == 0 ? B / 2 : B - k2;
                zsplit = k2 == 0;
            }
            const int kza = fft2::freq_at(LZ, pa), kzb = fft2::freq_at(LZ, p1);
            const int kzoa = kza <= LZ / 2 ? kza : LZ - kza, kzob = kzb <= LZ / 2 ? kzb : LZ - kzb;
            const unsigned fza = kza > LZ / 2 ? z.mz : 0u, fzb = kzb > LZ / 2 ? z.mz : 0u;
            // the lane's rows: position, reflection mask, Green group (octant point)
            const int pos0 = second0 ? p1 : pa, pos1 = p1;
            const unsigned m0 = fy ^ (c0 ? fx1 : fx0) ^ (second0 ? fzb : fza);
            const unsigned m1 = fy ^ (c1 ? fx1 : fx0) ^ fzb;
            const int grp0 = (zsplit && second0 ? 1 : 0) + (xsplit && c0 ? 2 : 0);
            const int grp1 = (zsplit && second1 ? 1 : 0) + (xsplit && c1 ? 2 : 0);
            // A fragments: x^T rows r0, r1, inputs (re, im) of components q, q + 4 (k-tile 0) and 8 + q (k-tile 1)
            unsigned ah[2][4], al[2][4];
            {
                const float2* x0 = s + pos0 * TB + slot0;
                const float2* x1 = s + pos1 * TB + slot1;
                const int comp[3] = {q, q + 4, 8 + q};
                unsigned h[2][3], l[2][3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const int b = comp[e];
                    split2(flip2(x0[b * GS], sbit(m0, b)), h[0][e], l[0][e]);
                    if (r1ok)
                        split2(flip2(x1[b * GS], sbit(m1, b)), h[1][e], l[1][e]);
                    else
                        h[1][e] = l[1][e] = 0u;
                }
                // k-tile 0: a0 (r0, q), a1 (r1, q), a2 (r0, q + 4), a3 (r1, q + 4); k-tile 1: (., 8 + q), zero
                ah[0][0] = h[0][0], ah[0][1] = h[1][0], ah[0][2] = h[0][1], ah[0][3] = h[1][1];
                al[0][0] = l[0][0], al[0][1] = l[1][0], al[0][2] = l[0][1], al[0][3] = l[1][1];
                ah[1][0] = h[0][2], ah[1][1] = h[1][2], ah[1][2] = 0u, ah[1][3] = 0u;
                al[1][0] = l[0][2], al[1][1] = l[1][2], al[1][2] = 0u, al[1][3] = 0u;
            }
            const int ngrp = (zsplit ? 2 : 1) * (xsplit ? 2 : 1);
#pragma unroll 1
            for (int gi = 0; gi < 4; ++gi) {
                if (!((gi & 1) ? zsplit : true) || !((gi & 2) ? xsplit : true)) continue;
                const int kxo = (gi & 2) ? kxo1 : kxo0, kzo = (gi & 1) ? kzob : kzoa;
                const uint2* gp = gbf + (((long long)kyo * z.Ox + kxo) * z.Oz + kzo) * 60;
                unsigned bh[9], bl[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    const uint2 v = __ldg(gp + tix[e]);
                    const unsigned vh = swp ? __byte_perm(v.x, 0, 0x1032) : v.x;
                    const unsigned vl = swp ? __byte_perm(v.y, 0, 0x1032) : v.y;
                    bh[e] = vh ^ flp[e];
                    bl[e] = vl ^ flp[e];
                }
                float d[3][4];
#pragma unroll
                for (int nt = 0; nt < 3; ++nt) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) d[nt][i] = 0.f;
                    // small partial products first
                    mma_bf16(d[nt], al[0], bh[3 * nt], bh[3 * nt + 1]);
                    mma_bf16(d[nt], al[1], bh[3 * nt + 2], 0u);
                    mma_bf16(d[nt], ah[0], bl[3 * nt], bl[3 * nt + 1]);
                    mma_bf16(d[nt], ah[1], bl[3 * nt + 2], 0u);
                    mma_bf16(d[nt], ah[0], bh[3 * nt], bh[3 * nt + 1]);
                    mma_bf16(d[nt], ah[1], bh[3 * nt + 2], 0u);
                }
                // D rows r0 (d[.][0..1]) and r1 (d[.][2..3]): output component 4 nt + q, (re, im)
                if (ngrp == 1 || grp0 == gi) {
#pragma unroll
                    for (int nt = 0; nt < 3; ++nt) {
                        const int a = 4 * nt + q;
                        s[a * GS + pos0 * TB + slot0] = flip2(make_float2(d[nt][0], d[nt][1]), sbit(m0, a));
                    }
                }
                if (r1ok && (ngrp == 1 || grp1 == gi)) {
#pragma unroll
                    for (int nt = 0; nt < 3; ++nt) {
                        const int a = 4 * nt + q;
                        s[a * GS + pos1 * TB + slot1] = flip2(make_float2(d[nt][2], d[nt][3]), sbit(m1, a));
                    }
                }
            }
        }
        __syncthreads();
        fft2::inverse<LZ, NT>(s, 12 * TB, line, TB, tw, nz);
        for (int idx = tid; idx < 12 * nz * RG; idx += NT) {
            const int rr = idx % RG, l = (idx / RG) % nz, a = idx / (RG * nz);
            if (rb + rr >= R) continue;
            float2* dst = z.w + ((long long)(rb + rr) * 12 * nz + (long long)a * nz + l) * plane + (long long)py * z.Lx + sc0;
            *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(s + a * GS + l * TB + 2 * rr);
        }
        __syncthreads();
    }
}

template <int LZ, int TB>
int launch_zb_LT(const vie_handle* h, const ZFArgs& z, cudaStream_t s, const char* name) {
    using Cfg = ZBCfg<LZ, TB>;
    constexpr size_t smem = Cfg::smem;
    VIE_CUDA(cudaFuncSetAttribute(zbf16_kernel<LZ, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long blocks = (long long)z.Ly * (z.Lx / 2);
    const double bytes = z.nact ? kDevCounted : 8.0 * (2.0 * z.R * 12 * z.nz * z.Ly * z.Lx + 60.0 * z.Ox * z.Oy * z.Oz);
    VIE_KLAUNCH_B(name, s, bytes,
                  zbf16_kernel<LZ, TB><<<(unsigned)blocks, Cfg::NT, smem, s>>>(z, h->greenbf, h->tw32 + LZ));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

int launch_zb(const vie_handle* h, const ZFArgs& z, cudaStream_t s, int tb, const char* name) {
#define VIE_ZB(L)                                              \
    case L:                                                    \
        if (tb == 8) return launch_zb_LT<L, 8>(h, z, s, name); \
        if (tb == 4) return launch_zb_LT<L, 4>(h, z, s, name); \
        break;
    switch (h->L[2]) {
        VIE_ZB(8)
        VIE_ZB(16)
        VIE_ZB(32)
        VIE_ZB(64)
        VIE_ZB(128)
        VIE_ZB(256)
        case 512:
            if (tb == 4) return launch_zb_LT<512, 4>(h, z, s, name);
            break;
    }
#undef VIE_ZB
    set_error("z pass: unsupported length or tile width");
    return VIE_EINVAL;
}

// bf16 (hi, lo) pairs of the FP32 octant tensors in the [Oy][Ox][Oz][60] layout
__global__ void split_green_kernel(const float2* __restrict__ g32t, uint2* __restrict__ gbf, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned hi, lo;
    split2(g32t[i], hi, lo);
    gbf[i] = make_uint2(hi, lo);
}

}  // namespace

int green_split_bf16(vie_handle* h) {
    const long long n = 60LL * h->O[0] * h->O[1] * h->O[2];
    VIE_KLAUNCH("green_split_bf16", h->stream,
                split_green_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->green32t, h->greenbf, n));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

// tile rows: 4 right-hand sides x 2 columns x 2 kz positions (TB = 8), or 2 x 2 x 2 in half a tile
// (TB = 4); the width for this launch is measured on first use of the shape (autotune.h)
static int zb_pick(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    int tb[2], n = 0;
    if (h->L[2] <= 256) tb[n++] = 8;
    tb[n++] = 4;
    const int key[5] = {1, h->L[2], z.Lx, z.Ly, z.nz};
    const int pick = autotune_pick(key, n, s, [&](int c, cudaStream_t ts, const ZFArgs& zt) {
        return launch_zb(h, zt, ts, tb[c], "autotune_zpass_bf16x3");
    }, z, [&](int c) { return "TB=" + std::to_string(tb[c]); });
    return tb[pick];
}

int zpass_bf16_fused(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    if (!h->greenbf) {
        set_error("internal: no bf16 Green tensors");
        return VIE_EINVAL;
    }
    return launch_zb(h, z, s, zb_pick(h, z, s), "zpass_block_bf16x3");
}

int zpass_bf16_tune(const vie_handle* h, const ZFArgs& z, cudaStream_t s) {
    zb_pick(h, z, s);
    return VIE_OK;
}
