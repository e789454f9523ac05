// FFT-accelerated matvec of the PWL current-based VIE (Section IV-A).
//
// y = op(x) for R right-hand sides at once.  The Toeplitz structure of the
// Galerkin matrix (Eq. 42-43) is embedded in a circulant of length L_i >= 2 N_i - 1
// per axis; the product is computed as
//   x-pass : zero-pad along x, forward FFT          x[R*12][Nz][Ny][Nx] -> W1[R*12][Nz][Ny][Lx]
//   y-pass : zero-pad along y, forward FFT          W1 -> W2[R*12][Nz][Ly][Lx]
//   z-pass : per (kx, ky) column and right-hand side: zero-pad along z, forward
//            FFT, 12 x 12 block product with the Green tensor at every kz,
//            inverse FFT, keep the first Nz planes           W2 -> W2 (in place)
//   y-inv  : inverse FFT along y, keep Ny                    W2 -> W1
//   x-inv  : inverse FFT along x, keep Nx, then the material and Gram terms
//            (op A: G x - chi (N - G) x;  op PA: x/eps - tau G^-1 (N - G) x)  W1 -> y
// The 1/(Lx Ly Lz) normalisation is folded into the stored Green tensor.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "block.cuh"
#include "fft.cuh"
#include "fft2.cuh"
#include "line2.cuh"
#include "zpass_f32.cuh"
#include "zpass_f64.cuh"

int zpass_bf16_fused(const vie_handle* h, const ZFArgs& z, cudaStream_t s);  // zpass_bf16.cu
int zpass_bf16_tune(const vie_handle* h, const ZFArgs& z, cudaStream_t s);   // zpass_bf16.cu

// y[3] = B(k) x[3] of the PWC system (the l = 1 sub-block): entry (p, q) is tensor 10 pq + 0
// (scalar pair (1, 1)) with sign +1
template <typename C>
__device__ __forceinline__ void block_product_pwc(C* xv, C* acc, const C* __restrict__ gp, long long tstride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = mk(decltype(xv[0].x)(0), decltype(xv[0].x)(0));
#pragma unroll
        for (int b = 0; b < 3; ++b) cfma(acc[a], gp[10 * pq_index(a, b) * tstride], xv[b]);
    }
}

// y[12] = B(k) x[12] at one frequency point; xv/acc in registers, Green values streamed once.
template <typename C>
__device__ __forceinline__ void block_product(C* xv, C* acc, const C* __restrict__ gp, long long tstride) {
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = mk(decltype(xv[0].x)(0), decltype(xv[0].x)(0));
#pragma unroll
    for (int t = 0; t < 60; ++t) {
        const C u = gp[t * tstride];
#pragma unroll
        for (int i = kBlock.start[t]; i < kBlock.start[t + 1]; ++i) {
            const int a = kBlock.e[i].a, b = kBlock.e[i].b;
            if (kBlock.e[i].s > 0)
                cfma(acc[a], u, xv[b]);
            else
                cfma(acc[a], cneg(u), xv[b]);
        }
    }
}

// y[12] = K(k) x[12] at one frequency point (VIE_OP_K): the 96 signed entries of the 30 tensors
template <typename C>
__device__ __forceinline__ void block_product_k(C* xv, C* acc, const C* __restrict__ gp, long long tstride) {
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = mk(decltype(xv[0].x)(0), decltype(xv[0].x)(0));
#pragma unroll
    for (int t = 0; t < 30; ++t) {
        const C u = gp[t * tstride];
#pragma unroll
        for (int i = kKBlock.start[t]; i < kKBlock.start[t + 1]; ++i) {
            const int a = kKBlock.e[i].a, b = kKBlock.e[i].b;
            if (kKBlock.e[i].s > 0)
                cfma(acc[a], u, xv[b]);
            else
                cfma(acc[a], cneg(u), xv[b]);
        }
    }
}

template <typename T, int L, int NC = 12>
struct ZCfg {
    static constexpr int TB0 = (sizeof(T) == 4 ? 1024 : 512) / L;
    static constexpr int TB = TB0 < 1 ? 1 : TB0;
    static constexpr int GS = L * TB;
    static constexpr int NT = sizeof(T) == 4 ? 512 : 256;
};

struct ZArgs {
    void* w;          // W2 [R*12][Nz][Ly][Lx], in place
    const void* green;
    int R, nz, Lx, Ly;
    int Ox, Oy, Oz;
    long long tstride;
    unsigned mx, my, mz;  // reflection flip masks per axis
    // spectrum of the xy kernels: row py holds ky = py / by + ay * (py % by) and stored column sc
    // holds kx = colkx[sc]; by = 0 and colkx = NULL for natural order
    const int* colkx;
    int ay, by;
};

// KOP: the K block (Eq. 8, 25) instead of the N block, on the 30 K tensors; a frequency point
// reflected along an odd number of axes also changes the block's overall sign (the curl's parity)
template <typename T, int L, int NC, bool KOP = false>
__global__ void __launch_bounds__(ZCfg<T, L, NC>::NT) zpass_kernel(ZArgs z, const typename CT<T>::C* twg) {
    using C = typename CT<T>::C;
    constexpr int TB = ZCfg<T, L, NC>::TB, GS = ZCfg<T, L, NC>::GS, NT = ZCfg<T, L, NC>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* tw = s + NC * GS;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += NT) tw[m] = twg[m];

    const int ntile = (z.Lx + TB - 1) / TB;
    const int py = blockIdx.x / ntile;
    const int ky = z.by ? py / z.by + z.ay * (py % z.by) : py;
    const int kx0 = (blockIdx.x % ntile) * TB;
    const long long plane = (long long)z.Ly * z.Lx;
    C* w = reinterpret_cast<C*>(z.w);
    const C* green = reinterpret_cast<const C*>(z.green);
    const C zero = mk(T(0), T(0));
    const int Lz = L;
    const int kyo = ky <= z.Ly / 2 ? ky : z.Ly - ky;
    const unsigned fy = ky > z.Ly / 2 ? z.my : 0u;

    for (int r = 0; r < z.R; ++r) {
        C* base = w + (long long)r * NC * z.nz * plane + (long long)py * z.Lx + kx0;
        for (int idx = tid; idx < NC * L * TB; idx += NT) {
            int tb = idx % TB;
            int l = (idx / TB) % L;
            int a = idx / (TB * L);
            C v = zero;
            if (l < z.nz && kx0 + tb < z.Lx) v = base[((long long)a * z.nz + l) * plane + tb];
            s[a * GS + l * TB + tb] = v;
        }
        __syncthreads();
        fft_smem<C, L, NC, TB, TB, GS, NT>(s, tw, -1);
        for (int p = tid; p < L * TB; p += NT) {
            int tb = p % TB;
            int kz = p / TB;
            if (kx0 + tb >= z.Lx) continue;
            const int kx = z.colkx ? z.colkx[kx0 + tb] : kx0 + tb;
            int kxo = kx <= z.Lx / 2 ? kx : z.Lx - kx;
            int kzo = kz <= Lz / 2 ? kz : Lz - kz;
            unsigned mask = fy ^ (kx > z.Lx / 2 ? z.mx : 0u) ^ (kz > Lz / 2 ? z.mz : 0u);
            unsigned omask = mask;  // output flips
            if (KOP && (((ky > z.Ly / 2) + (kx > z.Lx / 2) + (kz > Lz / 2)) & 1)) omask ^= 0xFFFu;
            C xv[NC], acc[NC];
#pragma unroll
            for (int b = 0; b < NC; ++b) {
                C v = s[b * GS + kz * TB + tb];
                xv[b] = ((mask >> b) & 1u) ? cneg(v) : v;
            }
            const C* gp = green + ((long long)kzo * z.Oy + kyo) * z.Ox + kxo;
            if constexpr (KOP)
                block_product_k(xv, acc, gp, z.tstride);
            else if constexpr (NC == 12)
                block_product(xv, acc, gp, z.tstride);
            else
                block_product_pwc(xv, acc, gp, z.tstride);
#pragma unroll
            for (int a = 0; a < NC; ++a) s[a * GS + kz * TB + tb] = ((omask >> a) & 1u) ? cneg(acc[a]) : acc[a];
        }
        __syncthreads();
        fft_smem<C, L, NC, TB, TB, GS, NT>(s, tw, +1);
        for (int idx = tid; idx < NC * z.nz * TB; idx += NT) {
            int tb = idx % TB;
            int l = (idx / TB) % z.nz;
            int a = idx / (TB * z.nz);
            if (kx0 + tb < z.Lx) base[((long long)a * z.nz + l) * plane + tb] = s[a * GS + l * TB + tb];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP32 three-kernel path (Lx = Ly = L and Lz in 8..128): two-pass FFTs (fft2.cuh)
// whose spectra stay in "transposed" order, so every element makes two round trips
// through shared memory per 1-D transform.
//
// Spectrum layout W2 [R*12][Nz][Ly][Lx]: row py holds ky = freq_at(Ly, py); stored
// column sc holds kx = colkx[sc].  The column order (built on the host) keeps mirror
// pairs (kx, Lx - kx) side by side, 4 pairs to an 8-column tile, with the self-mirrored
// columns 0 and Lx/2 in the last two slots; within every 16 stored columns the
// positions of the x transform differ modulo 16, which keeps the column gathers
// and scatters of the xy kernels free of shared-memory bank conflicts.
// ---------------------------------------------------------------------------
constexpr int kXYThreads = 256;

template <int L, typename C>
struct XYCfg {
    static constexpr int H = L / 2;   // rows that are non-zero before / needed after the y transform
    static constexpr int RS = L + 1;  // odd row stride of the x-transform buffer
    static constexpr int CW0 = sizeof(C) == 8 ? 32 : 16;
    static constexpr int CW = L < CW0 ? L : CW0;  // stored columns per y-transform chunk
    static constexpr int EPV = 16 / (int)sizeof(C);  // elements per 16-byte vector
    static constexpr int MINB = sizeof(C) == 8 ? 2 : 1;  // CTAs per SM
    static constexpr size_t smem = sizeof(C) * (size_t)(L * CW + H * RS + L) + sizeof(int4) * H + L;
};

// Forward: plane (r, alpha, z) of x -> W2 plane [Ly][Lx] (transposed ky, stored kx).  x is
// [R][12][Nz][Ny][Nx], or [R][12][ns] on a support (rows != NULL; zeros outside it).
template <int L, typename C>
__global__ void __launch_bounds__(kXYThreads, XYCfg<L, C>::MINB)
    xy_fwd_kernel(const C* __restrict__ x, C* __restrict__ w, int nx, int ny, int nz, const int4* __restrict__ rows,
                  long long ns, const unsigned char* __restrict__ cpos, const C* __restrict__ twg,
                  const int* __restrict__ rmap, MatvecEpi dc) {
    using Cfg = XYCfg<L, C>;
    constexpr int A = fft2::Split<L>::A, B = fft2::Split<L>::B, NT = kXYThreads, RS = Cfg::RS, CW = Cfg::CW;
    constexpr int EPV = Cfg::EPV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* ck = reinterpret_cast<C*>(smem_raw);  // [L][CW] chunk of stored columns
    C* xr = ck + L * CW;                     // [H][RS] rows after the x transform
    C* tw = xr + Cfg::H * RS;
    int4* rw = reinterpret_cast<int4*>(tw + L);  // [H] support rows of this plane
    unsigned char* pos = reinterpret_cast<unsigned char*>(rw + Cfg::H);
    const int tid = threadIdx.x;
    const long long p = blockIdx.x;  // spectrum plane; the input plane is pin (rmap: active right-hand sides)
    const long long rplanes = (long long)dc.nc * nz;  // planes per right-hand side
    if (dc.nact) {  // planes of right-hand sides beyond the device count are skipped
        const int cnt = *dc.nact;
        dev_bytes_add(dc.bctr, dc.bfix + dc.bper * cnt, cnt > 0);
        if (p / rplanes >= cnt) return;
    }
    for (int m = tid; m < L; m += NT) {
        tw[m] = twg[m];
        pos[m] = cpos[m];
    }
    const long long pin = rmap ? (long long)rmap[p / rplanes] * rplanes + p % rplanes : p;
    if (rows) {
        const int z = (int)(p % nz);
        for (int yy = tid; yy < ny; yy += NT) rw[yy] = rows[(long long)z * ny + yy];
        __syncthreads();
        const C* src = x + (pin / nz) * ns;
        for (int idx = tid; idx < ny * nx; idx += NT) {
            const int yy = idx / nx, xx = idx % nx;
            const int4 q = rw[yy];
            const bool in = xx >= q.x && xx < q.y;
            cp_async_elem(xr + yy * RS + xx, in ? src + q.z + (xx - q.x) : src, in);
        }
    } else {
        const C* src = x + pin * (long long)ny * nx;
        for (int idx = tid; idx < ny * nx; idx += NT) cp_async_elem(xr + (idx / nx) * RS + idx % nx, src + idx, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    fft2::forward<L, NT>(xr, ny, [](int n) { return n * RS; }, 1, tw, nx);
    C* dst = w + p * (long long)L * L;
#pragma unroll 1
    for (int k = 0; k < L / CW; ++k) {
        // y transform, pass 1: gather stored column k*CW + c from the x-transform rows
        for (int t = tid; t < CW * B; t += NT) {
            const int c = t % CW, b = t / CW;
            const C* col = xr + pos[k * CW + c];
            C v[A];
#pragma unroll
            for (int a = 0; a < A / 2; ++a) {  // ny <= L/2: the upper half is zero
                const int yy = b + B * a;
                v[a] = yy < ny ? col[yy * RS] : C{};
            }
            fft2::dft_half_in<A>(v, -1);
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) ck[(b + B * k1) * CW + c] = v[k1];
        }
        __syncthreads();
        for (int t = tid; t < CW * A; t += NT) {
            const int c = t % CW, k1 = t / CW;
            C* ln = ck + B * k1 * CW + c;
            C v[B];
#pragma unroll
            for (int b = 0; b < B; ++b) v[b] = ln[b * CW];
            fft2::DFT<B, C>::run(v, -1);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) ln[k2 * CW] = v[k2];
        }
        __syncthreads();
        for (int idx = tid; idx < L * CW / EPV; idx += NT) {
            const int q = idx / (CW / EPV), c2 = EPV * (idx % (CW / EPV));
            *reinterpret_cast<float4*>(dst + (long long)q * L + k * CW + c2) =
                *reinterpret_cast<const float4*>(ck + q * CW + c2);
        }
        __syncthreads();
    }
}

// Inverse: W2 plane -> y plane [Ny][Nx] with the material / Gram / preconditioner epilogue;
// CONV: also the plane's (N - G) x at every voxel to epi.conv (full grid).
template <int L, typename C, bool CONV>
__global__ void __launch_bounds__(kXYThreads, XYCfg<L, C>::MINB)
    xy_inv_kernel(const C* __restrict__ w, C* __restrict__ y, MatvecEpi epi, const unsigned char* __restrict__ cpos,
                  const C* __restrict__ twg) {
    using Cfg = XYCfg<L, C>;
    using R = decltype(C{}.x);
    constexpr int A = fft2::Split<L>::A, B = fft2::Split<L>::B, NT = kXYThreads, RS = Cfg::RS, CW = Cfg::CW;
    constexpr int EPV = Cfg::EPV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* ck = reinterpret_cast<C*>(smem_raw);
    C* xr = ck + L * CW;
    C* tw = xr + Cfg::H * RS;
    int4* rw = reinterpret_cast<int4*>(tw + L);
    unsigned char* pos = reinterpret_cast<unsigned char*>(rw + Cfg::H);
    const int tid = threadIdx.x;
    const int nx = epi.nx, ny = epi.ny, nz = epi.nz;
    const long long p = blockIdx.x;  // spectrum plane (r * nc + alpha) * nz + z; output plane po
    const int nc = epi.nc;
    const long long rplanes = (long long)nc * nz;  // planes per right-hand side
    if (epi.nact) {
        const int cnt = *epi.nact;
        dev_bytes_add(epi.bctr, epi.bfix + epi.bper * cnt, cnt > 0);
        if (p / rplanes >= cnt) return;
    }
    for (int m = tid; m < L; m += NT) {
        tw[m] = twg[m];
        pos[m] = cpos[m];
    }
    const long long po = epi.rmap ? (long long)epi.rmap[p / rplanes] * rplanes + p % rplanes : p;
    if (epi.rows)
        for (int yy = tid; yy < ny; yy += NT) rw[yy] = epi.rows[(p % nz) * ny + yy];
    const C* src = w + p * (long long)L * L;
#pragma unroll 1
    for (int k = 0; k < L / CW; ++k) {
        for (int idx = tid; idx < L * CW / EPV; idx += NT) {
            const int q = idx / (CW / EPV), c2 = EPV * (idx % (CW / EPV));
            cp_async16(ck + q * CW + c2, src + (long long)q * L + k * CW + c2);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        // inverse y transform, pass 1 (in place in the chunk)
        for (int t = tid; t < CW * A; t += NT) {
            const int c = t % CW, k1 = t / CW;
            C* ln = ck + B * k1 * CW + c;
            C v[B];
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k2] = ln[k2 * CW];
            fft2::DFT<B, C>::run(v, +1);
#pragma unroll
            for (int b = 1; b < B; ++b) v[b] = cmul(v[b], cconj(tw[b * k1]));
#pragma unroll
            for (int b = 0; b < B; ++b) ln[b * CW] = v[b];
        }
        __syncthreads();
        // pass 2: rows y < Ny scattered to the x-transform buffer at the column's x position
        for (int t = tid; t < CW * B; t += NT) {
            const int c = t % CW, b = t / CW;
            C v[A];
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[k1] = ck[(b + B * k1) * CW + c];
            fft2::dft_half_out<A>(v, +1);
            C* col = xr + pos[k * CW + c];
#pragma unroll
            for (int a = 0; a < A / 2; ++a) {  // ny <= L/2
                const int yy = b + B * a;
                if (yy < ny) col[yy * RS] = v[a];
            }
        }
        __syncthreads();
    }
    const long long base = po * (long long)ny * nx;
    const long long cbase = (po / nz) * epi.ns;  // component block on the support
    const C* xin = reinterpret_cast<const C*>(epi.x);
    // the epilogue's x values of this plane arrive in the free chunk buffer during the x transform
    const bool pre = epi.op != VIE_OP_NSCAT && L * CW >= ny * nx;
    if (pre) {
        for (int idx = tid; idx < ny * nx; idx += NT) {
            const int yy = idx / nx, xx = idx % nx;
            long long o = base + idx;
            bool in = true;
            if (epi.rows) {
                const int4 q = rw[yy];
                in = xx >= q.x && xx < q.y;
                o = in ? cbase + q.z + (xx - q.x) : cbase;
            }
            cp_async_elem(ck + idx, xin + o, in);
        }
        cp_async_commit();
    }
    fft2::inverse<L, NT>(xr, ny, [](int n) { return n * RS; }, 1, tw, nx);
    if (pre) {
        cp_async_wait<0>();
        __syncthreads();
    }
    const int alpha = (int)((p / nz) % nc);
    const long long zoff = (p % nz) * (long long)ny * nx;
    const R gl = (R)(comp_is_constant(alpha, nc) ? epi.g1 : epi.g234);
    const R ig = (R)1 / gl;
    const C* c1 = reinterpret_cast<const C*>(epi.c1);
    const C* c2 = reinterpret_cast<const C*>(epi.c2);
    C sh = mk((R)0, (R)0);  // shift of op PA for this plane's right-hand side
    if (epi.shift) {
        const double2 d = epi.shift[po / rplanes];
        sh = mk((R)d.x, (R)d.y);
    }
    C* conv = CONV ? reinterpret_cast<C*>(epi.conv) : nullptr;
#pragma unroll 4
    for (int idx = tid; idx < ny * nx; idx += NT) {
        const int yy = idx / nx, xx = idx % nx;
        long long o = base + idx;
        C v = xr[yy * RS + xx];
        if (CONV) conv[base + idx] = v;  // every voxel of the plane, full-grid layout
        if (epi.rows) {
            const int4 q = rw[yy];
            if (xx < q.x || xx >= q.y) continue;
            o = cbase + q.z + (xx - q.x);
        }
        if (epi.op == VIE_OP_A) {
            const C xv = pre ? ck[idx] : xin[o];
            v = csub(mk(gl * xv.x, gl * xv.y), cmul(c2[zoff + idx], v));
        } else if (epi.op == VIE_OP_PA) {
            const C xv = pre ? ck[idx] : xin[o];
            const C t = cmul(c2[zoff + idx], v);
            v = csub(cmul(csub(c1[zoff + idx], sh), xv), mk(ig * t.x, ig * t.y));
        }
        y[o] = v;
    }
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
template <typename T>
static const typename CT<T>::C* twiddles(const vie_handle* h, int L);
template <>
const float2* twiddles<float>(const vie_handle* h, int L) {
    return h->tw32 + L;
}
template <>
const double2* twiddles<double>(const vie_handle* h, int L) {
    return h->tw64 + L;
}

template <typename T, int L, bool EPI>
static int launch_line_L(const char* name, const vie_handle* h, const LineArgs& a, const MatvecEpi& e,
                         cudaStream_t s) {
    constexpr int TB = LineCfg<L>::TB, NT = LineCfg<L>::NT;
    size_t smem = line_fft_smem_bytes<T, L>();
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(line_fft_kernel<T, L, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    long long blocks = (long long)a.na * ((a.nb + TB - 1) / TB);
    if (blocks <= 0) return VIE_OK;
    if (blocks > 0x7fffffffLL) {
        set_error("line FFT grid too large");
        return VIE_EINVAL;
    }
    // algorithmic bytes: inputs read once, outputs written once (+ x and the coefficient maps in the epilogue)
    double bytes = (double)sizeof(typename CT<T>::C) * (double)a.na * a.nb * (a.n_in + a.n_out);
    if (EPI && e.op != VIE_OP_NSCAT)
        bytes += (double)sizeof(typename CT<T>::C) *
                 ((double)a.na * a.nb * a.n_out + (double)h->nv * (e.op == VIE_OP_PA ? 2 : 1));
    VIE_KLAUNCH_B(name, s, bytes,
                  line_fft_kernel<T, L, EPI><<<(unsigned)blocks, NT, smem, s>>>(a, twiddles<T>(h, L), e));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename T, bool EPI>
static int launch_line(const char* name, const vie_handle* h, int L, const LineArgs& a, const MatvecEpi& e,
                       cudaStream_t s) {
    switch (L) {
        case 2: return launch_line_L<T, 2, EPI>(name, h, a, e, s);
        case 4: return launch_line_L<T, 4, EPI>(name, h, a, e, s);
        case 8: return launch_line_L<T, 8, EPI>(name, h, a, e, s);
        case 16: return launch_line_L<T, 16, EPI>(name, h, a, e, s);
        case 32: return launch_line_L<T, 32, EPI>(name, h, a, e, s);
        case 64: return launch_line_L<T, 64, EPI>(name, h, a, e, s);
        case 128: return launch_line_L<T, 128, EPI>(name, h, a, e, s);
        case 256: return launch_line_L<T, 256, EPI>(name, h, a, e, s);
        case 512: return launch_line_L<T, 512, EPI>(name, h, a, e, s);
        case 1024: return launch_line_L<T, 1024, EPI>(name, h, a, e, s);
    }
    set_error("unsupported FFT length " + std::to_string(L));
    return VIE_EINVAL;
}

template <typename T, int L, int NC, bool KOP = false>
static int launch_z_L(const char* name, const vie_handle* h, const ZArgs& z, cudaStream_t s) {
    using C = typename CT<T>::C;
    using Cfg = ZCfg<T, L, NC>;
    constexpr int TB = Cfg::TB;
    size_t smem = sizeof(C) * (size_t)(NC * Cfg::GS + L);
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(zpass_kernel<T, L, NC, KOP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    long long blocks = (long long)z.Ly * ((z.Lx + TB - 1) / TB);
    // the z lines read and written once, and the octant tensors the block reads (60, 30 or 6)
    const double bytes = (double)sizeof(C) * (2.0 * z.R * NC * z.nz * z.Ly * z.Lx +
                                              (KOP ? 30.0 : (NC == 12 ? 60.0 : 6.0)) * z.Ox * z.Oy * z.Oz);
    VIE_KLAUNCH_B(name, s, bytes,
                  (zpass_kernel<T, L, NC, KOP><<<(unsigned)blocks, Cfg::NT, smem, s>>>(z, twiddles<T>(h, L))));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename T, int NC = 12, bool KOP = false>
static int launch_z(const char* name, const vie_handle* h, int L, const ZArgs& z, cudaStream_t s) {
    switch (L) {
        case 2: return launch_z_L<T, 2, NC, KOP>(name, h, z, s);
        case 4: return launch_z_L<T, 4, NC, KOP>(name, h, z, s);
        case 8: return launch_z_L<T, 8, NC, KOP>(name, h, z, s);
        case 16: return launch_z_L<T, 16, NC, KOP>(name, h, z, s);
        case 32: return launch_z_L<T, 32, NC, KOP>(name, h, z, s);
        case 64: return launch_z_L<T, 64, NC, KOP>(name, h, z, s);
        case 128: return launch_z_L<T, 128, NC, KOP>(name, h, z, s);
        case 256: return launch_z_L<T, 256, NC, KOP>(name, h, z, s);
        case 512: return launch_z_L<T, 512, NC, KOP>(name, h, z, s);
        case 1024: return launch_z_L<T, 1024, NC, KOP>(name, h, z, s);
    }
    set_error("unsupported FFT length " + std::to_string(L));
    return VIE_EINVAL;
}

// The fused xy kernels need a square xy circulant of 8..128 (the column map is built at
// setup only for such grids); the FP32 z pass with the block product needs Lz of 8..512.
static bool xy_ok(const vie_handle* h) { return h->colmap != nullptr; }
static bool zfused_ok(const vie_handle* h) { return h->L[2] >= 8 && h->L[2] <= 512 && h->L[0] >= 4; }

// in_elems: complex values of the matvec input (and output) vector
template <int L, typename C>
static int launch_xy_L(bool fwd, const vie_handle* h, const void* in, void* out, long long planes, int nx, int ny,
                       const MatvecEpi& e, const Support& sp, double in_elems, cudaStream_t s) {
    constexpr size_t smem = XYCfg<L, C>::smem;
    constexpr bool f32 = sizeof(C) == 8;
    // set on every call: the attribute is per device and launches may come from several threads
    VIE_CUDA(cudaFuncSetAttribute(xy_fwd_kernel<L, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VIE_CUDA(cudaFuncSetAttribute(xy_inv_kernel<L, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (sizeof(C) == 16)
        VIE_CUDA(cudaFuncSetAttribute(xy_inv_kernel<L, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    if (e.conv && sizeof(C) != 16) {
        set_error("internal: the convolution side output is FP64 only");
        return VIE_EINVAL;
    }
    if (planes > 0x7fffffffLL) {
        set_error("xy transform grid too large");
        return VIE_EINVAL;
    }
    const unsigned char* cpos = h->colmap + L;
    const C* tw = reinterpret_cast<const C*>(f32 ? (const void*)(h->tw32 + L) : (const void*)(h->tw64 + L));
    const double c = sizeof(C), plane_full = (double)L * L;
    // with a device count of right-hand sides (e.nact) the kernel adds its bytes on the device:
    // the part proportional to the planes transformed, per right-hand side of the grid, plus a fixed part
    const double rg = (double)planes / ((double)h->nc * h->nz);  // right-hand sides of the launch grid
    MatvecEpi ee = e;
    if (fwd) {
        const char* name = f32 ? "fft_xy_f32" : "fft_xy_f64";
        double bytes = c * (in_elems + planes * plane_full);
        if (e.nact) {
            ee.bctr = dev_bytes_ptr(name);
            ee.bfix = 0.0;
            ee.bper = bytes / rg;
            bytes = kDevCounted;
        }
        VIE_KLAUNCH_B(name, s, bytes,
                      xy_fwd_kernel<L, C><<<(unsigned)planes, kXYThreads, smem, s>>>(
                          (const C*)in, (C*)out, nx, ny, h->nz, sp.rows, sp.ns, cpos, tw, e.rmap, ee));
    } else {
        const double fixed = c * (double)h->nv * (e.op == VIE_OP_PA ? 2 : e.op == VIE_OP_A ? 1 : 0);
        const double per = c * (planes * plane_full + in_elems * (e.op == VIE_OP_NSCAT ? 1 : 2) +
                                (e.conv ? (double)planes * nx * ny : 0.0));
        double bytes = fixed + per;
        const bool conv64 = sizeof(C) == 16 && e.conv;
        const char* name = f32 ? "ifft_xy_epilogue_f32" : "ifft_xy_epilogue_f64";
        if (e.nact) {
            ee.bctr = dev_bytes_ptr(name);
            ee.bfix = fixed;
            ee.bper = per / rg;
            bytes = kDevCounted;
        }
        if constexpr (sizeof(C) == 16) {
            if (conv64) {
                VIE_KLAUNCH_B(name, s, bytes,
                              xy_inv_kernel<L, C, true><<<(unsigned)planes, kXYThreads, smem, s>>>(
                                  (const C*)in, (C*)out, ee, cpos, tw));
                VIE_CHECK_LAUNCH();
                return VIE_OK;
            }
        }
        VIE_KLAUNCH_B(name, s, bytes,
                      xy_inv_kernel<L, C, false><<<(unsigned)planes, kXYThreads, smem, s>>>((const C*)in, (C*)out, ee,
                                                                                           cpos, tw));
    }
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename C>
static int launch_xy(bool fwd, const vie_handle* h, const void* in, void* out, long long planes, int nx, int ny,
                     const MatvecEpi& e, const Support& sp, double in_elems, cudaStream_t s) {
    switch (h->L[0]) {
        case 8: return launch_xy_L<8, C>(fwd, h, in, out, planes, nx, ny, e, sp, in_elems, s);
        case 16: return launch_xy_L<16, C>(fwd, h, in, out, planes, nx, ny, e, sp, in_elems, s);
        case 32: return launch_xy_L<32, C>(fwd, h, in, out, planes, nx, ny, e, sp, in_elems, s);
        case 64: return launch_xy_L<64, C>(fwd, h, in, out, planes, nx, ny, e, sp, in_elems, s);
        case 128: return launch_xy_L<128, C>(fwd, h, in, out, planes, nx, ny, e, sp, in_elems, s);
    }
    set_error("xy transform: unsupported length");
    return VIE_EINVAL;
}

// Spectrum scratch of one matvec: W2 [R*12][Nz][Ly][Lx] on the fused xy path, W1
// [R*12][Nz][Ny][Lx] in front of it on the line-transform path (the only one that uses W1).
size_t matvec_workspace_bytes(const vie_handle* h, int nrhs, int precision) {
    size_t c = precision == VIE_FP64 ? sizeof(double2) : sizeof(float2);
    size_t comps = (size_t)nrhs * h->nc * h->nz;
    size_t w2 = comps * h->L[1] * h->L[0];
    size_t w1 = xy_ok(h) ? 0 : comps * h->ny * h->L[0];
    return c * (w1 + w2) + 256;
}

// ws: scratch of at least matvec_workspace_bytes(h, R, precision) bytes (spectrum buffers W1, W2);
// sp: support of x and y (only the FP32 three-kernel path takes vectors on a support)
// bf16: the FP32 path with the BF16x3 block product in the z pass (T = float only)
template <typename T>
static int matvec_impl(vie_handle* h, int R, const void* x, void* y, int op, cudaStream_t s, void* ws,
                       const Support& sp = Support{}, const double2* shift = nullptr, void* conv = nullptr,
                       const int* rmap = nullptr, const int* nact = nullptr, bool bf16 = false) {
    using C = typename CT<T>::C;
    const int nx = h->nx, ny = h->ny, nz = h->nz, Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    // rmap with its device count nact (fused xy path only): transform only the *nact right-hand
    // sides it lists; the launches are sized for all R and skip the rest on the device
    if (!xy_ok(h) || !nact) rmap = nullptr;
    if (!rmap) nact = nullptr;
    const int Rs = R;  // right-hand sides the spectrum has room for
    const int nc = h->nc;
    const long long comps = (long long)Rs * nc * nz;
    // W1 exists on the line-transform path only (matvec_workspace_bytes)
    C* W1 = reinterpret_cast<C*>(ws);
    C* W2 = xy_ok(h) ? W1 : W1 + comps * ny * Lx;
    MatvecEpi e{};
    e.x = x;
    e.op = op == VIE_OP_K ? VIE_OP_NSCAT : op;  // K: the plain product, no voxel-wise terms
    e.nc = nc;
    e.nx = nx, e.ny = ny, e.nz = nz;
    const double dV = h->dx * h->dy * h->dz;
    e.g1 = dV;
    e.g234 = dV / 12.0;
    if (sizeof(T) == 8) {
        e.c1 = h->ieps64;
        e.c2 = op == VIE_OP_A ? (const void*)h->chi64 : (const void*)h->tau64;
    } else {
        e.c1 = h->ieps32;
        e.c2 = op == VIE_OP_A ? (const void*)h->chi32 : (const void*)h->tau32;
    }
    e.rows = sp.rows;
    e.ns = sp.ns;
    e.shift = op == VIE_OP_PA ? shift : nullptr;
    e.conv = conv;
    e.rmap = rmap;
    e.nact = nact;
    MatvecEpi noepi{};
    noepi.nc = nc;
    MatvecEpi fwdmap{};  // the forward kernel reads only rmap, the count and nc
    fwdmap.rmap = rmap;
    fwdmap.nact = nact;
    fwdmap.nc = nc;
    // z pass on a spectrum whose row py holds ky = py / by + ay (py % by) and whose stored
    // columns follow colkx32: the fused kernels (FP32, FP64) where they apply, else the line z pass
    auto zpass = [&](int ay, int by) -> int {
        if (op == VIE_OP_K) {  // the K block on the 30 K tensors: the fused z passes, else the generic one
            if (bf16 || nc != 12 || !h->kgreen64) {
                set_error("the K operator runs in FP64 or FP32 on the PWL system");
                return VIE_EINVAL;
            }
            if (sizeof(T) == 4 && zfused_ok(h) && h->kgreen32t) {
                ZFArgs z{};
                z.w = reinterpret_cast<float2*>(W2);
                z.green_t = h->kgreen32t;
                z.colkx = h->colkx32;
                z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
                z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
                z.ay = ay, z.by = by;
                z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
                return zpass_f32_fused_k(h, z, s);
            }
            if (sizeof(T) == 8 && zfused_ok(h) && h->kgreen64t) {
                ZDArgs z{};
                z.w = reinterpret_cast<double2*>(W2);
                z.green_t = h->kgreen64t;
                z.colkx = h->colkx32;
                z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
                z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
                z.ay = ay, z.by = by;
                z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
                return zpass_f64_fused_k(h, z, s);
            }
            ZArgs z{};
            z.w = W2;
            z.green = sizeof(T) == 8 ? (const void*)h->kgreen64 : (const void*)h->kgreen32;
            z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
            z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
            z.tstride = (long long)h->O[0] * h->O[1] * h->O[2];
            z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
            z.colkx = h->colkx32;
            z.ay = ay, z.by = by;
            return launch_z<T, 12, true>(sizeof(T) == 8 ? "zpass_block_k_f64" : "zpass_block_k_f32", h, Lz, z, s);
        }
        if (nc == 3) {  // PWC: the generic z pass with the 3 x 3 block of the l = 1 tensors
            if (bf16) {
                set_error("the BF16x3 matvec is built for the PWL system only");
                return VIE_EINVAL;
            }
            ZArgs z{};
            z.w = W2;
            z.green = sizeof(T) == 8 ? (const void*)h->green64 : (const void*)h->green32;
            z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
            z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
            z.tstride = (long long)h->O[0] * h->O[1] * h->O[2];
            // reflection parity of component p (the constant function) under axis i: -1 iff p = i
            z.mx = 1u, z.my = 2u, z.mz = 4u;
            z.colkx = h->colkx32;
            z.ay = ay, z.by = by;
            return launch_z<T, 3>(sizeof(T) == 8 ? "zpass_block_pwc_f64" : "zpass_block_pwc_f32", h, Lz, z, s);
        }
        if (sizeof(T) == 4 && zfused_ok(h)) {
            ZFArgs z{};
            z.w = reinterpret_cast<float2*>(W2);
            z.green_t = h->green32t;
            z.colkx = h->colkx32;
            z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
            z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
            z.ay = ay, z.by = by;
            z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
            z.nact = nact;
            z.bctr = nact ? dev_bytes_ptr(bf16 ? "zpass_block_bf16x3" : "zpass_block_f32") : nullptr;
            if (bf16) return zpass_bf16_fused(h, z, s);
            return zpass_f32_fused(h, z, s);
        }
        if (bf16) {
            set_error("the BF16x3 matvec needs an FFT length along z of 8..512");
            return VIE_EINVAL;
        }
        if (sizeof(T) == 8 && zfused_ok(h)) {
            ZDArgs z{};
            z.w = reinterpret_cast<double2*>(W2);
            z.green_t = h->green64t;
            z.colkx = h->colkx32;
            z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
            z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
            z.ay = ay, z.by = by;
            z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
            z.nact = nact;
            z.bctr = nact ? dev_bytes_ptr("zpass_block_f64") : nullptr;
            return zpass_f64_fused(h, z, s);
        }
        ZArgs z{};
        z.w = W2;
        z.green = sizeof(T) == 8 ? (const void*)h->green64 : (const void*)h->green32;
        z.R = Rs, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
        z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
        z.tstride = (long long)h->O[0] * h->O[1] * h->O[2];
        z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
        z.colkx = h->colkx32;
        z.ay = ay, z.by = by;
        return launch_z<T>(sizeof(T) == 8 ? "zpass_block_f64" : "zpass_block_f32", h, Lz, z, s);
    };
    if (xy_ok(h)) {
        const double in_elems = sp.rows ? (double)Rs * nc * sp.ns : (double)comps * ny * nx;
        VIE_TRY(launch_xy<C>(true, h, x, W2, comps, nx, ny, fwdmap, sp, in_elems, s));
        VIE_TRY(zpass(fft2::split_a(Ly), Ly / fft2::split_a(Ly)));
        return launch_xy<C>(false, h, W2, y, comps, nx, ny, e, sp, in_elems, s);
    }
    if (sp.rows) {
        set_error("internal: the line-transform matvec takes full-grid vectors only");
        return VIE_EINVAL;
    }
    // The line transforms: the two-pass kernels (line2.cu) for lengths 8..512, else the radix-4
    // line kernels; the inverse x transform with the voxel-wise terms always on the radix-4 one.
    // Both store the x spectrum in the column order of colkx32; the y spectrum's rows are in
    // fft2's transposed order after the two-pass kernel (row py holds ky = py / B + A (py % B),
    // A B = Ly) and in natural order after the radix-4 one.
    const bool fp64 = sizeof(T) == 8;
    const bool x2 = line2_ok(Lx), y2 = line2_ok(Ly);
    // x-pass: lines along x, contiguous; frequencies stored in the column order of colkx32
    LineArgs a{};
    a.in = x;
    a.out = W1;
    a.na = 1;
    a.nb = (int)(comps * ny);
    a.ia = 0, a.il = 1, a.ib = nx;
    a.oa = 0, a.ol = 1, a.ob = Lx;
    a.n_in = nx, a.n_out = Lx, a.dir = -1;
    a.pout = h->colpos32;
    if (x2)
        VIE_TRY(line2_forward(fp64 ? "fft_x_f64" : "fft_x_f32", h, Lx, fp64, a, h->colkx32, s));
    else
        VIE_TRY((launch_line<T, false>(fp64 ? "fft_x_f64" : "fft_x_f32", h, Lx, a, noepi, s)));
    // y-pass
    a = LineArgs{};
    a.in = W1;
    a.out = W2;
    a.na = (int)comps;
    a.nb = Lx;
    a.ia = (long long)ny * Lx, a.il = Lx, a.ib = 1;
    a.oa = (long long)Ly * Lx, a.ol = Lx, a.ob = 1;
    a.n_in = ny, a.n_out = Ly, a.dir = -1;
    if (y2)
        VIE_TRY(line2_forward(fp64 ? "fft_y_f64" : "fft_y_f32", h, Ly, fp64, a, nullptr, s));
    else
        VIE_TRY((launch_line<T, false>(fp64 ? "fft_y_f64" : "fft_y_f32", h, Ly, a, noepi, s)));
    // z-pass with block product: row order (ay, by) of the y spectrum, the natural order as
    // (1, Ly) for the fused kernels' formula and (0, 0) for the line z pass
    if (y2)
        VIE_TRY(zpass(fft2::split_a(Ly), Ly / fft2::split_a(Ly)));
    else
        VIE_TRY(zfused_ok(h) ? zpass(1, Ly) : zpass(0, 0));
    // y-inverse
    a = LineArgs{};
    a.in = W2;
    a.out = W1;
    a.na = (int)comps;
    a.nb = Lx;
    a.ia = (long long)Ly * Lx, a.il = Lx, a.ib = 1;
    a.oa = (long long)ny * Lx, a.ol = Lx, a.ob = 1;
    a.n_in = Ly, a.n_out = ny, a.dir = +1;
    if (y2)
        VIE_TRY(line2_inverse(fp64 ? "ifft_y_f64" : "ifft_y_f32", h, Ly, fp64, a, nullptr, s));
    else
        VIE_TRY((launch_line<T, false>(fp64 ? "ifft_y_f64" : "ifft_y_f32", h, Ly, a, noepi, s)));
    // x-inverse (frequencies read from their stored columns) + crop + material/Gram terms
    a = LineArgs{};
    a.in = W1;
    a.out = y;
    a.na = 1;
    a.nb = (int)(comps * ny);
    a.ia = 0, a.il = 1, a.ib = Lx;
    a.oa = 0, a.ol = 1, a.ob = nx;
    a.n_in = Lx, a.n_out = nx, a.dir = +1;
    a.pin = h->colpos32;
    VIE_TRY((launch_line<T, true>(fp64 ? "ifft_x_epilogue_f64" : "ifft_x_epilogue_f32", h, Lx, a, e, s)));
    return VIE_OK;
}

// Runs the z-pass autotuner for nrhs right-hand sides of this precision and operator (the N
// block, or the K block with op VIE_OP_K) now, outside any stream capture, so that a CUDA graph
// captured later launches the tuned tile width.
int matvec_tune(vie_handle* h, int nrhs, int precision, cudaStream_t s, int op) {
    if (precision == VIE_FP64 || !zfused_ok(h) || h->nc != 12) return VIE_OK;
    if (op == VIE_OP_K) {
        if (precision != VIE_FP32) return VIE_OK;
        VIE_TRY(k_octants(h, s));
    }
    ZFArgs z{};
    z.w = nullptr;
    z.green_t = op == VIE_OP_K ? h->kgreen32t : h->green32t;
    z.colkx = h->colkx32;
    z.R = nrhs, z.nz = h->nz, z.Lx = h->L[0], z.Ly = h->L[1];
    z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
    // the row order of the y spectrum (transposed after the fused xy kernels and the two-pass
    // line kernels, natural after the radix-4 ones)
    const bool yt = xy_ok(h) || line2_ok(h->L[1]);
    const int ay = yt ? fft2::split_a(h->L[1]) : 1, by = yt ? h->L[1] / fft2::split_a(h->L[1]) : h->L[1];
    z.ay = ay, z.by = by;
    z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
    if (op == VIE_OP_K) return zpass_f32_tune_k(h, z, s);
    return precision == VIE_BF16X3 ? zpass_bf16_tune(h, z, s) : zpass_f32_tune(h, z, s);
}

static int matvec_full(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, cudaStream_t s,
                       void* conv) {
    if (op == VIE_OP_K) VIE_TRY(k_octants(h, s));
    VIE_TRY(ws_reserve(h, h->fft_ws, matvec_workspace_bytes(h, nrhs, precision)));
    if (precision == VIE_FP64) return matvec_impl<double>(h, nrhs, x, y, op, s, h->fft_ws.ptr, Support{}, nullptr, conv);
    return matvec_impl<float>(h, nrhs, x, y, op, s, h->fft_ws.ptr, Support{}, nullptr, conv, nullptr, nullptr,
                              precision == VIE_BF16X3);
}

int matvec_device(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, cudaStream_t s) {
    return matvec_full(h, nrhs, x, y, precision, op, s, nullptr);
}

// ---------------------------------------------------------------------------
// Vectors on a support: [R][12][ns] <-> full grid [R][12][Nz][Ny][Nx]
// ---------------------------------------------------------------------------
template <typename C>
__global__ void support_gather_kernel(const C* __restrict__ full, C* __restrict__ part, const int4* __restrict__ rows,
                                      long long ns, int nx, long long nrows, long long total) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // full-grid element
    if (e >= total) return;
    const int xx = (int)(e % nx);
    const long long row = (e / nx) % nrows, comp = e / (nx * nrows);
    const int4 q = rows[row];
    if (xx >= q.x && xx < q.y) part[comp * ns + q.z + (xx - q.x)] = full[e];
}
template <typename C>
__global__ void support_scatter_kernel(const C* __restrict__ part, C* __restrict__ full, const int4* __restrict__ rows,
                                       long long ns, int nx, long long nrows, long long total) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int xx = (int)(e % nx);
    const long long row = (e / nx) % nrows, comp = e / (nx * nrows);
    const int4 q = rows[row];
    full[e] = (xx >= q.x && xx < q.y) ? part[comp * ns + q.z + (xx - q.x)] : C{};
}

template <typename C>
static int support_copy(const vie_handle* h, int R, const void* src, void* dst, const Support& sp, bool gather,
                        cudaStream_t s) {
    const long long total = (long long)R * h->nc * (long long)h->nv;
    if (!sp.rows) {
        VIE_CUDA(cudaMemcpyAsync(dst, src, sizeof(C) * (size_t)total, cudaMemcpyDeviceToDevice, s));
        return VIE_OK;
    }
    const unsigned g = (unsigned)((total + 255) / 256);
    const long long nrows = (long long)h->ny * h->nz;
    if (gather)
        VIE_KLAUNCH("support_gather", s,
                    support_gather_kernel<C><<<g, 256, 0, s>>>((const C*)src, (C*)dst, sp.rows, sp.ns, h->nx, nrows,
                                                               total));
    else
        VIE_KLAUNCH("support_scatter", s,
                    support_scatter_kernel<C><<<g, 256, 0, s>>>((const C*)src, (C*)dst, sp.rows, sp.ns, h->nx, nrows,
                                                                total));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

int support_gather(const vie_handle* h, int R, const void* full, void* part, int precision, const Support& sp,
                   cudaStream_t s) {
    return precision == VIE_FP64 ? support_copy<double2>(h, R, full, part, sp, true, s)
                                 : support_copy<float2>(h, R, full, part, sp, true, s);
}
int support_scatter(const vie_handle* h, int R, const void* part, void* full, int precision, const Support& sp,
                    cudaStream_t s) {
    return precision == VIE_FP64 ? support_copy<double2>(h, R, part, full, sp, false, s)
                                 : support_copy<float2>(h, R, part, full, sp, false, s);
}

// y -= shift[r] x for vectors of n complex values per right-hand side
template <typename C>
__global__ void shift_sub_kernel(C* __restrict__ y, const C* __restrict__ x, const double2* __restrict__ shift,
                                 long long n) {
    const int r = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    using R = decltype(C{}.x);
    const long long o = (long long)r * n + e;
    y[o] = csub(y[o], cmul(mk((R)shift[r].x, (R)shift[r].y), x[o]));
}

int matvec_support(vie_handle* h, int R, const void* x, void* y, int precision, int op, const Support& sp, void* tmp,
                   cudaStream_t s, const double2* shift, void* conv, const int* rmap, const int* nact) {
    if (op != VIE_OP_PA) shift = nullptr;
    VIE_TRY(ws_reserve(h, h->fft_ws, matvec_workspace_bytes(h, R, precision)));
    if (xy_ok(h) || !sp.rows)
        return precision == VIE_FP64
                   ? matvec_impl<double>(h, R, x, y, op, s, h->fft_ws.ptr, sp, shift, conv, rmap, nact)
                   : matvec_impl<float>(h, R, x, y, op, s, h->fft_ws.ptr, sp, shift, conv, rmap, nact,
                                        precision == VIE_BF16X3);
    const size_t c = precision == VIE_FP64 ? sizeof(double2) : sizeof(float2);
    void* tx = tmp;
    void* ty = static_cast<char*>(tmp) + c * (size_t)R * h->nc * h->nv;
    VIE_TRY(support_scatter(h, R, x, tx, precision, sp, s));
    VIE_TRY(matvec_full(h, R, tx, ty, precision, op, s, conv));
    VIE_TRY(support_gather(h, R, ty, y, precision, sp, s));
    if (shift) {
        const long long n = (long long)h->nc * sp.ns;
        const dim3 g((unsigned)((n + 255) / 256), R);
        if (precision == VIE_FP64)
            VIE_KLAUNCH("matvec_shift", s,
                        shift_sub_kernel<double2><<<g, 256, 0, s>>>((double2*)y, (const double2*)x, shift, n));
        else
            VIE_KLAUNCH("matvec_shift", s,
                        shift_sub_kernel<float2><<<g, 256, 0, s>>>((float2*)y, (const float2*)x, shift, n));
        VIE_CHECK_LAUNCH();
    }
    return VIE_OK;
}

// Full forward 3-D FFT of [batch][Lz][Ly][Lx] complex double volumes, in place.
int fft3d_inplace64(vie_handle* h, double2* data, int batch, cudaStream_t s) {
    const int Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    MatvecEpi noepi{};
    LineArgs a{};
    a.in = data, a.out = data;
    a.na = 1, a.nb = batch * Lz * Ly;
    a.ia = 0, a.il = 1, a.ib = Lx, a.oa = 0, a.ol = 1, a.ob = Lx;
    a.n_in = Lx, a.n_out = Lx, a.dir = -1;
    VIE_TRY((launch_line<double, false>("green_fft_x", h, Lx, a, noepi, s)));
    a = LineArgs{};
    a.in = data, a.out = data;
    a.na = batch * Lz, a.nb = Lx;
    a.ia = (long long)Ly * Lx, a.il = Lx, a.ib = 1, a.oa = (long long)Ly * Lx, a.ol = Lx, a.ob = 1;
    a.n_in = Ly, a.n_out = Ly, a.dir = -1;
    VIE_TRY((launch_line<double, false>("green_fft_y", h, Ly, a, noepi, s)));
    a = LineArgs{};
    a.in = data, a.out = data;
    a.na = batch, a.nb = Ly * Lx;
    a.ia = (long long)Lz * Ly * Lx, a.il = (long long)Ly * Lx, a.ib = 1;
    a.oa = a.ia, a.ol = a.il, a.ob = 1;
    a.n_in = Lz, a.n_out = Lz, a.dir = -1;
    VIE_TRY((launch_line<double, false>("green_fft_z", h, Lz, a, noepi, s)));
    return VIE_OK;
}

// Stored column order of the FP32 spectrum (see the three-kernel path): colkx[sc] = kx of
// stored column sc, colkx[L + sc] = its position in the transposed order of the x transform.
// Mirror pairs fill tiles of 8 (two to a 16-column group chosen greedily so that their
// positions differ modulo 16); the last tile ends with the self-mirrored columns 0, L/2.
static bool build_colmap(int L, std::vector<unsigned char>& map) {
    map.assign(2 * L, 0);
    std::vector<int> kx(L, -1);
    std::vector<bool> used(L / 2, false);  // pair (j, L - j) for j = 1..L/2-1
    unsigned mask = 0;
    int group = -1;
    const int ntile = L / 8;
    for (int t = 0; t < ntile; ++t)
        for (int i = 0; i < (t < ntile - 1 ? 4 : 3); ++i) {
            const int sc = 8 * t + 2 * i;
            if (sc / 16 != group) group = sc / 16, mask = 0u;
            int pick = -1;
            for (int j = 1; j < L / 2 && pick < 0; ++j) {
                if (used[j]) continue;
                const int ra = fft2::tpos(L, j) % 16, rb = fft2::tpos(L, L - j) % 16;
                if (ra != rb && !((mask >> ra) & 1u) && !((mask >> rb) & 1u)) pick = j;
            }
            for (int j = 1; j < L / 2 && pick < 0; ++j)
                if (!used[j]) pick = j;
            if (pick < 0) return false;
            used[pick] = true;
            kx[sc] = pick, kx[sc + 1] = L - pick;
            mask |= (1u << (fft2::tpos(L, pick) % 16)) | (1u << (fft2::tpos(L, L - pick) % 16));
        }
    kx[L - 2] = 0, kx[L - 1] = L / 2;
    std::vector<bool> seen(L, false);
    for (int sc = 0; sc < L; ++sc) {
        if (kx[sc] < 0 || kx[sc] >= L || seen[kx[sc]]) return false;
        seen[kx[sc]] = true;
        map[sc] = (unsigned char)kx[sc];
        map[L + sc] = (unsigned char)fft2::tpos(L, kx[sc]);
    }
    return true;
}

int twiddle_setup(vie_handle* h) {
    // tables for L = 2^k, k = 1..10, stored at offset L (total 2048 entries)
    const int total = 2048;
    std::vector<double2> t64(total);
    std::vector<float2> t32(total);
    for (int L = 2; L <= 1024; L *= 2)
        for (int m = 0; m < L; ++m) {
            double ang = -2.0 * VIE_PI * (double)m / (double)L;
            double c = std::cos(ang), sn = std::sin(ang);
            t64[L + m] = make_double2(c, sn);
            t32[L + m] = make_float2((float)c, (float)sn);
        }
    VIE_CUDA(cudaMalloc(&h->tw64, total * sizeof(double2)));
    VIE_CUDA(cudaMalloc(&h->tw32, total * sizeof(float2)));
    h->bytes_held += total * (sizeof(double2) + sizeof(float2));
    VIE_CUDA(cudaMemcpy(h->tw64, t64.data(), total * sizeof(double2), cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(h->tw32, t32.data(), total * sizeof(float2), cudaMemcpyHostToDevice));
    h->colmap = nullptr;
    const int L = h->L[0];
    std::vector<int> kx32(L), pos32(L);
    for (int sc = 0; sc < L; ++sc) {  // mirror pairs, then the self-mirrored columns 0 and L/2
        const int j = sc / 2 + 1;
        kx32[sc] = sc < L - 2 ? ((sc & 1) ? L - j : j) : (sc == L - 2 ? 0 : L / 2);
    }
    if (L == h->L[1] && L >= 8 && L <= 128) {
        std::vector<unsigned char> map;
        if (!build_colmap(L, map)) {
            set_error("column map construction failed");
            return VIE_EDEVICE;
        }
        VIE_CUDA(cudaMalloc(&h->colmap, map.size()));
        h->bytes_held += map.size();
        VIE_CUDA(cudaMemcpy(h->colmap, map.data(), map.size(), cudaMemcpyHostToDevice));
        for (int sc = 0; sc < L; ++sc) kx32[sc] = map[sc];
    }
    for (int sc = 0; sc < L; ++sc) pos32[kx32[sc]] = sc;
    VIE_CUDA(cudaMalloc(&h->colkx32, sizeof(int) * 2 * L));
    h->colpos32 = h->colkx32 + L;
    h->bytes_held += sizeof(int) * 2 * L;
    VIE_CUDA(cudaMemcpy(h->colkx32, kx32.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(h->colpos32, pos32.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
    return VIE_OK;
}

// ---------------------------------------------------------------------------
// vie_matvec_noalloc: the same matvec with its spectrum buffers in a fixed,
// file-scope device array instead of handle-owned memory from cudaMalloc.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB, held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 256;
void* g_noalloc_addr[kMaxDevices];  // device address of the array, per device ordinal

// Device address of the scratch array on the current device, looked up once per device.
int noalloc_scratch(void** out) {
    int dev = -1;
    VIE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the static scratch table");
        return VIE_EDEVICE;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
            return VIE_EDEVICE;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return VIE_OK;
}

// p is device memory of `device` (or managed memory)
bool on_device(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}
}  // namespace

extern "C" int vie_matvec_noalloc(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op,
                                  void* stream) {
    if (!h || !x || !y) {
        set_error("NULL argument");
        return VIE_EINVAL;
    }
    if (nrhs < 1 || (precision != VIE_FP64 && precision != VIE_FP32) ||
        (op != VIE_OP_A && op != VIE_OP_PA && op != VIE_OP_NSCAT) || x == y) {
        set_error("invalid nrhs, precision, operator, or x == y");
        return VIE_EINVAL;
    }
    if (!on_device(x, h->device) || !on_device(y, h->device)) {
        set_error("vie_matvec_noalloc needs x and y in device memory of the handle's device (host buffers would "
                  "need staging memory)");
        return VIE_EINVAL;
    }
    int dev = -1;
    VIE_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) {
        set_error("the current device is not the handle's device");
        return VIE_EINVAL;
    }
    const size_t need = matvec_workspace_bytes(h, nrhs, precision);
    if (need > kNoAllocScratchBytes) {
        set_error("vie_matvec_noalloc: this call needs " + std::to_string(need) +
                  " bytes of scratch but the static scratch holds " + std::to_string(kNoAllocScratchBytes) +
                  " bytes; pass fewer right-hand sides per call or use vie_matvec");
        return VIE_EINVAL;
    }
    void* ws = nullptr;
    VIE_TRY(noalloc_scratch(&ws));
    cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : h->stream;
    if (precision == VIE_FP64) return matvec_impl<double>(h, nrhs, x, y, op, s, ws);
    return matvec_impl<float>(h, nrhs, x, y, op, s, ws);
}
