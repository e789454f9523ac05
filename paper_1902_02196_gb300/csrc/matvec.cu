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
#include "fft.cuh"

// ---------------------------------------------------------------------------
// Constant table: for each unique tensor t the (alpha, beta, sign) entries of the 12x12 block
// ---------------------------------------------------------------------------
struct BlockEntry {
    signed char a, b, s;
};
struct BlockTable {
    BlockEntry e[144];
    int start[61];
};
constexpr BlockTable make_block_table() {
    BlockTable T{};
    int n = 0;
    for (int t = 0; t < 60; ++t) {
        T.start[t] = n;
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b)
                if (tensor_of(a, b) == t) {
                    T.e[n].a = (signed char)a;
                    T.e[n].b = (signed char)b;
                    T.e[n].s = (signed char)sign_of(a, b);
                    ++n;
                }
    }
    T.start[60] = n;
    return T;
}
__device__ constexpr BlockTable kBlock = make_block_table();
static_assert(make_block_table().start[60] == 144, "every block entry maps to one of the 60 tensors");

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

template <typename T, int L>
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
};

template <typename T, int L>
__global__ void __launch_bounds__(ZCfg<T, L>::NT) zpass_kernel(ZArgs z, const typename CT<T>::C* twg) {
    using C = typename CT<T>::C;
    constexpr int TB = ZCfg<T, L>::TB, GS = ZCfg<T, L>::GS, NT = ZCfg<T, L>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* tw = s + 12 * GS;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += NT) tw[m] = twg[m];

    const int ntile = (z.Lx + TB - 1) / TB;
    const int ky = blockIdx.x / ntile;
    const int kx0 = (blockIdx.x % ntile) * TB;
    const long long plane = (long long)z.Ly * z.Lx;
    C* w = reinterpret_cast<C*>(z.w);
    const C* green = reinterpret_cast<const C*>(z.green);
    const C zero = mk(T(0), T(0));
    const int Lz = L;
    const int kyo = ky <= z.Ly / 2 ? ky : z.Ly - ky;
    const unsigned fy = ky > z.Ly / 2 ? z.my : 0u;

    for (int r = 0; r < z.R; ++r) {
        C* base = w + (long long)r * 12 * z.nz * plane + (long long)ky * z.Lx + kx0;
        for (int idx = tid; idx < 12 * L * TB; idx += NT) {
            int tb = idx % TB;
            int l = (idx / TB) % L;
            int a = idx / (TB * L);
            C v = zero;
            if (l < z.nz && kx0 + tb < z.Lx) v = base[((long long)a * z.nz + l) * plane + tb];
            s[a * GS + l * TB + tb] = v;
        }
        __syncthreads();
        fft_smem<C, L, 12, TB, TB, GS, NT>(s, tw, -1);
        for (int p = tid; p < L * TB; p += NT) {
            int tb = p % TB;
            int kz = p / TB;
            int kx = kx0 + tb;
            if (kx >= z.Lx) continue;
            int kxo = kx <= z.Lx / 2 ? kx : z.Lx - kx;
            int kzo = kz <= Lz / 2 ? kz : Lz - kz;
            unsigned mask = fy ^ (kx > z.Lx / 2 ? z.mx : 0u) ^ (kz > Lz / 2 ? z.mz : 0u);
            C xv[12], acc[12];
#pragma unroll
            for (int b = 0; b < 12; ++b) {
                C v = s[b * GS + kz * TB + tb];
                xv[b] = ((mask >> b) & 1u) ? cneg(v) : v;
            }
            const C* gp = green + ((long long)kzo * z.Oy + kyo) * z.Ox + kxo;
            block_product(xv, acc, gp, z.tstride);
#pragma unroll
            for (int a = 0; a < 12; ++a) s[a * GS + kz * TB + tb] = ((mask >> a) & 1u) ? cneg(acc[a]) : acc[a];
        }
        __syncthreads();
        fft_smem<C, L, 12, TB, TB, GS, NT>(s, tw, +1);
        for (int idx = tid; idx < 12 * z.nz * TB; idx += NT) {
            int tb = idx % TB;
            int l = (idx / TB) % z.nz;
            int a = idx / (TB * z.nz);
            if (kx0 + tb < z.Lx) base[((long long)a * z.nz + l) * plane + tb] = s[a * GS + l * TB + tb];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Fused plane kernels (FP32, Lx = Ly = L <= 128): a whole L x L plane of one
// component grid in shared memory, so the x and y transforms cost one HBM pass.
// Since L >= 2N - 1, at most L/2 rows are non-zero before the y transform and at
// most L/2 rows are needed after the inverse one.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(512) xy_fwd_kernel(const float2* __restrict__ x, float2* __restrict__ w, int nx,
                                                     int ny, const float2* __restrict__ twg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    float2* tw = s + L * L;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += 512) tw[m] = twg[m];
    const long long p = blockIdx.x;  // plane (component, z)
    const float2* src = x + p * (long long)ny * nx;
    for (int idx = tid; idx < L * L; idx += 512) {
        const int yy = idx / L, xx = idx % L;
        float2 v = make_float2(0.f, 0.f);
        if (yy < ny && xx < nx) v = src[yy * nx + xx];
        s[idx] = v;
    }
    __syncthreads();
    fft_smem<float2, L, L / 2, 1, 1, L, 512>(s, tw, -1);  // rows 0..L/2-1 along x
    fft_smem<float2, L, 1, L, L, 0, 512>(s, tw, -1);      // L columns along y
    float2* dst = w + p * (long long)L * L;
    for (int idx = tid; idx < L * L; idx += 512) dst[idx] = s[idx];
}

template <int L>
__global__ void __launch_bounds__(512) xy_inv_kernel(const float2* __restrict__ w, float2* __restrict__ y,
                                                     MatvecEpi epi, const float2* __restrict__ twg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    float2* tw = s + L * L;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += 512) tw[m] = twg[m];
    const long long p = blockIdx.x;  // plane (r * 12 + alpha) * nz + z
    const float2* src = w + p * (long long)L * L;
    for (int idx = tid; idx < L * L; idx += 512) s[idx] = src[idx];
    __syncthreads();
    fft_smem<float2, L, 1, L, L, 0, 512>(s, tw, +1);      // L columns along y
    fft_smem<float2, L, L / 2, 1, 1, L, 512>(s, tw, +1);  // rows 0..L/2-1 along x
    const int nx = epi.nx, ny = epi.ny, nz = epi.nz;
    const int alpha = (int)((p / nz) % 12);
    const long long zoff = (p % nz) * (long long)ny * nx;
    const long long base = p * (long long)ny * nx;
    const float gl = (float)((alpha % 4) == 0 ? epi.g1 : epi.g234);
    const float2* xin = reinterpret_cast<const float2*>(epi.x);
    const float2* c1 = reinterpret_cast<const float2*>(epi.c1);
    const float2* c2 = reinterpret_cast<const float2*>(epi.c2);
    for (int idx = tid; idx < ny * nx; idx += 512) {
        const int yy = idx / nx, xx = idx % nx;
        float2 v = s[yy * L + xx];
        const long long vox = zoff + idx;
        if (epi.op == VIE_OP_A) {
            float2 xv = xin[base + idx];
            v = csub(mk(gl * xv.x, gl * xv.y), cmul(c2[vox], v));
        } else if (epi.op == VIE_OP_PA) {
            float2 xv = xin[base + idx];
            float2 t = cmul(c2[vox], v);
            const float ig = 1.0f / gl;
            v = csub(cmul(c1[vox], xv), mk(ig * t.x, ig * t.y));
        }
        y[base + idx] = v;
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
    static bool configured = false;
    if (!configured) {
        VIE_CUDA(cudaFuncSetAttribute(line_fft_kernel<T, L, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        configured = true;
    }
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

template <typename T, int L>
static int launch_z_L(const char* name, const vie_handle* h, const ZArgs& z, cudaStream_t s) {
    using C = typename CT<T>::C;
    constexpr int TB = ZCfg<T, L>::TB;
    size_t smem = sizeof(C) * (size_t)(12 * ZCfg<T, L>::GS + L);
    static bool configured = false;
    if (!configured) {
        VIE_CUDA(cudaFuncSetAttribute(zpass_kernel<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    long long blocks = (long long)z.Ly * ((z.Lx + TB - 1) / TB);
    const double bytes = (double)sizeof(C) * (2.0 * z.R * 12 * z.nz * z.Ly * z.Lx + 60.0 * z.Ox * z.Oy * z.Oz);
    VIE_KLAUNCH_B(name, s, bytes,
                  zpass_kernel<T, L><<<(unsigned)blocks, ZCfg<T, L>::NT, smem, s>>>(z, twiddles<T>(h, L)));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename T>
static int launch_z(const char* name, const vie_handle* h, int L, const ZArgs& z, cudaStream_t s) {
    switch (L) {
        case 2: return launch_z_L<T, 2>(name, h, z, s);
        case 4: return launch_z_L<T, 4>(name, h, z, s);
        case 8: return launch_z_L<T, 8>(name, h, z, s);
        case 16: return launch_z_L<T, 16>(name, h, z, s);
        case 32: return launch_z_L<T, 32>(name, h, z, s);
        case 64: return launch_z_L<T, 64>(name, h, z, s);
        case 128: return launch_z_L<T, 128>(name, h, z, s);
        case 256: return launch_z_L<T, 256>(name, h, z, s);
        case 512: return launch_z_L<T, 512>(name, h, z, s);
        case 1024: return launch_z_L<T, 1024>(name, h, z, s);
    }
    set_error("unsupported FFT length " + std::to_string(L));
    return VIE_EINVAL;
}

template <int L>
static int launch_xy_L(bool fwd, const vie_handle* h, const void* in, void* out, long long planes, int nx, int ny,
                       const MatvecEpi& e, cudaStream_t s) {
    const size_t smem = sizeof(float2) * (size_t)(L * L + L);
    static bool configured = false;
    if (!configured) {
        VIE_CUDA(cudaFuncSetAttribute(xy_fwd_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VIE_CUDA(cudaFuncSetAttribute(xy_inv_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    const double plane_in = (double)nx * ny, plane_full = (double)L * L;
    if (fwd)
        VIE_KLAUNCH_B("fft_xy_f32", s, 8.0 * planes * (plane_in + plane_full),
                    xy_fwd_kernel<L><<<(unsigned)planes, 512, smem, s>>>((const float2*)in, (float2*)out, nx, ny,
                                                                        h->tw32 + L));
    else
        VIE_KLAUNCH_B("ifft_xy_epilogue_f32", s,
                      8.0 * (planes * (plane_full + plane_in * (e.op == VIE_OP_NSCAT ? 1 : 2)) +
                             (double)h->nv * (e.op == VIE_OP_PA ? 2 : e.op == VIE_OP_A ? 1 : 0)),
                    xy_inv_kernel<L><<<(unsigned)planes, 512, smem, s>>>((const float2*)in, (float2*)out, e,
                                                                        h->tw32 + L));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

static bool fused_xy_ok(const vie_handle* h) { return h->L[0] == h->L[1] && h->L[0] >= 8 && h->L[0] <= 128; }

static int launch_xy(bool fwd, const vie_handle* h, const void* in, void* out, long long planes, int nx, int ny,
                     const MatvecEpi& e, cudaStream_t s) {
    switch (h->L[0]) {
        case 8: return launch_xy_L<8>(fwd, h, in, out, planes, nx, ny, e, s);
        case 16: return launch_xy_L<16>(fwd, h, in, out, planes, nx, ny, e, s);
        case 32: return launch_xy_L<32>(fwd, h, in, out, planes, nx, ny, e, s);
        case 64: return launch_xy_L<64>(fwd, h, in, out, planes, nx, ny, e, s);
        case 128: return launch_xy_L<128>(fwd, h, in, out, planes, nx, ny, e, s);
    }
    set_error("fused xy path: unsupported length");
    return VIE_EINVAL;
}

size_t matvec_workspace_bytes(const vie_handle* h, int nrhs, int precision) {
    size_t c = precision == VIE_FP64 ? sizeof(double2) : sizeof(float2);
    size_t comps = (size_t)nrhs * 12 * h->nz;
    size_t w2 = comps * h->L[1] * h->L[0];
    size_t w1 = comps * h->ny * h->L[0];
    return c * (w1 + w2) + 256;
}

// ws: scratch of at least matvec_workspace_bytes(h, R, precision) bytes (spectrum buffers W1, W2)
template <typename T>
static int matvec_impl(vie_handle* h, int R, const void* x, void* y, int op, cudaStream_t s, void* ws) {
    using C = typename CT<T>::C;
    const int nx = h->nx, ny = h->ny, nz = h->nz, Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    const long long comps = (long long)R * 12 * nz;
    C* W1 = reinterpret_cast<C*>(ws);
    C* W2 = W1 + comps * ny * Lx;
    MatvecEpi noepi{};
    const bool fused = sizeof(T) == 4 && fused_xy_ok(h);
    if (fused) {
        VIE_TRY(launch_xy(true, h, x, W2, comps, nx, ny, noepi, s));
    } else {
        // x-pass: lines along x, contiguous
        LineArgs a{};
        a.in = x;
        a.out = W1;
        a.na = 1;
        a.nb = (int)(comps * ny);
        a.ia = 0, a.il = 1, a.ib = nx;
        a.oa = 0, a.ol = 1, a.ob = Lx;
        a.n_in = nx, a.n_out = Lx, a.dir = -1;
        VIE_TRY((launch_line<T, false>(sizeof(T) == 8 ? "fft_x_f64" : "fft_x_f32", h, Lx, a, noepi, s)));
        // y-pass
        a = LineArgs{};
        a.in = W1;
        a.out = W2;
        a.na = (int)comps;
        a.nb = Lx;
        a.ia = (long long)ny * Lx, a.il = Lx, a.ib = 1;
        a.oa = (long long)Ly * Lx, a.ol = Lx, a.ob = 1;
        a.n_in = ny, a.n_out = Ly, a.dir = -1;
        VIE_TRY((launch_line<T, false>(sizeof(T) == 8 ? "fft_y_f64" : "fft_y_f32", h, Ly, a, noepi, s)));
    }
    // z-pass with block product
    ZArgs z{};
    z.w = W2;
    z.green = sizeof(T) == 8 ? (const void*)h->green64 : (const void*)h->green32;
    z.R = R, z.nz = nz, z.Lx = Lx, z.Ly = Ly;
    z.Ox = h->O[0], z.Oy = h->O[1], z.Oz = h->O[2];
    z.tstride = (long long)h->O[0] * h->O[1] * h->O[2];
    z.mx = flip_mask(0), z.my = flip_mask(1), z.mz = flip_mask(2);
    VIE_TRY(launch_z<T>(sizeof(T) == 8 ? "zpass_block_f64" : "zpass_block_f32", h, Lz, z, s));
    MatvecEpi e{};
    e.x = x;
    e.op = op;
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
    if (fused) {
        VIE_TRY(launch_xy(false, h, W2, y, comps, nx, ny, e, s));
        return VIE_OK;
    }
    // y-inverse
    LineArgs a{};
    a.in = W2;
    a.out = W1;
    a.na = (int)comps;
    a.nb = Lx;
    a.ia = (long long)Ly * Lx, a.il = Lx, a.ib = 1;
    a.oa = (long long)ny * Lx, a.ol = Lx, a.ob = 1;
    a.n_in = Ly, a.n_out = ny, a.dir = +1;
    VIE_TRY((launch_line<T, false>(sizeof(T) == 8 ? "ifft_y_f64" : "ifft_y_f32", h, Ly, a, noepi, s)));
    // x-inverse + crop + material/Gram terms
    a = LineArgs{};
    a.in = W1;
    a.out = y;
    a.na = 1;
    a.nb = (int)(comps * ny);
    a.ia = 0, a.il = 1, a.ib = Lx;
    a.oa = 0, a.ol = 1, a.ob = nx;
    a.n_in = Lx, a.n_out = nx, a.dir = +1;
    VIE_TRY((launch_line<T, true>(sizeof(T) == 8 ? "ifft_x_epilogue_f64" : "ifft_x_epilogue_f32", h, Lx, a, e, s)));
    return VIE_OK;
}

int matvec_device(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, cudaStream_t s) {
    VIE_TRY(ws_reserve(h, h->fft_ws, matvec_workspace_bytes(h, nrhs, precision)));
    if (precision == VIE_FP64) return matvec_impl<double>(h, nrhs, x, y, op, s, h->fft_ws.ptr);
    return matvec_impl<float>(h, nrhs, x, y, op, s, h->fft_ws.ptr);
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

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
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
    if (!on_device(x) || !on_device(y)) {
        set_error("vie_matvec_noalloc needs device pointers for x and y (host buffers would need staging memory)");
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
