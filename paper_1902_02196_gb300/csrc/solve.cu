// Restarted, left-preconditioned GMRES on the device, batched over right-hand sides
// (Section IV-B: preconditioner P = M_eps G; Section V: GMRES with restart and a cap
// on the number of cycles), with an FP32 variant wrapped in FP64 iterative refinement.
//
// Arnoldi with classical Gram-Schmidt and a second pass where the new vector lost
// more than half of its squared norm; complex Givens rotations keep the Hessenberg
// matrix triangular and give the residual estimate |g_{j+1}|; at the end of a cycle
// H y = g is solved and x += V y.
//
// Memory traffic: the Krylov vectors are stored as u_i = n_i v_i with v_i orthonormal
// and n_i = ||u_i|| (close to 1) kept in FP64, so no separate normalisation pass is
// needed: the matvec writes op(u_j) straight into slot j+1, one pass computes every
// inner product u_i^H w and ||w||^2, and one pass subtracts the projections, rescales
// by 1/||w|| and returns the new squared norm.  The Hessenberg entries follow from
// those scalars: h_ij = (u_i^H w)/(n_i n_j), h_{j+1,j} = n_{j+1}/(sigma n_j) with sigma
// the rescale factor applied to the stored vector.
//
// Arithmetic: in the mixed mode the per-thread products and warp sums use FP32 (the
// Krylov vectors are FP32), block and grid reductions, the Hessenberg matrix, the
// rotations, the solution and every residual are FP64.  The plain mode is FP64
// throughout.  Every reduction uses a fixed partition of each right-hand side's
// vector, so one right-hand side's result does not depend on the others in a batch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

// algorithmic bytes moved by the Gram-Schmidt kernels: [0] dots, [1] update, [2] solution update
__device__ unsigned long long g_gs_bytes[3];

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxV = 130;  // basis vectors per pass (restart <= 128)

template <typename VC>
struct Prec;
template <>
struct Prec<float2> {
    using R = float;
    static constexpr int K = 4;  // complex values per thread per pass (32 bytes)
};
template <>
struct Prec<double2> {
    using R = double;
    static constexpr int K = 2;
};

template <typename C>
__device__ __forceinline__ C from_d(double2 v);
template <>
__device__ __forceinline__ float2 from_d<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}
template <>
__device__ __forceinline__ double2 from_d<double2>(double2 v) {
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 16-byte aligned address (a vector of nc ns float pairs per right-hand side starts on an odd
// element when nc ns is odd, as for the PWC system with an odd support)
__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// K consecutive complex values starting at element e0 of p (zero past n); 16-byte loads
// when the chunk is complete and aligned.
template <typename C, int K>
__device__ __forceinline__ void load_chunk(const C* __restrict__ p, long long e0, long long n, C* v) {
    if (e0 + K <= n && (sizeof(C) != 8 || al16(p + e0))) {
        if constexpr (sizeof(C) == 8) {
            const float4* q = reinterpret_cast<const float4*>(p + e0);
#pragma unroll
            for (int k = 0; k < K / 2; ++k) {
                const float4 t = q[k];
                v[2 * k] = make_float2(t.x, t.y);
                v[2 * k + 1] = make_float2(t.z, t.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = p[e0 + k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = e0 + k < n ? p[e0 + k] : C{};
    }
}
template <typename C, int K>
__device__ __forceinline__ void store_chunk(C* __restrict__ p, long long e0, long long n, const C* v) {
    if (e0 + K <= n && (sizeof(C) != 8 || al16(p + e0))) {
        if constexpr (sizeof(C) == 8) {
            float4* q = reinterpret_cast<float4*>(p + e0);
#pragma unroll
            for (int k = 0; k < K / 2; ++k) q[k] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) p[e0 + k] = v[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (e0 + k < n) p[e0 + k] = v[k];
    }
}

// partial[r][blk][i] = sum over the block's elements of conj(U_i) w (i < nvec) and, at i = nvec, |w|^2
template <typename VC>
__global__ void __launch_bounds__(kThreads) gs_dots_kernel(const VC* __restrict__ U, long long ustride,
                                                           const VC* __restrict__ w, long long n, int nvec,
                                                           double2* __restrict__ partial, int nblk,
                                                           const int* __restrict__ flag) {
    using R = typename Prec<VC>::R;
    constexpr int K = Prec<VC>::K;
    __shared__ double2 sh[kWarps][kMaxV + 1];
    const int r = blockIdx.y, blk = blockIdx.x;
    if (flag && !flag[r]) return;
    if (blk == 0 && threadIdx.x == 0) atomicAdd(&g_gs_bytes[0], (unsigned long long)(n * sizeof(VC) * (nvec + 1)));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long e0 = (long long)blk * (kThreads * K) + (long long)threadIdx.x * K;
    const long long roff = (long long)r * n;
    VC wv[K];
    load_chunk<VC, K>(w + roff, e0, n, wv);
    {
        R a = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) a += wv[k].x * wv[k].x + wv[k].y * wv[k].y;
        a = warp_sum(a);
        if (lane == 0) sh[wid][nvec] = make_double2((double)a, 0.0);
    }
#pragma unroll 2
    for (int i = 0; i < nvec; ++i) {
        VC uv[K];
        load_chunk<VC, K>(U + i * ustride + roff, e0, n, uv);
        R ar = 0, ai = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ar += uv[k].x * wv[k].x + uv[k].y * wv[k].y;
            ai += uv[k].x * wv[k].y - uv[k].y * wv[k].x;
        }
        ar = warp_sum(ar);
        ai = warp_sum(ai);
        if (lane == 0) sh[wid][i] = make_double2((double)ar, (double)ai);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= nvec; i += kThreads) {
        double2 s = make_double2(0, 0);
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s.x += sh[q][i].x, s.y += sh[q][i].y;
        partial[((long long)r * nblk + blk) * (nvec + 1) + i] = s;
    }
}

// w <- scale * (w - sum_i coef_i U_i), in place; npart[r][blk] = |new w|^2 over the block
template <typename VC>
__global__ void __launch_bounds__(kThreads) gs_update_kernel(const VC* __restrict__ U, long long ustride, VC* w,
                                                             long long n, int nvec, const double2* __restrict__ coef,
                                                             int ldc, const double* __restrict__ scale,
                                                             double* __restrict__ npart, int nblk,
                                                             const int* __restrict__ flag) {
    using R = typename Prec<VC>::R;
    constexpr int K = Prec<VC>::K;
    __shared__ VC c[kMaxV];
    __shared__ double shn[kWarps];
    const int r = blockIdx.y, blk = blockIdx.x;
    if (flag && !flag[r]) return;
    if (blk == 0 && threadIdx.x == 0) atomicAdd(&g_gs_bytes[1], (unsigned long long)(n * sizeof(VC) * (nvec + 2)));
    for (int i = threadIdx.x; i < nvec; i += kThreads) c[i] = from_d<VC>(coef[(long long)r * ldc + i]);
    __syncthreads();
    const long long e0 = (long long)blk * (kThreads * K) + (long long)threadIdx.x * K;
    const long long roff = (long long)r * n;
    VC acc[K];
    load_chunk<VC, K>(w + roff, e0, n, acc);
#pragma unroll 2
    for (int i = 0; i < nvec; ++i) {
        VC uv[K];
        load_chunk<VC, K>(U + i * ustride + roff, e0, n, uv);
        const VC ci = c[i];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            acc[k].x -= ci.x * uv[k].x - ci.y * uv[k].y;
            acc[k].y -= ci.x * uv[k].y + ci.y * uv[k].x;
        }
    }
    const R s = (R)scale[r];
    R a = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k].x *= s;
        acc[k].y *= s;
        a += acc[k].x * acc[k].x + acc[k].y * acc[k].y;
    }
    store_chunk<VC, K>(w + roff, e0, n, acc);
    a = warp_sum(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) shn[wid] = (double)a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) t += shn[q];
        npart[(long long)r * nblk + blk] = t;
    }
}

// out[r * ldo + i] = sum_blk partial[r][blk][i] for i < nv (fixed order); one block per (i, r)
__global__ void __launch_bounds__(kThreads) finalize2_kernel(const double2* __restrict__ partial, int nblk, int nv,
                                                             double2* __restrict__ out, int ldo,
                                                             const int* __restrict__ flag) {
    __shared__ double2 sh[kWarps];
    const int i = blockIdx.x, r = blockIdx.y;
    if (flag && !flag[r]) return;
    double2 a = make_double2(0, 0);
    for (int b = threadIdx.x; b < nblk; b += kThreads) {
        const double2 v = partial[((long long)r * nblk + b) * nv + i];
        a.x += v.x, a.y += v.y;
    }
    a.x = warp_sum(a.x);
    a.y = warp_sum(a.y);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < kWarps; ++q) s.x += sh[q].x, s.y += sh[q].y;
        out[(long long)r * ldo + i] = s;
    }
}

__global__ void __launch_bounds__(kThreads) finalize1_kernel(const double* __restrict__ part, int nblk,
                                                             double* __restrict__ out, const int* __restrict__ flag) {
    __shared__ double sh[kWarps];
    const int r = blockIdx.x;
    if (flag && !flag[r]) return;
    double a = 0;
    for (int b = threadIdx.x; b < nblk; b += kThreads) a += part[(long long)r * nblk + b];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < kWarps; ++q) s += sh[q];
        out[r] = s;
    }
}

__global__ void copy_norm_kernel(const double2* __restrict__ D, int ldd, double* out, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) out[r] = D[(long long)r * ldd].x;
}

// x[r] += sum_i c[r][i] U_i[r] (i < k[r]), or x[r] = that sum when overwrite is set; the sum
// in the basis precision, the update in FP64
template <typename VC>
__global__ void __launch_bounds__(kThreads) xupdate_kernel(const VC* __restrict__ U, long long ustride,
                                                           double2* __restrict__ x, long long n,
                                                           const double2* __restrict__ c, int ldc,
                                                           const int* __restrict__ k, int overwrite) {
    constexpr int K = Prec<VC>::K;
    __shared__ VC cs[kMaxV];
    const int r = blockIdx.y;
    const int kr = k[r];
    if (kr == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(&g_gs_bytes[2], (unsigned long long)(n * (sizeof(VC) * kr + 2 * sizeof(double2))));
    for (int i = threadIdx.x; i < kr; i += kThreads) cs[i] = from_d<VC>(c[(long long)r * ldc + i]);
    __syncthreads();
    const long long e0 = (long long)blockIdx.x * (kThreads * K) + (long long)threadIdx.x * K;
    const long long roff = (long long)r * n;
    VC acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = VC{};
    for (int i = 0; i < kr; ++i) {
        VC uv[K];
        load_chunk<VC, K>(U + i * ustride + roff, e0, n, uv);
        const VC ci = cs[i];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            acc[q].x += ci.x * uv[q].x - ci.y * uv[q].y;
            acc[q].y += ci.x * uv[q].y + ci.y * uv[q].x;
        }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const long long e = e0 + q;
        if (e < n) {
            double2 xv = overwrite ? make_double2(0.0, 0.0) : x[roff + e];
            xv.x += (double)acc[q].x;
            xv.y += (double)acc[q].y;
            x[roff + e] = xv;
        }
    }
}

// dst[r] = src[r] * s[r] (FP64 source), any destination precision
template <typename DC>
__global__ void scale_from64_kernel(const double2* __restrict__ src, DC* __restrict__ dst, long long n,
                                    const double* __restrict__ s) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long o = (long long)r * n + e;
    const double2 v = src[o];
    const double f = s[r];
    dst[o] = from_d<DC>(make_double2(v.x * f, v.y * f));
}

// out = a - b with b in FP32 (the FP32 matvec of a refinement correction)
__global__ void sub32_kernel(const double2* __restrict__ a, const float2* __restrict__ b, double2* __restrict__ out,
                             long long total) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    out[e] = make_double2(a[e].x - (double)b[e].x, a[e].y - (double)b[e].y);
}

__global__ void to32_kernel(const double2* __restrict__ a, float2* __restrict__ out, long long total) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    out[e] = make_float2((float)a[e].x, (float)a[e].y);
}

__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out,
                           long long total) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    out[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

// b~ = P^-1 b = b / (eps G_alpha); for the JM system (imu != NULL, nc = 24) the magnetization
// components 12..23 are divided by mu G_alpha instead
__global__ void precond_rhs_kernel(const double2* __restrict__ b, const double2* __restrict__ ieps,
                                   const double2* __restrict__ imu, double2* out, long long nv, int R, int nc,
                                   double g1, double g234) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv * nc * R) return;
    const long long vox = e % nv;
    int alpha = (int)((e / nv) % nc);
    const bool mag = imu && alpha >= 12;
    if (imu) alpha %= 12;
    const double ig = 1.0 / (comp_is_constant(alpha, imu ? 12 : nc) ? g1 : g234);
    const double2 v = b[e], c = mag ? imu[vox] : ieps[vox];
    out[e] = make_double2(ig * (v.x * c.x - v.y * c.y), ig * (v.x * c.y + v.y * c.x));
}

struct GState {
    int m;
    double2* H;      // [R][m+1][m]
    double2* cs;     // [R][m]  (real part used)
    double2* sn;     // [R][m]
    double2* g;      // [R][m+1]
    double2* y;      // [R][m]
    double2* D;      // [R][m+2]  inner products of the current pass, last = |w|^2
    double2* coef;   // [R][m+1]  projection coefficients of the current pass
    double* nrm;     // [R][m+1]  norms n_i of the stored vectors
    double* beta;    // [R]
    double* target;  // [R] absolute target for |g_{j+1}|
    double* scale;   // [R] rescale factor of the current pass
    double* sigma;   // [R] product of the rescale factors applied in this step
    double* F;       // [R] squared norm of the stored new vector
    int* active;     // [R]
    int* reflag;     // [R] second Gram-Schmidt pass needed
    int* k;          // [R] Arnoldi steps of the current cycle
    int* nactive;    // [1 + R]: the number of active right-hand sides, then their indices
    double2* shift;  // [R] shift of the Arnoldi matvec: w = (P^-1 A - shift) u_j
};

// start of a cycle: beta = ||r||, g = (beta, 0...), u_0 = r / beta (n_0 = 1), active = beta > target
__global__ void cycle_init_kernel(GState s, int R, const double* __restrict__ rn2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double beta = sqrt(fmax(rn2[r], 0.0));
    s.beta[r] = beta;
    for (int i = 0; i <= s.m; ++i) s.g[r * (s.m + 1) + i] = make_double2(0, 0);
    s.g[r * (s.m + 1)] = make_double2(beta, 0);
    s.k[r] = 0;
    const int act = (beta > s.target[r]) && beta > 0.0 && isfinite(beta);
    s.active[r] = act;
    s.scale[r] = act ? 1.0 / beta : 0.0;
    s.nrm[r * (s.m + 1)] = 1.0;
}

// after the first projection pass: H[:, j], coefficients, rescale 1/|w|
// (one block per right-hand side, a thread per entry i <= j)
__global__ void coef1_kernel(GState s, int R, int j) {
    const int r = blockIdx.x;
    if (r >= R || !s.active[r]) return;
    const int m = s.m;
    const double2* D = s.D + (long long)r * (m + 2);
    const double* n = s.nrm + (long long)r * (m + 1);
    double2* H = s.H + (long long)r * (m + 1) * m;
    const double nj = n[j];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 d = D[i];
        H[i * m + j] = make_double2(d.x / (n[i] * nj), d.y / (n[i] * nj));
        s.coef[(long long)r * (m + 1) + i] = make_double2(d.x / (n[i] * n[i]), d.y / (n[i] * n[i]));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double e = D[j + 1].x;
        const double sc = e > 0.0 ? 1.0 / sqrt(e) : 0.0;
        s.scale[r] = sc;
        s.sigma[r] = sc;
        // the matvec applied P^-1 A - shift: restore the diagonal entry, and shift the next
        // step by it (the Krylov space and H are those of P^-1 A; the shift only removes
        // the part of the new vector along u_j before the projections, which keeps the
        // Gram-Schmidt passes from cancelling most of it)
        double2 hjj = H[j * m + j];
        hjj.x += s.shift[r].x;
        hjj.y += s.shift[r].y;
        H[j * m + j] = hjj;
        if (isfinite(hjj.x) && isfinite(hjj.y)) s.shift[r] = hjj;
    }
}

// second pass where the rescaled new vector has squared length below 1/2
__global__ void reorth_kernel(GState s, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double f = s.F[r];
    const int fl = s.active[r] && f > 0.0 && f < 0.5;
    s.reflag[r] = fl;
    if (fl) s.scale[r] = 1.0 / sqrt(f);
}

// after the second projection pass: correction of H[:, j], coefficients, cumulative rescale
// (one block per right-hand side, a thread per entry i <= j)
__global__ void coef2_kernel(GState s, int R, int j) {
    const int r = blockIdx.x;
    if (r >= R || !s.reflag[r]) return;
    const int m = s.m;
    const double2* D = s.D + (long long)r * (m + 2);
    const double* n = s.nrm + (long long)r * (m + 1);
    double2* H = s.H + (long long)r * (m + 1) * m;
    const double f = n[j] * s.sigma[r];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 d = D[i];
        H[i * m + j].x += d.x / (n[i] * f);
        H[i * m + j].y += d.y / (n[i] * f);
        s.coef[(long long)r * (m + 1) + i] = make_double2(d.x / (n[i] * n[i]), d.y / (n[i] * n[i]));
    }
    __syncthreads();  // every thread has read sigma
    if (threadIdx.x == 0) s.sigma[r] *= s.scale[r];
}

// Givens step j for every active right-hand side
__global__ void givens_kernel(GState s, int R, int j) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !s.active[r]) return;
    const int m = s.m;
    double2* H = s.H + (long long)r * (m + 1) * m;
    double* n = s.nrm + (long long)r * (m + 1);
    const double nn = sqrt(fmax(s.F[r], 0.0));
    n[j + 1] = nn;
    const double hnext = (s.sigma[r] > 0.0 && n[j] > 0.0) ? nn / (s.sigma[r] * n[j]) : 0.0;
    for (int i = 0; i < j; ++i) {
        const double2 a = H[i * m + j], b = H[(i + 1) * m + j];
        const double c = s.cs[r * m + i].x;
        const double2 sn = s.sn[r * m + i];
        const double2 t = make_double2(c * a.x + sn.x * b.x - sn.y * b.y, c * a.y + sn.x * b.y + sn.y * b.x);
        const double2 bb = make_double2(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
        H[i * m + j] = t;
        H[(i + 1) * m + j] = bb;
    }
    const double2 a = H[j * m + j];
    const double b = hnext;
    const double aa = hypot(a.x, a.y);
    const double den = hypot(aa, b);
    double c;
    double2 sn;
    if (den == 0.0) {
        c = 1.0;
        sn = make_double2(0, 0);
    } else if (aa == 0.0) {
        c = 0.0;
        sn = make_double2(1.0, 0);
    } else {
        c = aa / den;
        sn = make_double2(a.x / aa * b / den, a.y / aa * b / den);  // (a/|a|) conj(b)/den, b real
    }
    s.cs[r * m + j] = make_double2(c, 0);
    s.sn[r * m + j] = sn;
    H[j * m + j] = make_double2(c * a.x + sn.x * b, c * a.y + sn.y * b);
    double2* g = s.g + r * (m + 1);
    const double2 gj = g[j];
    g[j + 1] = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
    s.k[r] = j + 1;
    const double res = hypot(g[j + 1].x, g[j + 1].y);
    if (res <= s.target[r] || hnext == 0.0 || !isfinite(res)) s.active[r] = 0;
}

// out[0] = number of active right-hand sides, out[1..] = their indices in increasing order
__global__ void count_active_kernel(const int* __restrict__ active, int R, int* out) {
    int c = 0;
    for (int r = 0; r < R; ++r)
        if (active[r]) out[1 + c++] = r;
    out[0] = c;
}

// back substitution H(0:k,0:k) y = g(0:k), then the update coefficients y_i / n_i
__global__ void trisolve_kernel(GState s, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int m = s.m, k = s.k[r];
    const double2* H = s.H + (long long)r * (m + 1) * m;
    const double2* g = s.g + r * (m + 1);
    const double* n = s.nrm + (long long)r * (m + 1);
    double2* y = s.y + r * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < k; ++q) {
            const double2 hq = H[i * m + q], yv = y[q];
            acc.x -= hq.x * yv.x - hq.y * yv.y;
            acc.y -= hq.x * yv.y + hq.y * yv.x;
        }
        const double2 d = H[i * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = dd > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                      : make_double2(0, 0);
    }
    for (int i = 0; i < k; ++i) {
        const double ni = n[i];
        y[i] = make_double2(y[i].x / ni, y[i].y / ni);
    }
}

// Residual of the cycle's least-squares solution in the Krylov basis: with the rotations
// Q = G_{k-1} ... G_0, r - A V_k y = V_{k+1} Q^H (0, ..., 0, g_k), so the coefficients of the
// stored vectors u_i = n_i v_i are t_i / n_i (i <= k); k1 = k + 1 vectors, 0 when k = 0.
__global__ void kresid_kernel(GState s, int R, int* __restrict__ k1) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int m = s.m, k = s.k[r];
    k1[r] = k > 0 ? k + 1 : 0;
    if (k == 0) return;
    double2* t = s.coef + (long long)r * (m + 1);
    const double* n = s.nrm + (long long)r * (m + 1);
    t[k] = s.g[r * (m + 1) + k];
    for (int i = k - 1; i >= 0; --i) {
        const double c = s.cs[r * m + i].x;
        const double2 sn = s.sn[r * m + i], b = t[i + 1];
        // (t_i, t_{i+1}) <- G_i^H (0, b) = (-sn b, c b)
        t[i] = make_double2(-(sn.x * b.x - sn.y * b.y), -(sn.x * b.y + sn.y * b.x));
        t[i + 1] = make_double2(c * b.x, c * b.y);
    }
    for (int i = 0; i <= k; ++i) t[i] = make_double2(t[i].x / n[i], t[i].y / n[i]);
}

// residual check of the outer loop; converged right-hand sides stay idle in later cycles
__global__ void check_kernel(const double* __restrict__ rn2, const double* __restrict__ bn2, double tol,
                             double eta_min, double* target, int* done, double* rel, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double rn = sqrt(fmax(rn2[r], 0.0)), bn = sqrt(fmax(bn2[r], 0.0));
    const double rr = bn > 0 ? rn / bn : 0.0;
    rel[r] = rr;
    done[r] = rr <= tol;
    target[r] = rr <= tol ? INFINITY : fmax(eta_min * rn, 0.5 * tol * bn);
}

// Forward-error estimate of the right-hand sides a sweep or cycle worked on (not done before it):
// err = ||dx|| / ||x|| * ||r_end|| / ||r_start||, dx the step's correction (Section IV-B residuals)
__global__ void err_est_kernel(const double* __restrict__ dn2, const double* __restrict__ xn2,
                               const double* __restrict__ rn2, const double* __restrict__ rn2_prev,
                               const int* __restrict__ done_prev, double* err, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || done_prev[r]) return;
    const double x = sqrt(fmax(xn2[r], 0.0)), d = sqrt(fmax(dn2[r], 0.0));
    const double r0 = sqrt(fmax(rn2_prev[r], 0.0)), r1 = sqrt(fmax(rn2[r], 0.0));
    err[r] = (x > 0.0 && r0 > 0.0) ? d / x * (r1 / r0) : 0.0;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Per (z, y) row: [x0, x1) spanning the voxels where chi, any right-hand side or the
// initial guess is non-zero ((0, 0) for a row with none).  One warp per row.
__global__ void support_rows_kernel(const double2* __restrict__ chi, const double2* __restrict__ b,
                                    const double2* __restrict__ guess, int ncomp, int nx, long long nrows,
                                    long long nv, int2* __restrict__ out) {
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    int lo = nx, hi = -1;
    for (int xx = lane; xx < nx; xx += 32) {
        const long long v = row * nx + xx;
        const double2 c = chi[v];
        bool nzv = c.x != 0.0 || c.y != 0.0;
        for (int q = 0; q < ncomp && !nzv; ++q) {
            const double2 t = b[(long long)q * nv + v];
            nzv = t.x != 0.0 || t.y != 0.0;
            if (guess && !nzv) {
                const double2 g = guess[(long long)q * nv + v];
                nzv = g.x != 0.0 || g.y != 0.0;
            }
        }
        if (nzv) {
            lo = min(lo, xx);
            hi = max(hi, xx);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) out[row] = hi >= lo ? make_int2(lo, hi + 1) : make_int2(0, 0);
}

// Support of a solve (Section III: unknowns where chi = 0 vanish when b does, since those
// rows of P^-1 A are the identity): rows of the grid restricted to the voxels where chi,
// b or the guess is non-zero; the full grid when that covers every voxel.
// chi: the material indicator (non-zero where the operator differs from the identity);
// ncomp: planes of nv values per right-hand side in b and the guess.
int build_support(vie_handle* h, int R, const double2* b, const double2* guess, Support* sp, cudaStream_t st,
                  const double2* chi, int ncomp) {
    const long long nrows = (long long)h->ny * h->nz;
    VIE_TRY(ws_reserve(h, h->support_ws, sizeof(int4) * (size_t)nrows + sizeof(int2) * (size_t)nrows));
    int4* rows = static_cast<int4*>(h->support_ws.ptr);
    int2* span = reinterpret_cast<int2*>(rows + nrows);
    const unsigned g = (unsigned)((nrows + 7) / 8);
    VIE_KLAUNCH("support_rows", st,
                support_rows_kernel<<<g, 256, 0, st>>>(chi, b, guess, R * ncomp, h->nx, nrows, (long long)h->nv,
                                                       span));
    VIE_CHECK_LAUNCH();
    std::vector<int2> hs(nrows);
    VIE_CUDA(cudaMemcpyAsync(hs.data(), span, sizeof(int2) * nrows, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    std::vector<int4> hr(nrows);
    long long off = 0;
    for (long long i = 0; i < nrows; ++i) {
        hr[i] = make_int4(hs[i].x, hs[i].y, (int)off, 0);
        off += hs[i].y - hs[i].x;
    }
    sp->ns = off;
    sp->rows = nullptr;
    if (off == (long long)h->nv || off == 0) return VIE_OK;
    if (off > 0x7fffffffLL) {
        set_error("support too large");
        return VIE_EINVAL;
    }
    VIE_CUDA(cudaMemcpyAsync(rows, hr.data(), sizeof(int4) * nrows, cudaMemcpyHostToDevice, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    sp->rows = rows;
    return VIE_OK;
}

// Arnoldi steps per chunk of a cycle (run_cycle), and chunks at most (restart <= 128)
constexpr int kChunk = 8;
constexpr int kMaxChunks = (kMaxV + kChunk - 1) / kChunk;

// A captured piece of a GMRES cycle (run_cycle) and the launch records of its kernels.
struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<CapRec> recs;
    bool replayed = false;  // replayed since its device times were last harvested
    ~CycleGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        stats_capture_release(recs);
    }
};

struct Solver {
    vie_handle* h;
    cudaStream_t st = nullptr;
    bool use_graph = false;
    bool jm = false;  // the full JM-VIE system (two currents per voxel)
    // per matvec precision (VIE_FP64, VIE_FP32, VIE_BF16X3): the chunks of a cycle, then its end
    CycleGraph graph[3][kMaxChunks + 1];
    int* pinned = nullptr;                // [kMaxChunks] active counts after each chunk (pinned host memory)
    cudaEvent_t chunk_ev[kMaxChunks] = {};  // end of each queued chunk
    ~Solver() {  // nothing of this solve may still run when its graphs and events go
        if (st) cudaStreamSynchronize(st);
        for (auto& e : chunk_ev)
            if (e) cudaEventDestroy(e);
    }
    int R, m;
    long long n;
    int nblk;
    double2* partial;  // [R][nblk][m+2]
    double* npart;     // [R][nblk]
    GState gs;

    template <typename VC>
    int dots(const VC* U, long long ustride, const VC* w, int nvec, const int* flag) {
        const dim3 g1(nblk, R);
        VIE_KLAUNCH("gs_dots", st,
                    gs_dots_kernel<VC><<<g1, kThreads, 0, st>>>(U, ustride, w, n, nvec, partial, nblk, flag));
        const dim3 g2(nvec + 1, R);
        VIE_KLAUNCH("gs_finalize", st,
                    finalize2_kernel<<<g2, kThreads, 0, st>>>(partial, nblk, nvec + 1, gs.D, m + 2, flag));
        VIE_CHECK_LAUNCH();
        return VIE_OK;
    }
    template <typename VC>
    int update(const VC* U, long long ustride, VC* w, int nvec, const int* flag) {
        const dim3 g1(nblk, R);
        VIE_KLAUNCH("gs_update", st,
                    gs_update_kernel<VC><<<g1, kThreads, 0, st>>>(U, ustride, w, n, nvec, gs.coef, m + 1, gs.scale,
                                                                 npart, nblk, flag));
        VIE_KLAUNCH("gs_norm", st, finalize1_kernel<<<R, kThreads, 0, st>>>(npart, nblk, gs.F, flag));
        VIE_CHECK_LAUNCH();
        return VIE_OK;
    }
    Support sp;        // support of the solver's vectors
    void* mv_tmp;      // full-grid scratch of matvec_support
    // squared 2-norm per right-hand side of an FP64 vector batch of length len (default n) into out[R]
    int norm2_64(const double2* v, double* out, long long len = 0) {
        if (len <= 0) len = n;
        const int nb = (int)((len + kThreads * Prec<double2>::K - 1) / (kThreads * Prec<double2>::K));
        const dim3 g1(nb, R);
        VIE_KLAUNCH("norm64", st,
                    gs_dots_kernel<double2><<<g1, kThreads, 0, st>>>(nullptr, 0, v, len, 0, partial, nb, nullptr));
        const dim3 g2(1, R);
        VIE_KLAUNCH("norm64_finalize", st,
                    finalize2_kernel<<<g2, kThreads, 0, st>>>(partial, nb, 1, gs.D, m + 2, nullptr));
        VIE_KLAUNCH("norm64_copy", st, copy_norm_kernel<<<(R + 127) / 128, 128, 0, st>>>(gs.D, m + 2, out, R));
        VIE_CHECK_LAUNCH();
        return VIE_OK;
    }
};

// Arnoldi steps [j0, j1) of a GMRES(m) cycle from the residual r64 (squared norms rn2), enqueued
// on the stream with no host read inside: every step works on the device's list of active
// right-hand sides (count_active before each step), so a step after every right-hand side has
// stopped finds an empty list and its kernels return at once.  The first chunk starts the cycle;
// every chunk ends by counting the right-hand sides still active.
template <typename VC>
int enqueue_steps(Solver& S, VC* U, const double2* r64, const double* rn2, int precision, int j0, int j1) {
    vie_handle* h = S.h;
    const int R = S.R;
    const long long n = S.n, ustride = (long long)R * n;
    cudaStream_t st = S.st;
    const unsigned gr = (unsigned)((R + 127) / 128);
    if (j0 == 0) {
        VIE_KLAUNCH("cycle_init", st, cycle_init_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs, R, rn2));
        const dim3 ge((unsigned)((n + 255) / 256), R);
        VIE_KLAUNCH("basis_init", st, scale_from64_kernel<VC><<<ge, 256, 0, st>>>(r64, U, n, S.gs.scale));
        VIE_CHECK_LAUNCH();
    }
    for (int j = j0; j < j1; ++j) {
        VIE_KLAUNCH("count_active", st, count_active_kernel<<<1, 1, 0, st>>>(S.gs.active, R, S.gs.nactive));
        VC* uj = U + j * ustride;
        VC* w = U + (j + 1) * ustride;
        // only the active right-hand sides (the others' w is never read)
        if (S.jm)  // every right-hand side transformed (the others' w is never read)
            VIE_TRY(jm_matvec_support(h, R, uj, w, VIE_OP_PA, S.sp, S.mv_tmp, st, S.gs.shift,
                                      sizeof(VC) == sizeof(double2) ? VIE_FP64 : VIE_FP32));
        else
            VIE_TRY(matvec_support(h, R, uj, w, precision, VIE_OP_PA, S.sp, S.mv_tmp, st, S.gs.shift, nullptr,
                                   S.gs.nactive + 1, S.gs.nactive));
        VIE_TRY(S.dots<VC>(U, ustride, w, j + 1, S.gs.active));
        VIE_KLAUNCH("arnoldi_coef", st, coef1_kernel<<<R, 128, 0, st>>>(S.gs, R, j));
        VIE_TRY(S.update<VC>(U, ustride, w, j + 1, S.gs.active));
        VIE_KLAUNCH("arnoldi_reorth", st, reorth_kernel<<<gr, 128, 0, st>>>(S.gs, R));
        VIE_TRY(S.dots<VC>(U, ustride, w, j + 1, S.gs.reflag));
        VIE_KLAUNCH("arnoldi_coef", st, coef2_kernel<<<R, 128, 0, st>>>(S.gs, R, j));
        VIE_TRY(S.update<VC>(U, ustride, w, j + 1, S.gs.reflag));
        VIE_KLAUNCH("givens", st, givens_kernel<<<gr, 128, 0, st>>>(S.gs, R, j));
        VIE_CHECK_LAUNCH();
    }
    VIE_KLAUNCH("count_active", st, count_active_kernel<<<1, 1, 0, st>>>(S.gs.active, R, S.gs.nactive));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

// end of a cycle: H y = g, x64 += V y
template <typename VC>
int enqueue_finish(Solver& S, VC* U, double2* x64) {
    const int R = S.R, m = S.m;
    const long long n = S.n, ustride = (long long)R * n;
    cudaStream_t st = S.st;
    const unsigned gr = (unsigned)((R + 127) / 128);
    VIE_KLAUNCH("trisolve", st, trisolve_kernel<<<gr, 128, 0, st>>>(S.gs, R));
    const dim3 gx((unsigned)((n + kThreads * Prec<VC>::K - 1) / (kThreads * Prec<VC>::K)), R);
    VIE_KLAUNCH("solution_update", st,
                xupdate_kernel<VC><<<gx, kThreads, 0, st>>>(U, ustride, x64, n, S.gs.y, m, S.gs.k, 0));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

// Runs `enqueue` on the stream: directly, or (S.use_graph) by replaying the CUDA graph G, which
// is captured from `enqueue` on first use (the buffers it touches stay the same for the solve).
template <class F>
int run_graph(Solver& S, CycleGraph& G, F enqueue) {
    cudaStream_t st = S.st;
    if (!S.use_graph) return enqueue();
    if (!G.exec) {
        cudaGraph_t graph = nullptr;
        VIE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        stats_capture_begin(&G.recs);
        const int rc = enqueue();
        stats_capture_end();
        const cudaError_t ec = cudaStreamEndCapture(st, &graph);
        if (rc < 0 || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (rc < 0) return rc;
            set_error(std::string("cycle graph capture failed: ") + cudaGetErrorString(ec));
            return VIE_EDEVICE;
        }
        const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            G.exec = nullptr;
            set_error(std::string("cycle graph instantiation failed: ") + cudaGetErrorString(ei));
            return VIE_EDEVICE;
        }
    }
    VIE_CUDA(cudaGraphLaunch(G.exec, st));
    stats_graph_replayed(G.recs);
    G.replayed = true;
    return VIE_OK;
}

// One GMRES(m) cycle from r64: the Arnoldi steps in chunks of kChunk, each (with S.use_graph) a
// CUDA graph replayed every cycle.  The host keeps one chunk queued ahead of the one it waits
// for, and stops queueing once a finished chunk left no right-hand side active, so the GPU does
// not wait for the host and at most one chunk of empty steps runs after the last right-hand side
// stops.  Then x64 += V y and the host reads each right-hand side's step count k.
// *still = number of right-hand sides that ended the cycle above their target.
template <typename VC>
int run_cycle(Solver& S, VC* U, double2* x64, const double2* r64, const double* rn2, int precision, int* it_rhs,
              int* mv_count, int* still) {
    const int R = S.R, m = S.m;
    cudaStream_t st = S.st;
    const int nch = (m + kChunk - 1) / kChunk;
    CycleGraph* G = S.graph[precision];
    int queued = 0;
    auto queue = [&](int c) -> int {
        const int j0 = c * kChunk, j1 = std::min(m, j0 + kChunk);
        VIE_TRY(run_graph(S, G[c], [&] { return enqueue_steps<VC>(S, U, r64, rn2, precision, j0, j1); }));
        VIE_CUDA(cudaMemcpyAsync(S.pinned + c, S.gs.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaEventRecord(S.chunk_ev[c], st));
        ++queued;
        return VIE_OK;
    };
    VIE_TRY(queue(0));
    for (int c = 0; c < nch; ++c) {
        if (queued < nch && queued == c + 1) VIE_TRY(queue(c + 1));  // keep one chunk ahead
        VIE_CUDA(cudaEventSynchronize(S.chunk_ev[c]));
        if (S.pinned[c] == 0) break;  // every right-hand side stopped in chunk c (or before)
    }
    VIE_TRY(run_graph(S, G[kMaxChunks], [&] { return enqueue_finish<VC>(S, U, x64); }));
    std::vector<int> k(R);
    int act = 0;
    VIE_CUDA(cudaMemcpyAsync(k.data(), S.gs.k, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaMemcpyAsync(&act, S.gs.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    if (S.use_graph)
        for (int c = 0; c <= kMaxChunks; ++c)
            if (G[c].replayed) {
                stats_graph_harvest(G[c].recs);
                G[c].replayed = false;
            }
    int kmax = 0;
    for (int r = 0; r < R; ++r) {
        it_rhs[r] += k[r];
        kmax = std::max(kmax, k[r]);
    }
    *mv_count += kmax;  // matvecs that transformed at least one right-hand side
    *still = act;
    return VIE_OK;
}

// r64 = residual of the last cycle from its Krylov basis (no matvec), rn2 = its squared norms
template <typename VC>
int krylov_residual(Solver& S, const VC* U, double2* r64, double* rn2, int* k1) {
    const int R = S.R;
    const long long n = S.n, ustride = (long long)R * n;
    cudaStream_t st = S.st;
    VIE_KLAUNCH("krylov_resid_coef", st, kresid_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs, R, k1));
    const dim3 gx((unsigned)((n + kThreads * Prec<VC>::K - 1) / (kThreads * Prec<VC>::K)), R);
    VIE_KLAUNCH("krylov_residual", st,
                xupdate_kernel<VC><<<gx, kThreads, 0, st>>>(U, ustride, r64, n, S.gs.coef, S.m + 1, k1, 1));
    VIE_CHECK_LAUNCH();
    return S.norm2_64(r64, rn2);
}

}  // namespace

int solve_device(vie_handle* h, int R, const double2* b, double2* x, double tol, int m, int maxit, int mode,
                 int flags, vie_solve_info* info, cudaStream_t st, bool jm) {
    if (m + 2 > kMaxV) {
        set_error("restart above 128 is not supported");
        return VIE_EINVAL;
    }
    h->fcache_valid = 0;  // a new solve replaces the point kept for vie_fields
    // the JM system (FP64, or FP32 inner solves with FP64 refinement): unknowns per voxel 24 = two
    // currents of 12, copied to and from the support as 2R vectors of 12 components; no point is
    // kept for vie_fields
    if (jm && mode != VIE_SOLVE_FP64 && mode != VIE_SOLVE_FP32_REFINE) {
        set_error("the JM-VIE system is solved in FP64 or FP32 with FP64 refinement");
        return VIE_EINVAL;
    }
    if (jm && !h->mu64) VIE_TRY(jm_materials(h, nullptr, nullptr, st));
    const int ncs = jm ? 24 : h->nc;  // unknowns per voxel of the system
    const int Rv = jm ? 2 * R : R;     // right-hand sides as the support copies see them
    const bool keep = !(flags & 4) && !jm;
    // vectors live on the support of the solve: [R][ncs][ns] (ncs = 12 PWL, 3 PWC, 24 JM)
    Support sp;
    VIE_TRY(build_support(h, R, b, (flags & 1) ? x : nullptr, &sp, st, jm ? h->jmsup64 : h->chi64, ncs));
    const long long nfull = (long long)ncs * (long long)h->nv;
    if (sp.ns == 0) {  // chi = 0 everywhere and b = 0: x = 0
        VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * (size_t)(R * nfull), st));
        VIE_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; info && r < R; ++r) info[r] = vie_solve_info{1, 0, 0, 0, 0, 0.0, (flags & 2) ? 0.0 : -1.0, 0.0};
        return VIE_OK;
    }
    const long long n = (long long)ncs * sp.ns;
    const bool mixed = mode == VIE_SOLVE_FP32_REFINE || mode == VIE_SOLVE_BF16X3_REFINE;
    const int inner = mode == VIE_SOLVE_BF16X3_REFINE ? VIE_BF16X3 : VIE_FP32;  // matvec of the inner GMRES
    const size_t vc = mixed ? sizeof(float2) : sizeof(double2);
    const int kpt = mixed ? Prec<float2>::K : Prec<double2>::K;
    const int nblk = (int)((n + kThreads * kpt - 1) / (kThreads * kpt));
    const int nblk64 = (int)((nfull + kThreads * Prec<double2>::K - 1) / (kThreads * Prec<double2>::K));
    const int nbmax = nblk > nblk64 ? nblk : nblk64;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oU = take(vc * (size_t)(m + 1) * R * n);
    const size_t oR = take(sizeof(double2) * (size_t)R * n);
    const size_t oBt = take(sizeof(double2) * (size_t)R * n);
    const size_t oT = take(sizeof(double2) * (size_t)R * n);
    const size_t oX = take(sizeof(double2) * (size_t)R * n);
    const size_t oFull = take(2 * sizeof(double2) * (size_t)R * nfull);  // full-grid scratch
    const size_t oPart = take(sizeof(double2) * (size_t)R * nbmax * (m + 2));
    const size_t oNp = take(sizeof(double) * (size_t)R * nbmax);
    const size_t oH = take(sizeof(double2) * (size_t)R * (m + 1) * m);
    const size_t oCs = take(sizeof(double2) * (size_t)R * m);
    const size_t oSn = take(sizeof(double2) * (size_t)R * m);
    const size_t oG = take(sizeof(double2) * (size_t)R * (m + 1));
    const size_t oY = take(sizeof(double2) * (size_t)R * m);
    const size_t oD = take(sizeof(double2) * (size_t)R * (m + 2));
    const size_t oCo = take(sizeof(double2) * (size_t)R * (m + 1));
    const size_t oNrm = take(sizeof(double) * (size_t)R * (m + 1));
    const size_t oBeta = take(sizeof(double) * R);
    const size_t oTarget = take(sizeof(double) * R);
    const size_t oScale = take(sizeof(double) * R);
    const size_t oSigma = take(sizeof(double) * R);
    const size_t oF = take(sizeof(double) * R);
    const size_t oAct = take(sizeof(int) * R);
    const size_t oRe = take(sizeof(int) * R);
    const size_t oK = take(sizeof(int) * R);
    const size_t oNact = take(sizeof(int) * (R + 1));
    const size_t oBn = take(sizeof(double) * R);
    const size_t oRn = take(sizeof(double) * R);
    const size_t oDone = take(sizeof(int) * R);
    const size_t oRel = take(sizeof(double) * R);
    const size_t oK1 = take(sizeof(int) * R);
    const size_t oShift = take(sizeof(double2) * R);
    const size_t oRs0 = take(sizeof(double2) * (size_t)R * n);  // residual at the start of the last sweep
    const size_t oXs0 = take(sizeof(double2) * (size_t)R * n);  // solution at the start of the last sweep
    const size_t oDn = take(sizeof(double) * R);
    const size_t oXn = take(sizeof(double) * R);
    const size_t oRnp = take(sizeof(double) * R);  // squared residual norms at the start of a step
    const size_t oDonep = take(sizeof(int) * R);   // converged before that step
    const size_t oErr = take(sizeof(double) * R);  // forward-error estimates
    VIE_TRY(ws_reserve(h, h->solve_ws, off));
    char* base = static_cast<char*>(h->solve_ws.ptr);
    Solver S;
    S.h = h;
    S.st = st;
    // CUDA graphs for the cycles unless flags bit 3 asks for direct launches; the legacy and
    // per-thread default streams cannot be captured
    S.use_graph = !(flags & 8) && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    S.jm = jm;
    // the largest spectrum scratch any matvec of this solve takes (FP64; the JM products transform
    // 2R vectors), reserved before the first cycle is captured so that no later reservation moves
    // the buffer under the graph; the JM operator's product scratch and K spectra likewise
    VIE_TRY(ws_reserve(h, h->fft_ws, matvec_workspace_bytes(h, Rv, VIE_FP64)));
    if (jm) {
        VIE_TRY(ws_reserve(h, h->jm_ws, 2 * sizeof(double2) * (size_t)R * 24 * h->nv));
        VIE_TRY(k_octants(h, st));
    }
    dev_bytes_ptr("zpass_block_f32");  // looks the counters' address up outside any capture
    if (mode == VIE_SOLVE_FP32_REFINE) VIE_TRY(matvec_tune(h, Rv, VIE_FP32, st));
    if (mode == VIE_SOLVE_FP32_REFINE && jm) VIE_TRY(matvec_tune(h, Rv, VIE_FP32, st, VIE_OP_K));
    if (mode == VIE_SOLVE_BF16X3_REFINE) VIE_TRY(matvec_tune(h, R, VIE_BF16X3, st));
    S.R = R;
    S.m = m;
    S.n = n;
    S.nblk = nblk;
    S.sp = sp;
    S.mv_tmp = base + oFull;
    S.partial = reinterpret_cast<double2*>(base + oPart);
    S.npart = reinterpret_cast<double*>(base + oNp);
    S.gs.m = m;
    S.gs.H = reinterpret_cast<double2*>(base + oH);
    S.gs.cs = reinterpret_cast<double2*>(base + oCs);
    S.gs.sn = reinterpret_cast<double2*>(base + oSn);
    S.gs.g = reinterpret_cast<double2*>(base + oG);
    S.gs.y = reinterpret_cast<double2*>(base + oY);
    S.gs.D = reinterpret_cast<double2*>(base + oD);
    S.gs.coef = reinterpret_cast<double2*>(base + oCo);
    S.gs.nrm = reinterpret_cast<double*>(base + oNrm);
    S.gs.beta = reinterpret_cast<double*>(base + oBeta);
    S.gs.target = reinterpret_cast<double*>(base + oTarget);
    S.gs.scale = reinterpret_cast<double*>(base + oScale);
    S.gs.sigma = reinterpret_cast<double*>(base + oSigma);
    S.gs.F = reinterpret_cast<double*>(base + oF);
    S.gs.active = reinterpret_cast<int*>(base + oAct);
    S.gs.reflag = reinterpret_cast<int*>(base + oRe);
    S.gs.k = reinterpret_cast<int*>(base + oK);
    S.gs.nactive = reinterpret_cast<int*>(base + oNact);
    S.gs.shift = reinterpret_cast<double2*>(base + oShift);
    VIE_CUDA(cudaMemsetAsync(S.gs.shift, 0, sizeof(double2) * R, st));  // the first step is unshifted
    double2* r64 = reinterpret_cast<double2*>(base + oR);
    double2* bt = reinterpret_cast<double2*>(base + oBt);
    double2* t64 = reinterpret_cast<double2*>(base + oT);
    double2* xs = reinterpret_cast<double2*>(base + oX);  // solution on the support
    double2* full0 = reinterpret_cast<double2*>(base + oFull);
    double2* full1 = full0 + (size_t)R * nfull;
    double* bn2 = reinterpret_cast<double*>(base + oBn);
    double* rn2 = reinterpret_cast<double*>(base + oRn);
    int* done = reinterpret_cast<int*>(base + oDone);
    double* rel = reinterpret_cast<double*>(base + oRel);
    int* k1 = reinterpret_cast<int*>(base + oK1);
    // pinned host words for the chunk counts: one buffer per host thread, kept for the thread's
    // lifetime (a solve is synchronous on its thread), so that solves do not allocate and free
    // pinned memory, which would synchronise the device under other streams' work
    struct PinnedCounts {
        int* p = nullptr;
        ~PinnedCounts() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local PinnedCounts pinned;
    if (!pinned.p) VIE_CUDA(cudaMallocHost(&pinned.p, sizeof(int) * kMaxChunks));
    S.pinned = pinned.p;
    struct SyncGuard {  // the copies into the pinned words have finished when the solve returns
        cudaStream_t s;
        ~SyncGuard() { cudaStreamSynchronize(s); }
    } guard{st};
    for (auto& e : S.chunk_ev) VIE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

    const long long total = (long long)R * n, total_full = (long long)R * nfull;
    const unsigned gt = (unsigned)((total + 255) / 256);
    const unsigned gtf = (unsigned)((total_full + 255) / 256);
    const unsigned gr = (unsigned)((R + 127) / 128);
    const double dV = h->dx * h->dy * h->dz;
    VIE_KLAUNCH("precond_rhs", st,
                precond_rhs_kernel<<<gtf, 256, 0, st>>>(b, h->ieps64, jm ? h->imu64 : nullptr, full0,
                                                        (long long)h->nv, R, ncs, dV, dV / 12.0));
    VIE_CHECK_LAUNCH();
    VIE_TRY(support_gather(h, Rv, full0, bt, VIE_FP64, sp, st));
    VIE_TRY(S.norm2_64(bt, bn2));
    if (flags & 1)
        VIE_TRY(support_gather(h, Rv, x, xs, VIE_FP64, sp, st));
    else
        VIE_CUDA(cudaMemsetAsync(xs, 0, sizeof(double2) * total, st));
    {
        // NaN or Inf in b or in the guess: rejected before any iteration (the squared norms
        // of P^-1 b and of the guess on the support are then not finite)
        double* xn0 = reinterpret_cast<double*>(base + oXn);
        VIE_TRY(S.norm2_64(xs, xn0));
        std::vector<double> hb(R), hx(R);
        VIE_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaMemcpyAsync(hx.data(), xn0, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r)
            if (!std::isfinite(hb[r]) || !std::isfinite(hx[r])) {
                set_error("right-hand side " + std::to_string(r) + (std::isfinite(hb[r]) ? ": the initial guess" : "") +
                          " holds a NaN or Inf");
                return VIE_EINVAL;
            }
    }

    if (keep) VIE_TRY(ws_reserve(h, h->fcache_ws, 2 * sizeof(double2) * (size_t)R * nfull));

    std::vector<int> it_rhs(R, 0), hdone(R, 0);
    std::vector<double> hrel(R, 0.0), htrue(R, -1.0);
    int mv64 = 0, mv32 = 0, sweeps = 0;
    const double eta_min = mixed ? 2e-5 : 0.0;
    bool x_is_zero = !(flags & 1);
    bool all = false;
    double2* rs0 = reinterpret_cast<double2*>(base + oRs0);
    double2* xs0 = reinterpret_cast<double2*>(base + oXs0);
    double* dn2 = reinterpret_cast<double*>(base + oDn);
    double* xn2 = reinterpret_cast<double*>(base + oXn);
    bool have_r0 = false;
    double* rn2_prev = reinterpret_cast<double*>(base + oRnp);
    int* done_prev = reinterpret_cast<int*>(base + oDonep);
    double* err = reinterpret_cast<double*>(base + oErr);
    VIE_CUDA(cudaMemsetAsync(err, 0, sizeof(double) * R, st));
    bool step_open = false;  // a sweep (mixed) or cycle (FP64) started from xs0 / rn2_prev / done_prev
    // start of a refinement sweep or FP64 cycle: keep its starting point (the refinement's residual
    // update and the error estimate use it)
    auto open_step = [&]() -> int {
        if (mixed) {
            VIE_CUDA(cudaMemcpyAsync(rs0, r64, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
            have_r0 = !x_is_zero;
        }
        VIE_CUDA(cudaMemcpyAsync(xs0, xs, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
        VIE_CUDA(cudaMemcpyAsync(rn2_prev, rn2, sizeof(double) * R, cudaMemcpyDeviceToDevice, st));
        VIE_CUDA(cudaMemcpyAsync(done_prev, done, sizeof(int) * R, cudaMemcpyDeviceToDevice, st));
        step_open = true;
        return VIE_OK;
    };
    // after the residual of the step's end point: the error estimate of the right-hand sides it moved
    auto close_step = [&]() -> int {
        if (!step_open) return VIE_OK;
        VIE_KLAUNCH("err_est", st, sub_kernel<<<gt, 256, 0, st>>>(xs, xs0, t64, total));
        VIE_TRY(S.norm2_64(t64, dn2));
        VIE_TRY(S.norm2_64(xs, xn2));
        VIE_KLAUNCH("err_est", st, err_est_kernel<<<gr, 128, 0, st>>>(dn2, xn2, rn2, rn2_prev, done_prev, err, R));
        VIE_CHECK_LAUNCH();
        step_open = false;
        return VIE_OK;
    };
    // Refinement residual.  The first one (after the first sweep) is b - A x with the FP64
    // matvec.  Later ones update the previous sweep's residual, r - A d with d the sweep's
    // correction, when |d| <= min(1e-3, 1e5 tol) |x| for every right-hand side: then A d in
    // FP32 carries an error of order 1e-7 |A| |d|, far below the FP64 rounding of r at the
    // tolerance, and the FP64 matvec is replaced by an FP32 one.
    auto residual = [&]() -> int {
        bool done_update = false;
        if (x_is_zero) {
            VIE_CUDA(cudaMemcpyAsync(r64, bt, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
            done_update = true;
        } else if (mixed && have_r0) {
            VIE_KLAUNCH("refine_correction", st, sub_kernel<<<gt, 256, 0, st>>>(xs, xs0, t64, total));
            VIE_TRY(S.norm2_64(t64, dn2));
            VIE_TRY(S.norm2_64(xs, xn2));
            std::vector<double> hd(R), hx(R);
            VIE_CUDA(cudaMemcpyAsync(hd.data(), dn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaMemcpyAsync(hx.data(), xn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaStreamSynchronize(st));
            const double ratio = std::min(1e-3, 1e5 * tol);
            bool small = true;
            for (int r = 0; r < R; ++r) small = small && hd[r] <= ratio * ratio * hx[r];
            if (small) {
                float2* d32 = reinterpret_cast<float2*>(base + oU);
                float2* ad32 = d32 + total;
                VIE_KLAUNCH("refine_correction", st, to32_kernel<<<gt, 256, 0, st>>>(t64, d32, total));
                if (jm)
                    VIE_TRY(jm_matvec_support(h, R, d32, ad32, VIE_OP_PA, sp, S.mv_tmp, st, nullptr, VIE_FP32));
                else
                    VIE_TRY(matvec_support(h, R, d32, ad32, VIE_FP32, VIE_OP_PA, sp, S.mv_tmp, st));
                ++mv32;
                VIE_KLAUNCH("residual_sub", st, sub32_kernel<<<gt, 256, 0, st>>>(rs0, ad32, r64, total));
                done_update = true;
            }
        }
        if (!done_update) {
            // the matvec also leaves (N - G) x on the full grid, kept with x for vie_fields
            double2* cx = keep ? static_cast<double2*>(h->fcache_ws.ptr) : nullptr;
            if (jm)
                VIE_TRY(jm_matvec_support(h, R, xs, t64, VIE_OP_PA, sp, S.mv_tmp, st, nullptr, VIE_FP64));
            else
                VIE_TRY(matvec_support(h, R, xs, t64, VIE_FP64, VIE_OP_PA, sp, S.mv_tmp, st, nullptr,
                                       keep ? cx + (size_t)R * nfull : nullptr));
            ++mv64;
            VIE_KLAUNCH("residual_sub", st, sub_kernel<<<gt, 256, 0, st>>>(bt, t64, r64, total));
            if (keep) {
                VIE_TRY(support_scatter(h, R, xs, cx, VIE_FP64, sp, st));
                h->fcache_R = R;
                h->fcache_valid = 1;
            }
        }
        VIE_TRY(S.norm2_64(r64, rn2));
        VIE_KLAUNCH("residual_check", st,
                    check_kernel<<<gr, 128, 0, st>>>(rn2, bn2, tol, eta_min, S.gs.target, done, rel, R));
        VIE_CHECK_LAUNCH();
        VIE_CUDA(cudaMemcpyAsync(hdone.data(), done, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaMemcpyAsync(hrel.data(), rel, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        all = true;
        for (int r = 0; r < R; ++r) all = all && hdone[r];
        return VIE_OK;
    };
    // Plain mode: the FP64 residual is recomputed at every restart.  Mixed mode: each
    // refinement sweep takes the FP64 residual, then runs FP32 GMRES cycles on the
    // correction until every right-hand side is below its sweep target, restarting from
    // the residual carried by the Krylov basis (no FP64 matvec inside a sweep).
    int cyc = 0;
    while (cyc < maxit) {
        VIE_TRY(residual());
        VIE_TRY(close_step());
        if (all) break;
        VIE_TRY(open_step());
        if (mixed) {
            ++sweeps;
            float2* U32 = reinterpret_cast<float2*>(base + oU);
            for (;;) {
                int still = 0;
                VIE_TRY(run_cycle<float2>(S, U32, xs, r64, rn2, inner, it_rhs.data(), &mv32, &still));
                ++cyc;
                x_is_zero = false;
                if (still == 0 || cyc >= maxit) break;
                VIE_TRY(krylov_residual<float2>(S, U32, r64, rn2, k1));
            }
        } else {
            int still = 0;
            VIE_TRY(run_cycle<double2>(S, reinterpret_cast<double2*>(base + oU), xs, r64, rn2, VIE_FP64,
                                       it_rhs.data(), &mv64, &still));
            ++cyc;
            x_is_zero = false;
        }
    }
    if (!all) {  // residual of the last iterate when the cycle cap was hit
        VIE_TRY(residual());
        VIE_TRY(close_step());
    }
    std::vector<double> herr(R, 0.0);
    VIE_CUDA(cudaMemcpyAsync(herr.data(), err, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    VIE_TRY(support_scatter(h, Rv, xs, x, VIE_FP64, sp, st));
    if (flags & 2) {
        // unpreconditioned residual ||b - A x|| / ||b|| on the full grid; its convolution at
        // the final x replaces the cached one for vie_fields
        double2* cx = keep ? static_cast<double2*>(h->fcache_ws.ptr) : nullptr;
        if (jm)
            VIE_TRY(jm_matvec_full(h, R, x, full0, VIE_OP_A, st));
        else
            VIE_TRY(matvec_support(h, R, x, full0, VIE_FP64, VIE_OP_A, Support{}, S.mv_tmp, st, nullptr,
                                   keep ? cx + (size_t)R * nfull : nullptr));
        ++mv64;
        if (keep) {
            VIE_CUDA(cudaMemcpyAsync(cx, x, sizeof(double2) * (size_t)R * nfull, cudaMemcpyDeviceToDevice, st));
            h->fcache_R = R;
            h->fcache_valid = 1;
        }
        VIE_KLAUNCH("residual_sub", st, sub_kernel<<<gtf, 256, 0, st>>>(b, full0, full1, total_full));
        VIE_TRY(S.norm2_64(full1, rn2, nfull));
        VIE_TRY(S.norm2_64(b, bn2, nfull));
        std::vector<double> a(R), c(R);
        VIE_CUDA(cudaMemcpyAsync(a.data(), rn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaMemcpyAsync(c.data(), bn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) htrue[r] = c[r] > 0 ? std::sqrt(a[r] / c[r]) : 0.0;
    }
    int rc = VIE_OK;
    for (int r = 0; r < R; ++r) {
        const bool conv = hrel[r] <= tol;
        if (!conv) rc = VIE_NOT_CONVERGED;
        if (info) {
            info[r].converged = conv;
            info[r].iterations = it_rhs[r];
            info[r].fp64_matvecs = mv64;
            info[r].fp32_matvecs = mv32;
            info[r].refinements = sweeps;
            info[r].resid = hrel[r];
            info[r].true_resid = htrue[r];
            info[r].err_est = herr[r];
        }
    }
    return rc;
}

int solve_device_bytes(double out[3], bool reset) {
    unsigned long long v[3] = {0, 0, 0};
    if (cudaMemcpyFromSymbol(v, g_gs_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        out[0] = out[1] = out[2] = 0;
        return VIE_EDEVICE;
    }
    for (int i = 0; i < 3; ++i) out[i] = (double)v[i];
    if (reset) {
        const unsigned long long z[3] = {0, 0, 0};
        if (cudaMemcpyToSymbol(g_gs_bytes, z, sizeof(z)) != cudaSuccess) {
            cudaGetLastError();
            return VIE_EDEVICE;
        }
    }
    return VIE_OK;
}
