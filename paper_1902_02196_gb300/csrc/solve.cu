// Restarted, left-preconditioned GMRES on the device, batched over right-hand sides
// (Section IV-B: preconditioner P = M_eps G; Section V: GMRES with restart and a cap
// on outer iterations), with an FP32 variant wrapped in FP64 iterative refinement.
//
// Per cycle and right-hand side r: v_0 = r/||r||; for j = 0..m-1 the Arnoldi step
// w = P^-1 A v_j, h = V^H w (classical Gram-Schmidt, a second pass when the norm
// drops by more than a factor 1/sqrt2), h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j};
// complex Givens rotations keep the Hessenberg matrix triangular and give the
// residual estimate |g_{j+1}|; at the end H y = g is solved and x += V y.
// Inner products, norms, the Hessenberg matrix, the rotations and the solution
// update are FP64 in both modes; only the Krylov vectors and the matvec are FP32
// in the mixed mode.  Reductions use a fixed partition of each vector, so the
// result for one right-hand side does not depend on the others in the batch.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 8;  // elements per thread per reduction block
constexpr int kSeg = kThreads * kPer;

__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
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

__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double2 s = make_double2(0, 0);
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) s.x += sh[i].x, s.y += sh[i].y;
    return s;  // valid in thread 0
}

// partial[r][blk][i] = sum_{e in block} conj(V_i[r][e]) w[r][e], i < nvec
template <typename VC, typename WC>
__global__ void __launch_bounds__(kThreads) dots_kernel(const VC* __restrict__ V, long long vstride, const WC* __restrict__ w,
                                                        long long n, int nvec, double2* __restrict__ partial, int nblk,
                                                        const int* __restrict__ flag) {
    __shared__ double2 sh[kThreads / 32];
    const int r = blockIdx.y, blk = blockIdx.x;
    if (flag && !flag[r]) return;
    const long long base = (long long)r * n + (long long)blk * kSeg;
    double2 wv[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        long long e = (long long)blk * kSeg + threadIdx.x + k * kThreads;
        wv[k] = e < n ? to_d(w[base + threadIdx.x + k * kThreads]) : make_double2(0, 0);
    }
    for (int i = 0; i < nvec; ++i) {
        const VC* vi = V + i * vstride + base;
        double2 acc = make_double2(0, 0);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            long long e = (long long)blk * kSeg + threadIdx.x + k * kThreads;
            if (e < n) {
                double2 a = to_d(vi[threadIdx.x + k * kThreads]);
                acc.x += a.x * wv[k].x + a.y * wv[k].y;
                acc.y += a.x * wv[k].y - a.y * wv[k].x;
            }
        }
        double2 s = block_sum(acc, sh);
        if (threadIdx.x == 0) partial[((long long)r * nblk + blk) * nvec + i] = s;
    }
}

// out[r * rs + i * is] (+)= sum_blk partial[r][blk][i]; one block per (i, r), fixed order.
__global__ void __launch_bounds__(kThreads) finalize_kernel(const double2* __restrict__ partial, int nblk, int nvec,
                                                            double2* out, long long rs, long long is, int accumulate,
                                                            const int* __restrict__ flag) {
    __shared__ double2 sh[kThreads / 32];
    const int i = blockIdx.x, r = blockIdx.y;
    if (flag && !flag[r]) return;
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < nblk; b += kThreads) {
        double2 v = partial[((long long)r * nblk + b) * nvec + i];
        acc.x += v.x, acc.y += v.y;
    }
    double2 s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double2* o = out + r * rs + i * is;
        if (accumulate) {
            o->x += s.x;
            o->y += s.y;
        } else {
            *o = s;
        }
    }
}

// w[r] -= sum_i h[r][i] V_i[r]   (h read from H column j: H[r][i][j] at hbase + r*hstride + i*hcol)
template <typename VC, typename WC>
__global__ void update_kernel(const VC* __restrict__ V, long long vstride, WC* __restrict__ w, long long n, int nvec,
                              const double2* __restrict__ h, long long hstride, long long hcol,
                              const int* __restrict__ flag) {
    const int r = blockIdx.y;
    if (flag && !flag[r]) return;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long o = (long long)r * n + e;
    double2 acc = to_d(w[o]);
    for (int i = 0; i < nvec; ++i) {
        double2 hv = h[r * hstride + i * hcol];
        double2 v = to_d(V[i * vstride + o]);
        acc.x -= hv.x * v.x - hv.y * v.y;
        acc.y -= hv.x * v.y + hv.y * v.x;
    }
    w[o] = from_d<WC>(acc);
}

// x[r] += scale[r] * sum_i y[r][i] V_i[r] for i < k[r]
template <typename VC>
__global__ void xupdate_kernel(const VC* __restrict__ V, long long vstride, double2* __restrict__ x, long long n,
                               const double2* __restrict__ y, int ystride, const int* __restrict__ k) {
    const int r = blockIdx.y;
    const int kr = k[r];
    if (kr == 0) return;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long o = (long long)r * n + e;
    double2 acc = x[o];
    for (int i = 0; i < kr; ++i) {
        double2 yv = y[r * ystride + i];
        double2 v = to_d(V[i * vstride + o]);
        acc.x += yv.x * v.x - yv.y * v.y;
        acc.y += yv.x * v.y + yv.y * v.x;
    }
    x[o] = acc;
}

// dst[r] = src[r] * s[r] (s real), types may differ
template <typename SC, typename DC>
__global__ void scale_kernel(const SC* __restrict__ src, DC* __restrict__ dst, long long n,
                             const double* __restrict__ s) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long o = (long long)r * n + e;
    double2 v = to_d(src[o]);
    const double f = s[r];
    dst[o] = from_d<DC>(make_double2(v.x * f, v.y * f));
}

// out = a - b (FP64)
__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out,
                           long long total) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    out[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

// b~ = P^-1 b = b / (eps G_alpha)
__global__ void precond_rhs_kernel(const double2* __restrict__ b, const double2* __restrict__ ieps, double2* out,
                                   long long nv, int R, double g1, double g234) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv * 12 * R) return;
    const long long vox = e % nv;
    const int alpha = (int)((e / nv) % 12);
    const double ig = 1.0 / (alpha % 4 == 0 ? g1 : g234);
    double2 v = b[e], c = ieps[vox];
    out[e] = make_double2(ig * (v.x * c.x - v.y * c.y), ig * (v.x * c.y + v.y * c.x));
}

struct GState {
    double2* H;    // [R][m+1][m]
    double2* cs;   // [R][m]   (real part used)
    double2* sn;   // [R][m]
    double2* g;    // [R][m+1]
    double2* y;    // [R][m]
    double2* tmp;  // [R] scratch (norms)
    double* beta;  // [R]
    double* target;  // [R] absolute target for |g_{j+1}|
    double* sc;    // [R] scale factors
    int* active;   // [R]
    int* k;        // [R] Arnoldi steps of the current cycle
    int* nactive;  // [1]
    int m;
};

// start of a cycle: beta = ||r||, g = (beta, 0...), active = beta > target, scale = 1/beta
__global__ void cycle_init_kernel(GState s, int R, const double2* __restrict__ nrm2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double beta = sqrt(fmax(nrm2[r].x, 0.0));
    s.beta[r] = beta;
    for (int i = 0; i <= s.m; ++i) s.g[r * (s.m + 1) + i] = make_double2(0, 0);
    s.g[r * (s.m + 1)] = make_double2(beta, 0);
    s.k[r] = 0;
    const int act = (beta > s.target[r]) && beta > 0.0 && isfinite(beta);
    s.active[r] = act;
    s.sc[r] = act ? 1.0 / beta : 0.0;
}

// Givens step j for every active RHS; nrm2 = ||w||^2 after orthogonalisation.
__global__ void givens_kernel(GState s, int R, int j, const double2* __restrict__ nrm2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (!s.active[r]) {
        s.sc[r] = 0.0;
        return;
    }
    const int m = s.m;
    double2* H = s.H + (long long)r * (m + 1) * m;
    const double hnext = sqrt(fmax(nrm2[r].x, 0.0));
    H[(j + 1) * m + j] = make_double2(hnext, 0);
    for (int i = 0; i < j; ++i) {
        double2 a = H[i * m + j], b = H[(i + 1) * m + j];
        double c = s.cs[r * m + i].x;
        double2 sn = s.sn[r * m + i];
        // t = c a + sn b ; b' = -conj(sn) a + c b
        double2 t = make_double2(c * a.x + sn.x * b.x - sn.y * b.y, c * a.y + sn.x * b.y + sn.y * b.x);
        double2 bb = make_double2(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
        H[i * m + j] = t;
        H[(i + 1) * m + j] = bb;
    }
    double2 a = H[j * m + j];
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
    H[(j + 1) * m + j] = make_double2(0, 0);
    double2* g = s.g + r * (m + 1);
    double2 gj = g[j];
    g[j + 1] = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
    s.k[r] = j + 1;
    const double res = hypot(g[j + 1].x, g[j + 1].y);
    const bool done = res <= s.target[r] || hnext == 0.0 || !isfinite(res);
    s.sc[r] = (hnext > 0.0 && isfinite(hnext)) ? 1.0 / hnext : 0.0;
    if (done) s.active[r] = 0;
}

__global__ void count_active_kernel(const int* __restrict__ active, int R, int* out) {
    int c = 0;
    for (int r = 0; r < R; ++r) c += active[r];
    *out = c;
}

// reorthogonalisation flag: second Gram-Schmidt pass where ||w_after||^2 < 0.5 ||w_before||^2
__global__ void reorth_flag_kernel(const double2* __restrict__ before, const double2* __restrict__ after,
                                   const int* __restrict__ active, int* flag, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    flag[r] = active[r] && (after[r].x < 0.5 * before[r].x);
}

// back substitution H(0:k,0:k) y = g(0:k) per RHS
__global__ void trisolve_kernel(GState s, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int m = s.m, k = s.k[r];
    const double2* H = s.H + (long long)r * (m + 1) * m;
    const double2* g = s.g + r * (m + 1);
    double2* y = s.y + r * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < k; ++q) {
            double2 h = H[i * m + q], yv = y[q];
            acc.x -= h.x * yv.x - h.y * yv.y;
            acc.y -= h.x * yv.y + h.y * yv.x;
        }
        double2 d = H[i * m + i];
        double dd = d.x * d.x + d.y * d.y;
        y[i] = dd > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                      : make_double2(0, 0);
    }
}

}  // namespace


namespace {

// H[r][i][j] += c[r][i] for the right-hand sides that took a second Gram-Schmidt pass
__global__ void add_col_kernel(double2* H, long long rs, long long is, const double2* __restrict__ c, long long cs,
                               int nvec, const int* __restrict__ flag, int R) {
    const int r = blockIdx.x;
    if (r >= R || !flag[r]) return;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        double2* o = H + r * rs + i * is;
        double2 v = c[r * cs + i];
        o->x += v.x;
        o->y += v.y;
    }
}

__global__ void check_kernel(const double2* __restrict__ rn2, const double2* __restrict__ bn2, double tol,
                             double eta_min, double* target, int* done, double* rel, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double rn = sqrt(fmax(rn2[r].x, 0.0)), bn = sqrt(fmax(bn2[r].x, 0.0));
    const double rr = bn > 0 ? rn / bn : 0.0;
    rel[r] = rr;
    done[r] = rr <= tol;
    // inner target: the absolute residual this cycle must reach; converged right-hand sides stay idle
    target[r] = rr <= tol ? INFINITY : fmax(eta_min * rn, 0.5 * tol * bn);
}

struct Solver {
    vie_handle* h;
    cudaStream_t st;
    int R, m;
    long long n;
    int nblk;
    double2* partial;
    GState gs;
    int* reflag;
    double2* nrm_before;
    double2* nrm_after;
    double2* ctmp;  // [R][m+1]
    int* host_i;    // pinned scratch

    template <typename VC, typename WC>
    int dots(const VC* V, long long vstride, const WC* w, int nvec, double2* out, long long rs, long long is,
             int accumulate, const int* flag) {
        dim3 g1(nblk, R);
        VIE_KLAUNCH("dots", st, dots_kernel<VC, WC><<<g1, kThreads, 0, st>>>(V, vstride, w, n, nvec, partial, nblk, flag));
        dim3 g2(nvec, R);
        VIE_KLAUNCH("finalize", st, finalize_kernel<<<g2, kThreads, 0, st>>>(partial, nblk, nvec, out, rs, is, accumulate, flag));
        VIE_CHECK_LAUNCH();
        return VIE_OK;
    }
    template <typename C>
    int norm2(const C* w, double2* out, const int* flag) {
        return dots<C, C>(w, 0, w, 1, out, 1, 0, 0, flag);
    }
};

template <typename VC>
int run_cycle(Solver& S, VC* V, VC* W, double2* x64, const double2* r64, int precision, int* it_rhs, int* mv_count) {
    vie_handle* h = S.h;
    const int R = S.R, m = S.m;
    const long long n = S.n, vstride = (long long)R * n;
    cudaStream_t st = S.st;
    const dim3 ge((unsigned)((n + 255) / 256), R);
    const long long hrs = (long long)(m + 1) * m;
    VIE_TRY(S.norm2(r64, S.gs.tmp, nullptr));
    VIE_KLAUNCH("cycle_init", st, cycle_init_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs, R, S.gs.tmp));
    VIE_KLAUNCH("scale", st, scale_kernel<double2, VC><<<ge, 256, 0, st>>>(r64, V, n, S.gs.sc));
    VIE_CHECK_LAUNCH();
    for (int j = 0; j < m; ++j) {
        VIE_KLAUNCH("count_active", st, count_active_kernel<<<1, 1, 0, st>>>(S.gs.active, R, S.gs.nactive));
        VIE_CUDA(cudaMemcpyAsync(S.host_i, S.gs.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        if (*S.host_i == 0) break;
        VC* vj = V + j * vstride;
        VIE_TRY(matvec_device(h, R, vj, W, precision, VIE_OP_PA, st));
        ++*mv_count;
        // first classical Gram-Schmidt pass: H[:, j] = V^H w ; w -= V H[:, j]
        VIE_TRY(S.norm2(W, S.nrm_before, S.gs.active));
        VIE_TRY((S.dots<VC, VC>(V, vstride, W, j + 1, S.gs.H + j, hrs, m, 0, S.gs.active)));
        VIE_KLAUNCH("update", st, update_kernel<VC, VC><<<ge, 256, 0, st>>>(V, vstride, W, n, j + 1, S.gs.H + j, hrs, m, S.gs.active));
        VIE_CHECK_LAUNCH();
        VIE_TRY(S.norm2(W, S.nrm_after, S.gs.active));
        // second pass only where the norm dropped below 1/sqrt2 of its value
        VIE_KLAUNCH("reorth_flag", st, reorth_flag_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.nrm_before, S.nrm_after, S.gs.active, S.reflag, R));
        VIE_TRY((S.dots<VC, VC>(V, vstride, W, j + 1, S.ctmp, m + 1, 1, 0, S.reflag)));
        VIE_KLAUNCH("update", st, update_kernel<VC, VC><<<ge, 256, 0, st>>>(V, vstride, W, n, j + 1, S.ctmp, m + 1, 1, S.reflag));
        VIE_KLAUNCH("add_col", st, add_col_kernel<<<R, 64, 0, st>>>(S.gs.H + j, hrs, m, S.ctmp, m + 1, j + 1, S.reflag, R));
        VIE_TRY(S.norm2(W, S.nrm_after, S.reflag));
        VIE_KLAUNCH("givens", st, givens_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs, R, j, S.nrm_after));
        VIE_KLAUNCH("scale", st, scale_kernel<VC, VC><<<ge, 256, 0, st>>>(W, V + (j + 1) * vstride, n, S.gs.sc));
        VIE_CHECK_LAUNCH();
    }
    VIE_KLAUNCH("trisolve", st, trisolve_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs, R));
    VIE_KLAUNCH("xupdate", st, xupdate_kernel<VC><<<ge, 256, 0, st>>>(V, vstride, x64, n, S.gs.y, m, S.gs.k));
    VIE_CHECK_LAUNCH();
    std::vector<int> k(R);
    VIE_CUDA(cudaMemcpyAsync(k.data(), S.gs.k, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) it_rhs[r] += k[r];
    return VIE_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

int solve_device(vie_handle* h, int R, const double2* b, double2* x, double tol, int m, int maxit, int mode,
                 int use_guess, vie_solve_info* info, cudaStream_t st) {
    const long long n = 12LL * (long long)h->nv;
    const bool mixed = mode == VIE_SOLVE_FP32_REFINE;
    const size_t vc = mixed ? sizeof(float2) : sizeof(double2);
    const int nblk = (int)((n + kSeg - 1) / kSeg);
    // carve the workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oV = take(vc * (size_t)(m + 1) * R * n);
    const size_t oW = take(vc * (size_t)R * n);
    const size_t oR = take(sizeof(double2) * R * n);
    const size_t oBt = take(sizeof(double2) * R * n);
    const size_t oT = take(sizeof(double2) * R * n);
    const size_t oPart = take(sizeof(double2) * (size_t)R * nblk * (m + 1));
    const size_t oH = take(sizeof(double2) * (size_t)R * (m + 1) * m);
    const size_t oCs = take(sizeof(double2) * (size_t)R * m);
    const size_t oSn = take(sizeof(double2) * (size_t)R * m);
    const size_t oG = take(sizeof(double2) * (size_t)R * (m + 1));
    const size_t oY = take(sizeof(double2) * (size_t)R * m);
    const size_t oTmp = take(sizeof(double2) * R);
    const size_t oBeta = take(sizeof(double) * R);
    const size_t oTarget = take(sizeof(double) * R);
    const size_t oSc = take(sizeof(double) * R);
    const size_t oAct = take(sizeof(int) * R);
    const size_t oK = take(sizeof(int) * R);
    const size_t oNact = take(sizeof(int));
    const size_t oRe = take(sizeof(int) * R);
    const size_t oNb = take(sizeof(double2) * R);
    const size_t oNa = take(sizeof(double2) * R);
    const size_t oC = take(sizeof(double2) * (size_t)R * (m + 1));
    const size_t oBn = take(sizeof(double2) * R);
    const size_t oDone = take(sizeof(int) * R);
    const size_t oRel = take(sizeof(double) * R);
    VIE_TRY(ws_reserve(h, h->solve_ws, off));
    char* base = static_cast<char*>(h->solve_ws.ptr);
    Solver S;
    S.h = h;
    S.st = st;
    S.R = R;
    S.m = m;
    S.n = n;
    S.nblk = nblk;
    S.partial = reinterpret_cast<double2*>(base + oPart);
    S.gs.H = reinterpret_cast<double2*>(base + oH);
    S.gs.cs = reinterpret_cast<double2*>(base + oCs);
    S.gs.sn = reinterpret_cast<double2*>(base + oSn);
    S.gs.g = reinterpret_cast<double2*>(base + oG);
    S.gs.y = reinterpret_cast<double2*>(base + oY);
    S.gs.tmp = reinterpret_cast<double2*>(base + oTmp);
    S.gs.beta = reinterpret_cast<double*>(base + oBeta);
    S.gs.target = reinterpret_cast<double*>(base + oTarget);
    S.gs.sc = reinterpret_cast<double*>(base + oSc);
    S.gs.active = reinterpret_cast<int*>(base + oAct);
    S.gs.k = reinterpret_cast<int*>(base + oK);
    S.gs.nactive = reinterpret_cast<int*>(base + oNact);
    S.gs.m = m;
    S.reflag = reinterpret_cast<int*>(base + oRe);
    S.nrm_before = reinterpret_cast<double2*>(base + oNb);
    S.nrm_after = reinterpret_cast<double2*>(base + oNa);
    S.ctmp = reinterpret_cast<double2*>(base + oC);
    double2* r64 = reinterpret_cast<double2*>(base + oR);
    double2* bt = reinterpret_cast<double2*>(base + oBt);
    double2* t64 = reinterpret_cast<double2*>(base + oT);
    double2* bn2 = reinterpret_cast<double2*>(base + oBn);
    int* done = reinterpret_cast<int*>(base + oDone);
    double* rel = reinterpret_cast<double*>(base + oRel);
    int* pinned = nullptr;
    VIE_CUDA(cudaMallocHost(&pinned, sizeof(int) * 4));
    S.host_i = pinned;
    struct PinGuard {
        int* p;
        ~PinGuard() { cudaFreeHost(p); }
    } guard{pinned};

    const long long total = (long long)R * n;
    const unsigned gt = (unsigned)((total + 255) / 256);
    const double dV = h->dx * h->dy * h->dz;
    VIE_KLAUNCH("precond_rhs", st, precond_rhs_kernel<<<gt, 256, 0, st>>>(b, h->ieps64, bt, (long long)h->nv, R, dV, dV / 12.0));
    VIE_CHECK_LAUNCH();
    VIE_TRY(S.norm2(bt, bn2, nullptr));
    if (!use_guess) VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * total, st));

    std::vector<int> it_rhs(R, 0);
    int mv64 = 0, mv32 = 0, sweeps = 0;
    std::vector<int> hdone(R, 0);
    const double eta_min = mixed ? 2e-5 : 0.0;
    bool x_is_zero = !use_guess;
    for (int cyc = 0; cyc < maxit; ++cyc) {
        if (x_is_zero) {
            VIE_CUDA(cudaMemcpyAsync(r64, bt, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
        } else {
            VIE_TRY(matvec_device(h, R, x, t64, VIE_FP64, VIE_OP_PA, st));
            ++mv64;
            VIE_KLAUNCH("sub", st, sub_kernel<<<gt, 256, 0, st>>>(bt, t64, r64, total));
        }
        VIE_TRY(S.norm2(r64, S.gs.tmp, nullptr));
        VIE_KLAUNCH("check", st, check_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs.tmp, bn2, tol, eta_min, S.gs.target, done, rel, R));
        VIE_CHECK_LAUNCH();
        VIE_CUDA(cudaMemcpyAsync(hdone.data(), done, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        bool all = true;
        for (int r = 0; r < R; ++r) all = all && hdone[r];
        if (all) break;
        if (mixed) {
            float2* V = reinterpret_cast<float2*>(base + oV);
            float2* W = reinterpret_cast<float2*>(base + oW);
            VIE_TRY(run_cycle<float2>(S, V, W, x, r64, VIE_FP32, it_rhs.data(), &mv32));
            ++sweeps;
        } else {
            double2* V = reinterpret_cast<double2*>(base + oV);
            double2* W = reinterpret_cast<double2*>(base + oW);
            VIE_TRY(run_cycle<double2>(S, V, W, x, r64, VIE_FP64, it_rhs.data(), &mv64));
        }
        x_is_zero = false;
    }
    // final residuals in FP64: preconditioned and unpreconditioned
    std::vector<double> hrel(R), htrue(R);
    {
        VIE_TRY(matvec_device(h, R, x, t64, VIE_FP64, VIE_OP_PA, st));
        VIE_KLAUNCH("sub", st, sub_kernel<<<gt, 256, 0, st>>>(bt, t64, r64, total));
        VIE_TRY(S.norm2(r64, S.gs.tmp, nullptr));
        VIE_KLAUNCH("check", st, check_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs.tmp, bn2, tol, eta_min, S.gs.target, done, rel, R));
        VIE_CUDA(cudaMemcpyAsync(hrel.data(), rel, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_TRY(matvec_device(h, R, x, t64, VIE_FP64, VIE_OP_A, st));
        VIE_KLAUNCH("sub", st, sub_kernel<<<gt, 256, 0, st>>>(b, t64, r64, total));
        VIE_TRY(S.norm2(r64, S.gs.tmp, nullptr));
        VIE_TRY(S.norm2(b, bn2, nullptr));
        VIE_KLAUNCH("check", st, check_kernel<<<(R + 127) / 128, 128, 0, st>>>(S.gs.tmp, bn2, tol, eta_min, S.gs.target, done, rel, R));
        VIE_CUDA(cudaMemcpyAsync(htrue.data(), rel, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
    }
    int rc = VIE_OK;
    for (int r = 0; r < R; ++r) {
        const bool conv = hrel[r] <= tol;
        if (!conv) rc = VIE_NOT_CONVERGED;
        if (info) {
            info[r].converged = conv;
            info[r].iterations = it_rhs[r];
            info[r].fp64_matvecs = mv64 + 2;
            info[r].fp32_matvecs = mv32;
            info[r].refinements = sweeps;
            info[r].resid = hrel[r];
            info[r].true_resid = htrue[r];
        }
    }
    return rc;
}
