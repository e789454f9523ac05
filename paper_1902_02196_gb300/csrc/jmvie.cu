// Full JM-VIE (Eq. 13-15): polarization current j and magnetization current m together, for
// scatterers with a relative permeability mu_r = mu' - i mu'' (Eq. 1-2, chi_m = mu_r - 1, Eq. 7).
//
// Both currents take the PWL functions of Section III.  The magnetization unknown is scaled,
// m' = m / eta0, and the second row of Eq. 15 divided by eta0; with c_e eta0 = c_m / eta0 = i k0
// the Galerkin system is
//     [ M_eps G - M_chie N      i k0 M_chie K      ] [j ]   [ c_e M_chie e_inc  ]
//     [ -i k0 M_chim K          M_mu G - M_chim N  ] [m'] = [ i k0 M_chim h_inc ]
// so that both unknowns have the same size (j ~ c_e e, m' ~ c_e e as well), and the
// preconditioner is P = diag(M_eps G, M_mu G).  Vectors are [R][2][12][nz][ny][nx]: j, then m'.
//
// The operator is composed from the library's matvecs on the 2R stacked currents: one (N - G)
// product (VIE_OP_NSCAT) and one K product (Eq. 8), then one element-wise kernel that forms both
// rows (N = (N - G) + G, and eps - chi_e = mu - chi_m = 1):
//     row j : G j  - chi_e (N - G) j  + i k0 chi_e K m'
//     row m': G m' - chi_m (N - G) m' - i k0 chi_m K j
// (P^-1 A divides each row by eps G, resp. mu G).  The products run in FP64, or in FP32 for the
// inner solves of the mixed-precision mode (FP64 refinement around them); the material maps stay
// FP64 and are rounded in the combining kernel.  Off the tissue path: tissue is non-magnetic,
// which reduces the system to Eq. 16.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

// eta0 = sqrt(mu0 / eps0) = 1 / (eps0 c0), with mu0 = 1 / (eps0 c0^2)
constexpr double kEta0 = 1.0 / (VIE_EPS0 * VIE_C0);

unsigned grid1(long long n) { return (unsigned)((n + 255) / 256); }

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// mu = mr - i mi, chi_m = mu - 1, 1/mu, and the support indicator |chi_e| + |chi_m|
__global__ void jm_materials_kernel(const double* __restrict__ mr, const double* __restrict__ mi, long long nv,
                                    const double2* __restrict__ chie, double2* mu, double2* chim, double2* imu,
                                    double2* sup) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double2 m = make_double2(mr ? mr[v] : 1.0, mi ? -mi[v] : 0.0);
    mu[v] = m;
    chim[v] = make_double2(m.x - 1.0, m.y);
    imu[v] = zdiv(make_double2(1.0, 0.0), m);
    const double2 c = chie[v];
    sup[v] = make_double2(hypot(c.x, c.y) + hypot(m.x - 1.0, m.y), 0.0);
}

template <typename C>
__device__ __forceinline__ C to_c(double2 v);
template <>
__device__ __forceinline__ double2 to_c<double2>(double2 v) {
    return v;
}
template <>
__device__ __forceinline__ float2 to_c<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}
template <typename C>
__device__ __forceinline__ C cdiv(C a, C b) {
    const auto d = b.x * b.x + b.y * b.y;
    C r;
    r.x = (a.x * b.x + a.y * b.y) / d;
    r.y = (a.y * b.x - a.x * b.y) / d;
    return r;
}

// y = A x (op VIE_OP_A) or P^-1 A x - shift x (op VIE_OP_PA), from x, nx = (N - G) x and kx = K x,
// all [R][2][12][nv], in the precision of C (the material maps are read in FP64 and rounded)
template <typename C>
__global__ void jm_combine_kernel(const C* __restrict__ x, const C* __restrict__ nx, const C* __restrict__ kx,
                                  const double2* __restrict__ eps, const double2* __restrict__ chie,
                                  const double2* __restrict__ mu, const double2* __restrict__ chim, C* __restrict__ y,
                                  long long nv, int R, int op, double k0, double g1, double g234,
                                  const double2* __restrict__ shift) {
    using T = decltype(C{}.x);
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long half_len = 12 * nv;
    if (e >= 2 * half_len * R) return;
    const long long r = e / (2 * half_len);
    const long long rem = e - r * 2 * half_len;
    const int half = (int)(rem / half_len);
    const int alpha = (int)((rem / nv) % 12);
    const long long v = e % nv;
    const long long eo = half ? e - half_len : e + half_len;  // the same unknown of the other current
    const T g = (T)(comp_is_constant(alpha, 12) ? g1 : g234);
    const C c = to_c<C>(half ? chim[v] : chie[v]);
    // coupling: + i k0 c K m' in row j, - i k0 c K j in row m'
    const T s = (T)(half ? -k0 : k0);
    const C ko = kx[eo];
    const C cpl = cmul(c, mk(-s * ko.y, s * ko.x));
    const C cn = cmul(c, nx[e]);
    const C xv = x[e];
    C out;
    if (op == VIE_OP_A) {
        out = mk(g * xv.x - cn.x + cpl.x, g * xv.y - cn.y + cpl.y);
    } else {
        const C m = to_c<C>(half ? mu[v] : eps[v]);
        const C t = cdiv(mk((cpl.x - cn.x) / g, (cpl.y - cn.y) / g), m);
        const C xm = cdiv(xv, m);
        out = mk(xm.x + t.x, xm.y + t.y);
        if (shift) {
            const C sx = cmul(to_c<C>(shift[r]), xv);
            out.x -= sx.x;
            out.y -= sx.y;
        }
    }
    y[e] = out;
}

// b = (c_e chi_e e_inc, i k0 chi_m h_inc) per right-hand side
__global__ void jm_rhs_kernel(const double2* __restrict__ einc, const double2* __restrict__ hinc,
                              const double2* __restrict__ chie, const double2* __restrict__ chim, double2 ce,
                              double k0, long long nv, int R, double2* __restrict__ b) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over [R][12][nv]
    if (e >= 12 * nv * R) return;
    const long long r = e / (12 * nv), rem = e % (12 * nv), v = e % nv;
    const double2 be = zmul(zmul(ce, chie[v]), einc[e]);
    const double2 bm = zmul(zmul(make_double2(0.0, k0), chim[v]), hinc[e]);
    b[r * 24 * nv + rem] = be;
    b[r * 24 * nv + 12 * nv + rem] = bm;
}

// Tested total fields divided by G (Eq. 13):
//   e = (e_inc + (N - G) j / c_e - eta0 K m') / G,   h = (h_inc + K j + (N - G) m' / (i k0)) / G
// and the absorbed-power density per voxel, electric plus magnetic loss:
//   p = [1/2 Re{sum G |j|^2 / (c_e chi_e)} + 1/2 Re{eta0 sum G |m'|^2 / (i k0 chi_m)}] / dV,
// with per-block partial sums of p dV.  One thread per (right-hand side, voxel).
__global__ void jm_fields_kernel(const double2* __restrict__ x, const double2* __restrict__ nx,
                                 const double2* __restrict__ kx, const double2* __restrict__ einc,
                                 const double2* __restrict__ hinc, const double2* __restrict__ chie,
                                 const double2* __restrict__ chim, double2 ce, double k0, double eta0, double g1,
                                 double g234, double dV, long long nv, double2* __restrict__ eout,
                                 double2* __restrict__ hout, double* __restrict__ pout, double* __restrict__ partial) {
    __shared__ double sh[256];
    const int r = blockIdx.y;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double pv = 0.0;
    if (v < nv) {
        const double2 inv_ce = zdiv(make_double2(1.0, 0.0), ce);
        const double2 inv_ik0 = make_double2(0.0, -1.0 / k0);
        double qe = 0.0, qm = 0.0;
        for (int a = 0; a < 12; ++a) {
            const double G = comp_is_constant(a, 12) ? g1 : g234;
            const long long oj = ((long long)r * 24 + a) * nv + v, om = oj + 12 * nv;
            const long long oi = ((long long)r * 12 + a) * nv + v;
            const double2 nj = zmul(nx[oj], inv_ce), nm = zmul(nx[om], inv_ik0);
            const double2 e = make_double2((einc[oi].x + nj.x - eta0 * kx[om].x) / G,
                                           (einc[oi].y + nj.y - eta0 * kx[om].y) / G);
            const double2 hh = make_double2((hinc[oi].x + kx[oj].x + nm.x) / G, (hinc[oi].y + kx[oj].y + nm.y) / G);
            if (eout) eout[oi] = e;
            if (hout) hout[oi] = hh;
            const double2 xj = x[oj], xm = x[om];
            qe += G * (xj.x * xj.x + xj.y * xj.y);
            qm += G * (xm.x * xm.x + xm.y * xm.y);
        }
        const double2 ce_ = chie[v], cm_ = chim[v];
        if (ce_.x != 0.0 || ce_.y != 0.0) pv += 0.5 * zdiv(make_double2(qe, 0.0), zmul(ce, ce_)).x;
        if (cm_.x != 0.0 || cm_.y != 0.0) pv += 0.5 * zdiv(make_double2(eta0 * qm, 0.0), zmul(make_double2(0.0, k0), cm_)).x;
        if (pout) pout[(long long)r * nv + v] = pv / dV;
    }
    sh[threadIdx.x] = pv;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = sh[0];
}

// out[r] = sum of the nblk partials of right-hand side r, in a fixed order (one block per r)
__global__ void jm_sum_kernel(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
    __shared__ double sh[256];
    const int r = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) a += partial[(long long)r * nblk + b];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = sh[0];
}

// y -= shift[r] x for vectors of n complex values per right-hand side
template <typename C>
__global__ void jm_shift_kernel(C* __restrict__ y, const C* __restrict__ x, const double2* __restrict__ shift,
                                long long n) {
    const int r = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long o = (long long)r * n + e;
    const C sx = cmul(to_c<C>(shift[r]), x[o]);
    y[o] = mk(y[o].x - sx.x, y[o].y - sx.y);
}

// (N - G) and K of the 2R stacked currents into the handle's JM scratch, in FP64 or FP32
template <typename C>
int jm_products(vie_handle* h, int R, const C* x, C** nx, C** kx, cudaStream_t s) {
    const int prec = sizeof(C) == 16 ? VIE_FP64 : VIE_FP32;
    const size_t per = sizeof(C) * (size_t)R * 24 * h->nv;
    VIE_TRY(ws_reserve(h, h->jm_ws, 2 * per));
    *nx = static_cast<C*>(h->jm_ws.ptr);
    *kx = *nx + (size_t)R * 24 * h->nv;
    VIE_TRY(matvec_device(h, 2 * R, x, *nx, prec, VIE_OP_NSCAT, s));
    VIE_TRY(matvec_device(h, 2 * R, x, *kx, prec, VIE_OP_K, s));
    return VIE_OK;
}

template <typename C>
int jm_matvec_full_t(vie_handle* h, int R, const C* x, C* y, int op, cudaStream_t s, const double2* shift) {
    if (!h->mu64) VIE_TRY(jm_materials(h, nullptr, nullptr, s));
    C *nx = nullptr, *kx = nullptr;
    VIE_TRY(jm_products<C>(h, R, x, &nx, &kx, s));
    const long long nv = (long long)h->nv;
    const double dV = h->dx * h->dy * h->dz;
    VIE_KLAUNCH("jm_combine", s,
                jm_combine_kernel<C><<<grid1(24 * nv * R), 256, 0, s>>>(x, nx, kx, h->eps64, h->chi64, h->mu64,
                                                                       h->chim64, y, nv, R, op, h->k0, dV, dV / 12.0,
                                                                       op == VIE_OP_PA ? shift : nullptr));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

template <typename C>
int jm_matvec_support_t(vie_handle* h, int R, const C* x, C* y, int op, const Support& sp, void* tmp, cudaStream_t s,
                        const double2* shift) {
    if (!sp.rows) return jm_matvec_full_t<C>(h, R, x, y, op, s, shift);
    const int prec = sizeof(C) == 16 ? VIE_FP64 : VIE_FP32;
    C* tx = static_cast<C*>(tmp);
    C* ty = tx + (size_t)R * 24 * h->nv;
    VIE_TRY(support_scatter(h, 2 * R, x, tx, prec, sp, s));
    VIE_TRY(jm_matvec_full_t<C>(h, R, tx, ty, op, s, nullptr));
    VIE_TRY(support_gather(h, 2 * R, ty, y, prec, sp, s));
    if (shift && op == VIE_OP_PA) {
        const long long n = 24 * sp.ns;
        VIE_KLAUNCH("jm_shift", s, jm_shift_kernel<C><<<dim3(grid1(n), R), 256, 0, s>>>(y, x, shift, n));
        VIE_CHECK_LAUNCH();
    }
    return VIE_OK;
}

}  // namespace

int jm_materials(vie_handle* h, const double* mr, const double* mi, cudaStream_t s) {
    const size_t nv = h->nv;
    if (!h->mu64) {
        double2* p = nullptr;
        if (cudaMalloc(&p, 4 * sizeof(double2) * nv) != cudaSuccess) {
            cudaGetLastError();
            set_error("permeability allocation failed");
            return VIE_ENOMEM;
        }
        h->mu64 = p;
        h->chim64 = p + nv;
        h->imu64 = p + 2 * nv;
        h->jmsup64 = p + 3 * nv;
        h->bytes_held += 4 * sizeof(double2) * nv;
    }
    VIE_KLAUNCH("jm_materials", s,
                jm_materials_kernel<<<grid1((long long)nv), 256, 0, s>>>(mr, mi, (long long)nv, h->chi64, h->mu64,
                                                                        h->chim64, h->imu64, h->jmsup64));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

int jm_matvec_full(vie_handle* h, int R, const double2* x, double2* y, int op, cudaStream_t s, const double2* shift) {
    return jm_matvec_full_t<double2>(h, R, x, y, op, s, shift);
}

int jm_matvec_support(vie_handle* h, int R, const void* x, void* y, int op, const Support& sp, void* tmp,
                      cudaStream_t s, const double2* shift, int precision) {
    if (precision == VIE_FP64)
        return jm_matvec_support_t<double2>(h, R, static_cast<const double2*>(x), static_cast<double2*>(y), op, sp, tmp,
                                            s, shift);
    if (precision == VIE_FP32)
        return jm_matvec_support_t<float2>(h, R, static_cast<const float2*>(x), static_cast<float2*>(y), op, sp, tmp,
                                           s, shift);
    set_error("the JM-VIE runs in FP64 or FP32");
    return VIE_EINVAL;
}

int jm_rhs_device(vie_handle* h, int R, const double2* einc, const double2* hinc, double2* b, cudaStream_t s) {
    if (!h->mu64) VIE_TRY(jm_materials(h, nullptr, nullptr, s));
    const long long nv = (long long)h->nv;
    const double2 ce = make_double2(0.0, h->omega * VIE_EPS0);
    VIE_KLAUNCH("jm_rhs", s,
                jm_rhs_kernel<<<grid1(12 * nv * R), 256, 0, s>>>(einc, hinc, h->chi64, h->chim64, ce, h->k0, nv, R, b));
    VIE_CHECK_LAUNCH();
    return VIE_OK;
}

int jm_fields_device(vie_handle* h, int R, const double2* x, const double2* einc, const double2* hinc, double2* eout,
                     double2* hout, double* p_abs, double* P_abs_host, cudaStream_t s) {
    if (!h->mu64) VIE_TRY(jm_materials(h, nullptr, nullptr, s));
    double2 *nx = nullptr, *kx = nullptr;
    VIE_TRY(jm_products<double2>(h, R, x, &nx, &kx, s));
    const long long nv = (long long)h->nv;
    const int nblk = (int)((nv + 255) / 256);
    VIE_TRY(ws_reserve(h, h->post_ws, sizeof(double) * (size_t)R * (nblk + 1)));
    double* partial = static_cast<double*>(h->post_ws.ptr);
    double* tot = partial + (size_t)R * nblk;
    const double dV = h->dx * h->dy * h->dz;
    const double2 ce = make_double2(0.0, h->omega * VIE_EPS0);
    VIE_KLAUNCH("jm_fields", s,
                jm_fields_kernel<<<dim3(nblk, R), 256, 0, s>>>(x, nx, kx, einc, hinc, h->chi64, h->chim64, ce, h->k0,
                                                               kEta0, dV, dV / 12.0, dV, nv, eout, hout, p_abs,
                                                               partial));
    VIE_KLAUNCH("jm_fields", s, jm_sum_kernel<<<R, 256, 0, s>>>(partial, nblk, tot));
    VIE_CHECK_LAUNCH();
    if (P_abs_host) {
        VIE_CUDA(cudaMemcpyAsync(P_abs_host, tot, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
    }
    return VIE_OK;
}
