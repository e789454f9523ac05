// Low multilinear rank (Tucker) compression of the 60 Toeplitz defining tensors of N - G
// (Section III-C: the defining tensors compress by low multilinear rank decompositions).
//
// Each tensor T[nz][ny][nx] (offsets d >= 0, FP64) is written as
//     T ~ C x_z U_z x_y U_y x_x U_x,   C = T x_z U_z^H x_y U_y^H x_x U_x^H,
// with orthonormal factors U_k (n_k x r_k).  The factor of mode k spans the range of the mode-k
// unfolding T_(k) up to a discarded energy of at most tol^2 ||T||^2 / 3, so that (the three
// projections being orthogonal) ||T - T~||_F <= tol ||T||_F.  The range is found from the Gram
// matrix G_k = T_(k) T_(k)^H (device) by a diagonally pivoted Cholesky factorisation stopped
// when the trace of the remaining Schur complement falls below the threshold (host, O(n^2 r)):
// that trace bounds the energy of T_(k) outside the span of the chosen columns, so the error
// bound holds, with ranks at least those of the truncated SVD (which are minimal for the same
// criterion).  Because the Gram matrix squares the singular values, tol must stay above about
// 1e-7 in FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"

int green_embed(vie_handle* h, double2* T, bool keep_table);  // green.cu

namespace {

using cplx = std::complex<double>;
constexpr int kT = 60;  // unique tensors

// G[t][i][j] = sum_k A_t(k, i) conj(A_t(k, j)), A_t(k, i) = T[t nd + (k / kc) sa + (k % kc) sc + i si]
struct GramGeo {
    long long sa, sc, si, K;
    int kc, n;
};

__global__ void __launch_bounds__(256) gram_kernel(const double2* __restrict__ T, long long nd, GramGeo g,
                                                   double2* __restrict__ G) {
    __shared__ double2 As[16][17], Bs[16][17];
    const int t = blockIdx.z;
    const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const double2* base = T + (long long)t * nd;
    const bool imajor = g.si == 1;  // load with the fastest thread index along i (else along k)
    double ar = 0.0, ai = 0.0;
    for (long long k0 = 0; k0 < g.K; k0 += 16) {
        const int lk = imajor ? ty : tx, li = imajor ? tx : ty;
        const long long k = k0 + lk;
        double2 va = make_double2(0.0, 0.0), vb = va;
        if (k < g.K) {
            const long long o = (k / g.kc) * g.sa + (k % g.kc) * g.sc;
            if (i0 + li < g.n) va = base[o + (long long)(i0 + li) * g.si];
            if (j0 + li < g.n) vb = base[o + (long long)(j0 + li) * g.si];
        }
        As[lk][li] = va;
        Bs[lk][li] = vb;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double2 a = As[kk][ty], b = Bs[kk][tx];
            ar += a.x * b.x + a.y * b.y;  // a conj(b)
            ai += a.y * b.x - a.x * b.y;
        }
        __syncthreads();
    }
    const int i = i0 + ty, j = j0 + tx;
    if (i < g.n && j < g.n) G[((long long)t * g.n + i) * g.n + j] = make_double2(ar, ai);
}

// One mode product per tensor t: the input [d2][d1][d0] at in + in_off[t], the output at
// out + out_off[t] with the dimension of axis `ax` (0 = z, 1 = y, 2 = x) replaced by m.
//   compress (expand = 0): out[.. a ..] = sum_i in[.. i ..] conj(U[i][a]), U: [n][r], m = r
//   expand   (expand = 1): out[.. i ..] = sum_a in[.. a ..] U[i][a],       U: [n][r], m = n
struct ModeDesc {
    long long in_off, out_off, u_off;
    int d[3];  // input dims (z, y, x)
    int m;     // output size along ax
    int ldu;   // r (columns of U)
};

__global__ void mode_product_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                    const double2* __restrict__ U, const ModeDesc* __restrict__ desc, int ax,
                                    int expand) {
    const ModeDesc D = desc[blockIdx.y];
    int od[3] = {D.d[0], D.d[1], D.d[2]};
    od[ax] = D.m;
    const long long total = (long long)od[0] * od[1] * od[2];
    const int len = D.d[ax];  // contracted length
    long long sin[3] = {(long long)D.d[1] * D.d[2], D.d[2], 1};
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int c2 = (int)(e % od[2]);
        const int c1 = (int)((e / od[2]) % od[1]);
        const int c0 = (int)(e / ((long long)od[2] * od[1]));
        int c[3] = {c0, c1, c2};
        const int p = c[ax];
        c[ax] = 0;
        const double2* src = in + D.in_off + c[0] * sin[0] + c[1] * sin[1] + c[2] * sin[2];
        const long long st = sin[ax];
        const double2* u = U + D.u_off;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < len; ++q) {
            const double2 v = src[q * st];
            double2 w;
            if (expand) {
                w = u[(long long)p * D.ldu + q];
            } else {
                w = u[(long long)q * D.ldu + p];
                w.y = -w.y;
            }
            sr += v.x * w.x - v.y * w.y;
            si += v.x * w.y + v.y * w.x;
        }
        out[D.out_off + e] = make_double2(sr, si);
    }
}

// partial[t][blk] = (sum |A - B|^2, sum |A|^2) over the block's elements of tensor t
__global__ void diff_norm_kernel(const double2* __restrict__ A, const double2* __restrict__ B, long long nd,
                                 double2* __restrict__ partial) {
    __shared__ double s0[256], s1[256];
    const int t = blockIdx.y;
    double a0 = 0.0, a1 = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nd; e += (long long)gridDim.x * blockDim.x) {
        const double2 x = A[(long long)t * nd + e], y = B[(long long)t * nd + e];
        a0 += (x.x - y.x) * (x.x - y.x) + (x.y - y.y) * (x.y - y.y);
        a1 += x.x * x.x + x.y * x.y;
    }
    s0[threadIdx.x] = a0;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s0[threadIdx.x] += s0[threadIdx.x + s];
            s1[threadIdx.x] += s1[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)t * gridDim.x + blockIdx.x] = make_double2(s0[0], s1[0]);
}

// Orthonormal basis (n x r, row-major [n][r]) of the range of the Hermitian PSD matrix G (n x n)
// up to a remaining Schur trace <= thr: diagonally pivoted Cholesky, then modified Gram-Schmidt
// applied twice to the chosen columns.  At least one column.
std::vector<cplx> range_basis(const cplx* G, int n, double thr, int* rank) {
    std::vector<double> d(n);
    for (int i = 0; i < n; ++i) d[i] = std::max(G[(size_t)i * n + i].real(), 0.0);
    std::vector<cplx> L;  // column-major n x r
    std::vector<char> used(n, 0);
    int r = 0;
    for (;;) {
        double rest = 0.0;
        for (int i = 0; i < n; ++i)
            if (!used[i]) rest += d[i];
        if ((r > 0 && rest <= thr) || r == n) break;
        int p = -1;
        for (int i = 0; i < n; ++i)
            if (!used[i] && (p < 0 || d[i] > d[p])) p = i;
        if (d[p] <= 0.0) {
            if (r > 0) break;
            d[p] = 1.0;  // a zero matrix: any single direction
        }
        const double piv = std::sqrt(d[p]);
        L.resize((size_t)(r + 1) * n);
        cplx* l = L.data() + (size_t)r * n;
        for (int i = 0; i < n; ++i) {
            cplx v = G[(size_t)i * n + p];
            for (int k = 0; k < r; ++k) v -= L[(size_t)k * n + i] * std::conj(L[(size_t)k * n + p]);
            l[i] = used[i] ? cplx(0.0) : v / piv;
        }
        l[p] = piv;
        used[p] = 1;
        for (int i = 0; i < n; ++i)
            if (!used[i]) d[i] = std::max(d[i] - std::norm(l[i]), 0.0);
        d[p] = 0.0;
        ++r;
    }
    // orthonormalise the columns (two passes of modified Gram-Schmidt); drop dependent ones
    std::vector<cplx> Q;
    int q = 0;
    for (int k = 0; k < r; ++k) {
        std::vector<cplx> v(L.begin() + (size_t)k * n, L.begin() + (size_t)(k + 1) * n);
        double n0 = 0.0;
        for (auto& z : v) n0 += std::norm(z);
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < q; ++j) {
                cplx dot = 0.0;
                for (int i = 0; i < n; ++i) dot += std::conj(Q[(size_t)j * n + i]) * v[i];
                for (int i = 0; i < n; ++i) v[i] -= dot * Q[(size_t)j * n + i];
            }
        double nn = 0.0;
        for (auto& z : v) nn += std::norm(z);
        if (!(nn > 1e-24 * n0) || nn == 0.0) continue;
        const double s = 1.0 / std::sqrt(nn);
        for (auto& z : v) z *= s;
        Q.insert(Q.end(), v.begin(), v.end());
        ++q;
    }
    if (q == 0) {  // degenerate: the first unit vector
        Q.assign(n, cplx(0.0));
        Q[0] = 1.0;
        q = 1;
    }
    *rank = q;
    std::vector<cplx> U((size_t)n * q);  // row-major [n][q]
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < n; ++i) U[(size_t)i * q + j] = Q[(size_t)j * n + i];
    return U;
}

int launch_modes(const double2* in, double2* out, const double2* U, const std::vector<ModeDesc>& hd, ModeDesc* dd,
                 int ax, int expand, cudaStream_t s) {
    VIE_CUDA(cudaMemcpyAsync(dd, hd.data(), sizeof(ModeDesc) * hd.size(), cudaMemcpyHostToDevice, s));
    VIE_KLAUNCH("tucker_mode_product", s,
                mode_product_kernel<<<dim3(256, (unsigned)hd.size()), 256, 0, s>>>(in, out, U, dd, ax, expand));
    VIE_CHECK_LAUNCH();
    VIE_CUDA(cudaStreamSynchronize(s));  // hd is reused by the next step
    return VIE_OK;
}

}  // namespace

// Reconstruction T~ [60][nz][ny][nx] of the handle's Tucker form into out (device).
int tucker_reconstruct(vie_handle* h, double2* out, cudaStream_t s) {
    if (!h->tucker) {
        set_error("the handle holds no Tucker form");
        return VIE_EINVAL;
    }
    const int n[3] = {h->nz, h->ny, h->nx};
    const long long nd = (long long)h->nv;
    const double2* base = static_cast<const double2*>(h->tucker);
    // scratch for the two intermediate products: [rz][ry][nx] <= [nz][ny][nx] and [rz][ny][nx]
    double2* w = nullptr;
    ModeDesc* dd = nullptr;
    if (cudaMalloc(&w, sizeof(double2) * 2 * kT * nd) != cudaSuccess || cudaMalloc(&dd, sizeof(ModeDesc) * kT) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w);
        set_error("Tucker reconstruction scratch allocation failed");
        return VIE_ENOMEM;
    }
    double2* w1 = w;
    double2* w2 = w + kT * nd;
    std::vector<ModeDesc> hd(kT);
    int rc = VIE_OK;
    // expand x: [rz][ry][rx] -> [rz][ry][nx]
    for (int t = 0; t < kT; ++t) {
        const int* r = h->tucker_rank[t];  // (x, y, z)
        hd[t] = ModeDesc{h->tucker_off[t], (long long)t * nd, h->tucker_off[t] + (long long)r[2] * r[1] * r[0] +
                                                              (long long)n[0] * r[2] + (long long)n[1] * r[1],
                         {r[2], r[1], r[0]}, n[2], r[0]};
    }
    rc = launch_modes(base, w1, base, hd, dd, 2, 1, s);
    // expand y: [rz][ry][nx] -> [rz][ny][nx]
    for (int t = 0; rc == VIE_OK && t < kT; ++t) {
        const int* r = h->tucker_rank[t];
        hd[t] = ModeDesc{(long long)t * nd, (long long)t * nd, h->tucker_off[t] + (long long)r[2] * r[1] * r[0] +
                                                                   (long long)n[0] * r[2],
                         {r[2], r[1], n[2]}, n[1], r[1]};
    }
    if (rc == VIE_OK) rc = launch_modes(w1, w2, base, hd, dd, 1, 1, s);
    // expand z: [rz][ny][nx] -> [nz][ny][nx]
    for (int t = 0; rc == VIE_OK && t < kT; ++t) {
        const int* r = h->tucker_rank[t];
        hd[t] = ModeDesc{(long long)t * nd, (long long)t * nd, h->tucker_off[t] + (long long)r[2] * r[1] * r[0],
                         {r[2], n[1], n[2]}, n[0], r[2]};
    }
    if (rc == VIE_OK) rc = launch_modes(w2, out, base, hd, dd, 0, 1, s);
    cudaFree(w);
    cudaFree(dd);
    return rc;
}

// Tucker compression of the 60 tensors T (device [60][nz][ny][nx]) into the handle's Tucker
// form; ranks[t] = (r_x, r_y, r_z), err[t] = ||T - T~|| / ||T|| (host arrays, optional).
int tucker_compress(vie_handle* h, const double2* T, double tol, int* ranks, double* err, cudaStream_t s) {
    const int n[3] = {h->nz, h->ny, h->nx};
    const long long nd = (long long)h->nv;
    // Gram matrices of the three unfoldings, mode order (z, y, x)
    size_t goff[3], gtot = 0;
    for (int k = 0; k < 3; ++k) {
        goff[k] = gtot;
        gtot += (size_t)kT * n[k] * n[k];
    }
    double2* G = nullptr;
    if (cudaMalloc(&G, sizeof(double2) * gtot) != cudaSuccess) {
        cudaGetLastError();
        set_error("Gram matrix allocation failed");
        return VIE_ENOMEM;
    }
    const GramGeo geo[3] = {
        // z: rows i = z, k = (y, x) contiguous
        {1, 0, (long long)n[1] * n[2], (long long)n[1] * n[2], 1, n[0]},
        // y: rows i = y, k = (z, x)
        {(long long)n[1] * n[2], 1, n[2], (long long)n[0] * n[2], n[2], n[1]},
        // x: rows i = x, k = (z, y)
        {n[2], 0, 1, (long long)n[0] * n[1], 1, n[2]},
    };
    for (int k = 0; k < 3; ++k) {
        const unsigned b = (unsigned)((n[k] + 15) / 16);
        VIE_KLAUNCH("tucker_gram", s, gram_kernel<<<dim3(b, b, kT), dim3(16, 16), 0, s>>>(T, nd, geo[k], G + goff[k]));
    }
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(G);
        set_error("Gram kernel launch failed");
        return VIE_EDEVICE;
    }
    std::vector<cplx> hG(gtot);
    if (cudaMemcpyAsync(hG.data(), G, sizeof(double2) * gtot, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(G);
        set_error("Gram matrix copy failed");
        return VIE_EDEVICE;
    }
    cudaFree(G);
    // factors per tensor and mode; the Tucker form of tensor t is stored as
    //   core [rz][ry][rx], U_z [nz][rz], U_y [ny][ry], U_x [nx][rx]
    std::vector<std::vector<cplx>> Uf(3 * kT);
    int rk[kT][3];  // (z, y, x)
    for (int t = 0; t < kT; ++t) {
        double norm2 = 0.0;
        for (int i = 0; i < n[0]; ++i) norm2 += hG[goff[0] + ((size_t)t * n[0] + i) * n[0] + i].real();
        const double thr = tol * tol * norm2 / 3.0;
        for (int k = 0; k < 3; ++k)
            Uf[3 * t + k] = range_basis(hG.data() + goff[k] + (size_t)t * n[k] * n[k], n[k], thr, &rk[t][k]);
    }
    long long total = 0;
    long long off[kT];
    for (int t = 0; t < kT; ++t) {
        off[t] = total;
        total += (long long)rk[t][0] * rk[t][1] * rk[t][2] + (long long)n[0] * rk[t][0] + (long long)n[1] * rk[t][1] +
                 (long long)n[2] * rk[t][2];
    }
    std::vector<cplx> hform((size_t)total, cplx(0.0));
    for (int t = 0; t < kT; ++t) {
        long long o = off[t] + (long long)rk[t][0] * rk[t][1] * rk[t][2];
        for (int k = 0; k < 3; ++k) {
            std::copy(Uf[3 * t + k].begin(), Uf[3 * t + k].end(), hform.begin() + o);
            o += (long long)n[k] * rk[t][k];
        }
    }
    double2* form = nullptr;
    double2* w = nullptr;
    ModeDesc* dd = nullptr;
    auto fail = [&](int code, const char* msg) {
        cudaGetLastError();
        cudaFree(form);
        cudaFree(w);
        cudaFree(dd);
        set_error(msg);
        return code;
    };
    if (cudaMalloc(&form, sizeof(double2) * (size_t)total) != cudaSuccess ||
        cudaMalloc(&w, sizeof(double2) * 2 * kT * nd) != cudaSuccess ||
        cudaMalloc(&dd, sizeof(ModeDesc) * kT) != cudaSuccess)
        return fail(VIE_ENOMEM, "Tucker form allocation failed");
    if (cudaMemcpyAsync(form, hform.data(), sizeof(double2) * (size_t)total, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(VIE_EDEVICE, "Tucker factor copy failed");
    // core: compress x, then y, then z
    double2 *w1 = w, *w2 = w + kT * nd;
    std::vector<ModeDesc> hd(kT);
    for (int t = 0; t < kT; ++t) {
        const long long ux = off[t] + (long long)rk[t][0] * rk[t][1] * rk[t][2] + (long long)n[0] * rk[t][0] +
                             (long long)n[1] * rk[t][1];
        hd[t] = ModeDesc{(long long)t * nd, (long long)t * nd, ux, {n[0], n[1], n[2]}, rk[t][2], rk[t][2]};
    }
    int rc = launch_modes(T, w1, form, hd, dd, 2, 0, s);
    for (int t = 0; rc == VIE_OK && t < kT; ++t) {
        const long long uy = off[t] + (long long)rk[t][0] * rk[t][1] * rk[t][2] + (long long)n[0] * rk[t][0];
        hd[t] = ModeDesc{(long long)t * nd, (long long)t * nd, uy, {n[0], n[1], rk[t][2]}, rk[t][1], rk[t][1]};
    }
    if (rc == VIE_OK) rc = launch_modes(w1, w2, form, hd, dd, 1, 0, s);
    for (int t = 0; rc == VIE_OK && t < kT; ++t) {
        const long long uz = off[t] + (long long)rk[t][0] * rk[t][1] * rk[t][2];
        hd[t] = ModeDesc{(long long)t * nd, off[t], uz, {n[0], rk[t][1], rk[t][2]}, rk[t][0], rk[t][0]};
    }
    if (rc == VIE_OK) rc = launch_modes(w2, form, form, hd, dd, 0, 0, s);
    cudaFree(w);
    cudaFree(dd);
    w = nullptr;
    dd = nullptr;
    if (rc < 0) return fail(rc, "Tucker core computation failed");
    // install in the handle (replacing an earlier form)
    if (h->tucker) {
        cudaFree(h->tucker);
        h->bytes_held -= h->tucker_bytes;
    }
    h->tucker = form;
    h->tucker_bytes = sizeof(double2) * (size_t)total;
    h->bytes_held += h->tucker_bytes;
    for (int t = 0; t < kT; ++t) {
        h->tucker_off[t] = off[t];
        h->tucker_rank[t][0] = rk[t][2];  // (x, y, z)
        h->tucker_rank[t][1] = rk[t][1];
        h->tucker_rank[t][2] = rk[t][0];
        if (ranks)
            for (int k = 0; k < 3; ++k) ranks[3 * t + k] = h->tucker_rank[t][k];
    }
    if (err) {
        double2* R = nullptr;
        double2* part = nullptr;
        constexpr int nb = 64;
        if (cudaMalloc(&R, sizeof(double2) * kT * nd) != cudaSuccess ||
            cudaMalloc(&part, sizeof(double2) * kT * nb) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(R);
            set_error("Tucker error scratch allocation failed");
            return VIE_ENOMEM;
        }
        rc = tucker_reconstruct(h, R, s);
        if (rc == VIE_OK) {
            VIE_KLAUNCH("tucker_error", s, diff_norm_kernel<<<dim3(nb, kT), 256, 0, s>>>(T, R, nd, part));
            std::vector<double2> hp(kT * nb);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(hp.data(), part, sizeof(double2) * kT * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                set_error("Tucker error reduction failed");
                rc = VIE_EDEVICE;
            } else {
                for (int t = 0; t < kT; ++t) {
                    double a = 0.0, b = 0.0;
                    for (int i = 0; i < nb; ++i) a += hp[t * nb + i].x, b += hp[t * nb + i].y;
                    err[t] = b > 0.0 ? std::sqrt(a / b) : 0.0;
                }
            }
        }
        cudaFree(R);
        cudaFree(part);
    }
    return rc;
}

// vie_green_tucker's work: compress the handle's table; with `apply`, rebuild the Green spectra
// from the reconstruction and keep the Tucker form in place of the table.
int green_tucker(vie_handle* h, double tol, bool apply, int* ranks, double* err, size_t* bytes) {
    cudaStream_t s = h->stream;
    double2* T = h->toeplitz;
    double2* own = nullptr;
    if (!T) {  // an earlier application dropped the table: start from the reconstruction
        if (cudaMalloc(&own, sizeof(double2) * kT * h->nv) != cudaSuccess) {
            cudaGetLastError();
            set_error("Toeplitz scratch allocation failed");
            return VIE_ENOMEM;
        }
        int rc = tucker_reconstruct(h, own, s);
        if (rc < 0) {
            cudaFree(own);
            return rc;
        }
        T = own;
    }
    int rc = tucker_compress(h, T, tol, ranks, err, s);
    if (rc == VIE_OK && apply) {
        double2* R = nullptr;
        if (cudaMalloc(&R, sizeof(double2) * kT * h->nv) != cudaSuccess) {
            cudaGetLastError();
            set_error("reconstruction allocation failed");
            rc = VIE_ENOMEM;
        } else {
            rc = tucker_reconstruct(h, R, s);
            if (rc == VIE_OK) rc = green_embed(h, R, false);  // takes R
            else cudaFree(R);
            if (rc == VIE_OK && h->toeplitz) {
                cudaFree(h->toeplitz);
                h->toeplitz = nullptr;
                h->bytes_held -= sizeof(double2) * kT * h->nv;
            }
        }
    }
    if (own) cudaFree(own);
    if (rc == VIE_OK && bytes) *bytes = h->tucker_bytes;
    return rc;
}
