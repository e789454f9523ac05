// K operator matvec (K u = curl S u, Eq. 8), FP64: y = K x for nrhs vectors by circulant
// embedding and 3-D FFTs (Section IV-A), the tested scattered magnetic field h~ = K x
// (Eq. 13: h_sca = K j).
//
// The 30 Toeplitz tensors P_t (green.cu, assemble_k_kernel) are embedded into full 2N
// circulants, the entries at negative offsets taken from the reflection parities of the
// block table (kblock.h), and transformed once per handle (kept in a table keyed by the
// handle, released with it).  A matvec pads x into [12R][Lz][Ly][Lx], transforms forward,
// applies the signed 12 x 12 K block at every frequency point, and transforms back as
// conj(FFT(conj(.))) with the same forward transform; the 1/(Lx Ly Lz) of the inverse is
// folded into the block product.  Correctness path: full spectra, no octant storage.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "kblock.h"

int green_k_toeplitz(vie_handle* h, double2* out, cudaStream_t s);  // green.cu

namespace {

std::mutex g_kmu;
std::unordered_map<const vie_handle*, double2*> g_kspec;  // [30][Lz][Ly][Lx] transformed circulants

// circulant of the 30 tensors: C_t(j) = P_t(d), d = j (j < N) or j - L (j > L - N), else 0 per axis
__global__ void embed_k_kernel(const double2* __restrict__ P, int nx, int ny, int nz, int Lx, int Ly, int Lz,
                               double2* __restrict__ C) {
    const long long vol = (long long)Lx * Ly * Lz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= vol * 30) return;
    const int t = (int)(gid / vol);
    const long long j = gid % vol;
    const int J[3] = {(int)(j % Lx), (int)((j / Lx) % Ly), (int)(j / ((long long)Lx * Ly))};
    const int N[3] = {nx, ny, nz}, Lv[3] = {Lx, Ly, Lz};
    // representative entry of tensor t = 10 jd + ll: (p, q) = (jd + 1, jd + 2) mod 3
    const int jd = t / 10, ll = t % 10;
    const int LA[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4}, LB[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
    const int a = 4 * ((jd + 1) % 3) + LA[ll] - 1, b = 4 * ((jd + 2) % 3) + LB[ll] - 1;
    int d[3];
    int sgn = 1;
    for (int i = 0; i < 3; ++i) {
        if (J[i] < N[i]) {
            d[i] = J[i];
        } else if (J[i] > Lv[i] - N[i]) {
            d[i] = Lv[i] - J[i];
            sgn *= kblock::reflection(a, b, i);
        } else {
            C[gid] = make_double2(0, 0);
            return;
        }
    }
    double2 v = P[(long long)t * nx * ny * nz + ((long long)d[2] * ny + d[1]) * nx + d[0]];
    if (sgn < 0) v = make_double2(-v.x, -v.y);
    C[gid] = v;
}

// W[r][a] (vol each) <- x[r][a] zero-padded from [nz][ny][nx] to [Lz][Ly][Lx]
__global__ void pad_kernel(const double2* __restrict__ x, int nx, int ny, int nz, int Lx, int Ly, int Lz,
                           long long planes, double2* __restrict__ W) {
    const long long vol = (long long)Lx * Ly * Lz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= vol * planes) return;
    const long long c = gid / vol, j = gid % vol;
    const int jx = (int)(j % Lx), jy = (int)((j / Lx) % Ly), jz = (int)(j / ((long long)Lx * Ly));
    double2 v = make_double2(0, 0);
    if (jx < nx && jy < ny && jz < nz) v = x[((c * nz + jz) * ny + jy) * nx + jx];
    W[gid] = v;
}

// at every frequency point of every right-hand side: Y_a = s sum_b sign(a, b) KS_t(a,b) X_b, stored
// conjugated for the inverse by the forward transform; s = 1 / (Lx Ly Lz)
__global__ void kblock_kernel(double2* __restrict__ W, const double2* __restrict__ KS, long long vol, int R,
                              double s) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= vol * R) return;
    const long long r = gid / vol, k = gid % vol;
    double2* w = W + r * 12 * vol + k;
    double2 X[12];
#pragma unroll
    for (int b = 0; b < 12; ++b) X[b] = w[b * vol];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        double2 acc = make_double2(0, 0);
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const int t = kblock::tensor(a, b);
            if (t < 0) continue;
            const double2 g = KS[(long long)t * vol + k];
            const double sg = (double)kblock::sign(a, b);
            acc.x += sg * (g.x * X[b].x - g.y * X[b].y);
            acc.y += sg * (g.x * X[b].y + g.y * X[b].x);
        }
        w[a * vol] = make_double2(s * acc.x, -s * acc.y);
    }
}

// y[c] <- conj(W[c]) cropped from [Lz][Ly][Lx] to [nz][ny][nx]
__global__ void crop_conj_kernel(const double2* __restrict__ W, int nx, int ny, int nz, int Lx, int Ly, int Lz,
                                 long long planes, double2* __restrict__ y) {
    const long long nv = (long long)nx * ny * nz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nv * planes) return;
    const long long c = gid / nv, i = gid % nv;
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    const double2 v = W[c * (long long)Lx * Ly * Lz + ((long long)iz * Ly + iy) * Lx + ix];
    y[gid] = make_double2(v.x, -v.y);
}

unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

// the transformed K circulants of this handle, built on first use
int kspectrum(vie_handle* h, cudaStream_t s, const double2** out) {
    std::lock_guard<std::mutex> lk(g_kmu);
    auto it = g_kspec.find(h);
    if (it != g_kspec.end()) {
        *out = it->second;
        return VIE_OK;
    }
    const int Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    const long long vol = (long long)Lx * Ly * Lz, nd = (long long)h->nv;
    double2 *P = nullptr, *C = nullptr;
    if (cudaMalloc(&P, sizeof(double2) * 30 * nd) != cudaSuccess ||
        cudaMalloc(&C, sizeof(double2) * 30 * vol) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(P);
        cudaFree(C);
        set_error("K spectrum allocation failed");
        return VIE_ENOMEM;
    }
    int rc = green_k_toeplitz(h, P, s);
    if (rc == VIE_OK) {
        VIE_KLAUNCH("k_embed", s, embed_k_kernel<<<blocks(vol * 30), 256, 0, s>>>(P, h->nx, h->ny, h->nz, Lx, Ly, Lz, C));
        if (cudaGetLastError() != cudaSuccess) rc = (set_error("K embed launch"), VIE_EDEVICE);
    }
    if (rc == VIE_OK) rc = fft3d_inplace64(h, C, 30, s);
    if (rc == VIE_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = (set_error("K spectrum sync"), VIE_EDEVICE);
    cudaFree(P);
    if (rc != VIE_OK) {
        cudaFree(C);
        return rc;
    }
    g_kspec[h] = C;
    h->bytes_held += sizeof(double2) * 30 * (size_t)vol;  // counted until kmatvec_release
    *out = C;
    return VIE_OK;
}

// right-hand sides per pass of the K matvec: the padded spectra of a pass ([12 Rc][Lz][Ly][Lx]
// FP64) stay within 4 GiB of scratch, one right-hand side at least
constexpr size_t kKPassBytes = size_t(4) << 30;

}  // namespace

// y = K x, FP64, x and y device [R][12][nz][ny][nx]; the right-hand sides go through in passes
// of at most kKPassBytes of padded spectra each
int kmatvec_device(vie_handle* h, int R, const double2* x, double2* y, cudaStream_t s) {
    const double2* KS = nullptr;
    VIE_TRY(kspectrum(h, s, &KS));
    const int Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    const long long vol = (long long)Lx * Ly * Lz, nv = (long long)h->nv;
    const size_t per_rhs = sizeof(double2) * 12 * (size_t)vol;
    const int Rc = (int)std::max<size_t>(1, std::min<size_t>((size_t)R, kKPassBytes / per_rhs));
    VIE_TRY(ws_reserve(h, h->post_ws, per_rhs * (size_t)Rc));
    double2* W = static_cast<double2*>(h->post_ws.ptr);
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int Rp = std::min(Rc, R - r0);
        const long long planes = 12LL * Rp;
        const double2* xp = x + (long long)r0 * 12 * nv;
        double2* yp = y + (long long)r0 * 12 * nv;
        VIE_KLAUNCH("k_pad", s,
                    pad_kernel<<<blocks(vol * planes), 256, 0, s>>>(xp, h->nx, h->ny, h->nz, Lx, Ly, Lz, planes, W));
        VIE_CHECK_LAUNCH();
        VIE_TRY(fft3d_inplace64(h, W, (int)planes, s));
        VIE_KLAUNCH("k_block", s, kblock_kernel<<<blocks(vol * Rp), 256, 0, s>>>(W, KS, vol, Rp, 1.0 / (double)vol));
        VIE_CHECK_LAUNCH();
        VIE_TRY(fft3d_inplace64(h, W, (int)planes, s));
        VIE_KLAUNCH("k_crop", s,
                    crop_conj_kernel<<<blocks(nv * planes), 256, 0, s>>>(W, h->nx, h->ny, h->nz, Lx, Ly, Lz, planes,
                                                                           yp));
        VIE_CHECK_LAUNCH();
    }
    return VIE_OK;
}

// frees the handle's K spectrum, if any (called when the handle is released)
void kmatvec_release(vie_handle* h) {
    std::lock_guard<std::mutex> lk(g_kmu);
    auto it = g_kspec.find(h);
    if (it == g_kspec.end()) return;
    cudaFree(it->second);
    g_kspec.erase(it);
    h->bytes_held -= sizeof(double2) * 30 * (size_t)h->L[0] * h->L[1] * h->L[2];
}
