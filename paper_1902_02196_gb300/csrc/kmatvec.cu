// K operator (K u = curl S u, Eq. 8): its Green tensors in octant storage for the matvec, so
// that y = K x (the tested scattered magnetic field h~ = K x, Eq. 13: h_sca = K j) runs the
// same transforms as the N operator (Section IV-A) with the K block in the z pass, in FP64 or
// FP32: the fused z passes with KOP (zpass_f32.cu, zpass_f64.cu), or the generic one
// (matvec.cu, zpass_kernel with KOP) for FFT lengths along z outside 8..512.
//
// The 30 Toeplitz tensors P_t (green.cu, assemble_k_kernel) are embedded into full 2N
// circulants, the entries at negative offsets taken from the reflection parities of the block
// table (kblock.h), transformed, and their octant k_i in [0, L_i/2] kept, scaled by
// 1/(Lx Ly Lz), as [30][Oz][Oy][Ox] in FP64 and FP32, and once more in both as [Oy][Ox][Oz][30]
// (the 30 values of a point side by side, for the fused z passes).  The other octants follow
// in the z pass from the same parities: K(R_i k) = -S_i K(k) S_i.  Built on the first K product
// of a handle and released with it.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kblock.h"

int green_k_toeplitz(vie_handle* h, double2* out, cudaStream_t s);  // green.cu

namespace {

std::mutex g_kmu;  // the first K product of a handle builds its spectra once

// circulants of tensors t0 .. t0 + nt - 1: C_t(j) = P_t(d), d = j (j < N) or j - L (j > L - N),
// else 0 per axis, with the reflection parity of the tensor's representative entry
__global__ void embed_k_kernel(const double2* __restrict__ P, int nx, int ny, int nz, int Lx, int Ly, int Lz, int t0,
                               int nt, double2* __restrict__ C) {
    const long long vol = (long long)Lx * Ly * Lz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= vol * nt) return;
    const int t = t0 + (int)(gid / vol);
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

// octant k_i in [0, L_i/2] of the transformed circulants of tensors t0 .. t0 + nt - 1, scaled
__global__ void k_octant_kernel(const double2* __restrict__ C, int Lx, int Ly, int Lz, int t0, int nt, double scale,
                                double2* __restrict__ g64, float2* __restrict__ g32, float2* __restrict__ g32t,
                                double2* __restrict__ g64t) {
    const int Ox = Lx / 2 + 1, Oy = Ly / 2 + 1, Oz = Lz / 2 + 1;
    const long long ovol = (long long)Ox * Oy * Oz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= ovol * nt) return;
    const int tl = (int)(gid / ovol);
    const long long o = gid % ovol;
    const int kx = (int)(o % Ox), ky = (int)((o / Ox) % Oy), kz = (int)(o / ((long long)Ox * Oy));
    double2 v = C[(long long)tl * Lx * Ly * Lz + ((long long)kz * Ly + ky) * Lx + kx];
    v.x *= scale;
    v.y *= scale;
    const long long dst = (long long)(t0 + tl) * ovol + o;
    g64[dst] = v;
    g32[dst] = make_float2((float)v.x, (float)v.y);
    const long long dt = (((long long)ky * Ox + kx) * Oz + kz) * 30 + t0 + tl;
    g32t[dt] = make_float2((float)v.x, (float)v.y);
    g64t[dt] = v;
}

unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// the K octant spectra of the handle (h->kgreen64, h->kgreen32), built on first use
int k_octants(vie_handle* h, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_kmu);
    if (h->kgreen64) return VIE_OK;
    const int Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    const long long vol = (long long)Lx * Ly * Lz, nd = (long long)h->nv;
    const long long ovol = (long long)h->O[0] * h->O[1] * h->O[2];
    const int chunk = (int)std::max<long long>(1, std::min<long long>(30, (4LL << 30) / (vol * (long long)sizeof(double2))));
    double2 *P = nullptr, *C = nullptr, *g64 = nullptr, *g64t = nullptr;
    float2 *g32 = nullptr, *g32t = nullptr;
    auto fail = [&](int code, const char* msg) {
        cudaGetLastError();
        cudaFree(P);
        cudaFree(C);
        cudaFree(g64);
        cudaFree(g32);
        cudaFree(g32t);
        cudaFree(g64t);
        set_error(msg);
        return code;
    };
    if (cudaMalloc(&P, sizeof(double2) * 30 * nd) != cudaSuccess ||
        cudaMalloc(&C, sizeof(double2) * vol * chunk) != cudaSuccess ||
        cudaMalloc(&g64, sizeof(double2) * 30 * ovol) != cudaSuccess ||
        cudaMalloc(&g32, sizeof(float2) * 30 * ovol) != cudaSuccess ||
        cudaMalloc(&g32t, sizeof(float2) * 30 * ovol) != cudaSuccess ||
        cudaMalloc(&g64t, sizeof(double2) * 30 * ovol) != cudaSuccess)
        return fail(VIE_ENOMEM, "K spectrum allocation failed");
    int rc = green_k_toeplitz(h, P, s);
    for (int t0 = 0; rc == VIE_OK && t0 < 30; t0 += chunk) {
        const int nt = std::min(chunk, 30 - t0);
        VIE_KLAUNCH("k_embed", s,
                    embed_k_kernel<<<blocks(vol * nt), 256, 0, s>>>(P, h->nx, h->ny, h->nz, Lx, Ly, Lz, t0, nt, C));
        if (cudaGetLastError() != cudaSuccess) return fail(VIE_EDEVICE, "K embed launch failed");
        rc = fft3d_inplace64(h, C, nt, s);
        if (rc < 0) break;
        VIE_KLAUNCH("k_octant", s,
                    k_octant_kernel<<<blocks(ovol * nt), 256, 0, s>>>(C, Lx, Ly, Lz, t0, nt, 1.0 / (double)vol, g64,
                                                                      g32, g32t, g64t));
        if (cudaGetLastError() != cudaSuccess) return fail(VIE_EDEVICE, "K octant launch failed");
    }
    if (rc == VIE_OK && cudaStreamSynchronize(s) != cudaSuccess) return fail(VIE_EDEVICE, "K spectrum sync failed");
    if (rc < 0) {
        cudaFree(P);
        cudaFree(C);
        cudaFree(g64);
        cudaFree(g32);
        cudaFree(g32t);
        cudaFree(g64t);
        return rc;
    }
    cudaFree(P);
    cudaFree(C);
    h->kgreen64 = g64;
    h->kgreen32 = g32;
    h->kgreen32t = g32t;
    h->kgreen64t = g64t;
    h->bytes_held += 2 * (sizeof(double2) + sizeof(float2)) * 30 * (size_t)ovol;  // until kmatvec_release
    return VIE_OK;
}

// y = K x, FP64, x and y device [R][12][nz][ny][nx]
int kmatvec_device(vie_handle* h, int R, const double2* x, double2* y, cudaStream_t s) {
    return matvec_device(h, R, x, y, VIE_FP64, VIE_OP_K, s);
}

// frees the handle's K spectra, if any (called when the handle is released)
void kmatvec_release(vie_handle* h) {
    if (!h->kgreen64) return;
    cudaFree(h->kgreen64);
    cudaFree(h->kgreen32);
    cudaFree(h->kgreen32t);
    cudaFree(h->kgreen64t);
    h->kgreen64 = nullptr;
    h->kgreen32 = nullptr;
    h->kgreen32t = nullptr;
    h->kgreen64t = nullptr;
    h->bytes_held -= 2 * (sizeof(double2) + sizeof(float2)) * 30 * (size_t)h->O[0] * h->O[1] * h->O[2];
}
