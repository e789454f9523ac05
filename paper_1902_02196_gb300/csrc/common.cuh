// Internal declarations shared by the translation units of libvie.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vie.h"

// ---------------------------------------------------------------------------
// Complex helpers on float2 / double2
// ---------------------------------------------------------------------------
template <typename T>
struct CT;
template <>
struct CT<float> {
    using C = float2;
};
template <>
struct CT<double> {
    using C = double2;
};

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C>
__host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C>
__host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C>
__host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C>
__host__ __device__ __forceinline__ C cneg(C a) { return mk(-a.x, -a.y); }
// multiply by -i (dir = -1) or +i (dir = +1)
template <typename C>
__host__ __device__ __forceinline__ C cmul_i(C a, int dir) { return dir < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x); }
// acc += a * b
template <typename C>
__host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cfma_f(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

// ---------------------------------------------------------------------------
// The 60 unique tensors of N (Section III-C): t = 10 * pq + ll.
//   pq : unordered vector pair (xx, xy, xz, yy, yz, zz)
//   ll : ordered scalar pair l <= l' ((1,1),(1,2),(1,3),(1,4),(2,2),(2,3),(2,4),(3,3),(3,4),(4,4))
// Entry (alpha = 4p + l - 1, beta = 4q + l' - 1) of the 12 x 12 block equals
// sgn * U_t with, for l > l', the swap relation N^{pl,ql'} = (-1)^{[l>1]+[l'>1]} N^{pl',ql}
// (reciprocity combined with the point-inversion parity of the PWL functions).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pq_index(int p, int q) {
    return p > q ? pq_index(q, p) : (p == 0 ? q : (p == 1 ? 2 + q : 5));
}
__host__ __device__ constexpr int ll_index(int l, int lp) {  // 1-based, l <= lp
    return l > lp ? ll_index(lp, l) : (l == 1 ? lp - 1 : (l == 2 ? 2 + lp : (l == 3 ? 4 + lp : 9)));
}
__host__ __device__ constexpr int tensor_of(int a, int b) {
    return 10 * pq_index(a / 4, b / 4) + ll_index(a % 4 + 1, b % 4 + 1);
}
__host__ __device__ constexpr int sign_of(int a, int b) {
    return ((a % 4) > (b % 4)) ? ((((a % 4) > 0) + ((b % 4) > 0)) % 2 ? -1 : 1) : 1;
}
// reflection parity of component alpha under x_i -> -x_i: -1 if p == i, times -1 if N^l is linear along i
__host__ __device__ constexpr int parity_of(int a, int i) {
    return ((a / 4 == i) ? -1 : 1) * ((a % 4 == i + 1) ? -1 : 1);
}
// Gram entry of component alpha (Eq. 33): G^1 = DV for the constant function, DV/12 for the
// linear ones; in the PWC layout (nc = 3 components per voxel) every component is a constant function
__host__ __device__ __forceinline__ bool comp_is_constant(int alpha, int nc) { return nc == 3 || alpha % 4 == 0; }

// bit mask over the 12 components of parity -1 under reflection of axis i
__host__ __device__ constexpr unsigned flip_mask(int i) {
    unsigned m = 0;
    for (int a = 0; a < 12; ++a)
        if (parity_of(a, i) < 0) m |= 1u << a;
    return m;
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct vie_handle {
    int nx, ny, nz;
    int nc;  // unknowns per voxel: 12 (PWL, 4 scalar functions x 3 components) or 3 (PWC: l = 1 only)
    double dx, dy, dz;
    double freq, omega, k0;
    int L[3];   // FFT lengths (x, y, z), powers of two >= 2N - 1
    int O[3];   // octant sizes L/2 + 1
    size_t nv;  // nx*ny*nz
    cudaStream_t stream;
    int device;
    // per-voxel coefficients (complex): eps, chi, tau, 1/eps; double and float copies
    double2 *eps64, *chi64, *tau64, *ieps64;
    float2 *chi32, *tau32, *ieps32;
    // FFT'd circulant Green tensors (of N - G), octant k_i in [0, L_i/2], pre-scaled by 1/(Lx Ly Lz):
    // layout [60][Oz][Oy][Ox]
    double2* green64;
    float2* green32;
    // FP32 copy in the layout of the z pass of the FP32 three-kernel path: [Oy][Ox][Oz][60]
    float2* green32t;
    // FP64 copy in the same layout, for the FP64 fused z pass
    double2* green64t;
    // the 30 K tensors' transformed circulants, octant storage [30][Oz][Oy][Ox], scaled by
    // 1/(Lx Ly Lz), FP64 and FP32 (kmatvec.cu, built on the first K product)
    double2* kgreen64;
    float2* kgreen32;
    // copies [Oy][Ox][Oz][30] for the fused z passes with the K block (zpass_f32.cu, zpass_f64.cu)
    float2* kgreen32t;
    double2* kgreen64t;
    // bf16 split of green32t in the same layout, for the BF16x3 z pass: per tensor (hi, lo),
    // each a bf16 (re, im) pair with hi = bf16(v), lo = bf16(v - hi)
    uint2* greenbf;
    // stored column order of that path's spectrum: [Lx] kx per stored column, then [Lx]
    // positions of those kx in the x transform's output order (square L <= 128 only, else null)
    unsigned char* colmap;
    // stored column order of every matvec spectrum, any Lx: colkx32[sc] = kx of stored column sc
    // (mirror pairs (kx, Lx - kx) side by side, columns 0 and Lx/2 last; the order of colmap
    // when that exists), colpos32[kx] = its stored column
    int* colkx32;
    int* colpos32;
    // twiddle tables exp(-2 pi i m / L) for L = 2^k, k = 1..11, concatenated at offset L
    double2* tw64;
    float2* tw32;
    // scratch
    Workspace fft_ws;    // matvec spectrum buffers
    Workspace stage_ws;  // host-buffer staging
    Workspace solve_ws;  // solver vectors
    Workspace support_ws;  // support rows of the current solve
    Workspace post_ws;     // vie_fields scratch
    // The point of the last FP64 residual matvec of vie_solve, for vie_fields: the solution
    // x1 and the convolution (N - G) x1, both full grid [fcache_R][12][nz][ny][nx] FP64
    // (x1 first, then the product); valid for fcache_R right-hand sides when fcache_valid.
    Workspace fcache_ws;
    int fcache_R;
    int fcache_valid;
    // full JM-VIE (jmvie.cu), allocated together on first use: relative permeability mu, chi_m = mu - 1,
    // 1/mu and the support indicator |chi_e| + |chi_m|, each [nz][ny][nx] (mu = 1 until set)
    double2 *mu64, *chim64, *imu64, *jmsup64;
    Workspace jm_ws;  // (N - G) x and K x of the stacked currents
    double2* toeplitz;   // [60][nz][ny][nx] Toeplitz tensors of N - G for offsets d >= 0 (NULL once a
                         // Tucker form replaced it, see tucker.cu)
    // Tucker form of the 60 tensors (tucker.cu): per tensor t at element offset tucker_off[t] the
    // core [rz][ry][rx], then U_z [nz][rz], U_y [ny][ry], U_x [nx][rx]; tucker_rank[t] = (rx, ry, rz)
    void* tucker;
    size_t tucker_bytes;
    long long tucker_off[60];
    int tucker_rank[60][3];
    size_t bytes_held;
    // set when green64/32/32t, toeplitz, the twiddle tables and colmap belong to another
    // handle (a template kept in a server's Green cache) and must not be freed with this one
    int shared_green;
    // set for a server request's handle: its own memory (material maps, workspaces) is
    // allocated and freed in stream order on its stream (cudaMallocAsync / cudaFreeAsync from the
    // device's memory pool), so that a request's allocations and frees do not synchronise the
    // device under the other requests' work
    int async_alloc;
};

// vie_setup with an optional template: when share != NULL the new handle takes the
// template's Green tensors, twiddles and column map (same grid, voxel and frequency
// required) and computes only its own material maps.
// ext (optional, no template): the caller's Toeplitz table [144][2nz-1][2ny-1][2nx-1] complex128
// (host or device) from which the Green tensors are taken instead of being computed
// (vie_setup_green_external).
// nc: unknowns per voxel, 12 (PWL) or 3 (PWC, vie_setup flag VIE_SETUP_PWC).
int handle_create(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma,
                  const vie_handle* share, vie_handle** out, const void* ext = nullptr, int nc = 12);
// device bytes held by a handle's Green tensors, twiddles and column map (shared part)
size_t handle_green_bytes(const vie_handle* h);

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
#define VIE_CUDA(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_) + " at " + __FILE__ + ":" +  \
                      std::to_string(__LINE__));                                                       \
            return e_ == cudaErrorMemoryAllocation ? VIE_ENOMEM : VIE_EDEVICE;                         \
        }                                                                                              \
    } while (0)
#define VIE_CHECK_LAUNCH() VIE_CUDA(cudaGetLastError())
#define VIE_TRY(expr)             \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ < 0) return rc_;  \
    } while (0)

int ws_reserve(vie_handle* h, Workspace& w, size_t bytes);
// device memory owned by handle h: stream-ordered on h's stream when h->async_alloc, else plain
cudaError_t dev_malloc(const vie_handle* h, void** p, size_t bytes);
void dev_free(const vie_handle* h, void* p);

// ---------------------------------------------------------------------------
// Launch accounting (stats.cu): every kernel launch of the library is counted per
// kernel name; when timing is enabled, CUDA events recorded on the launch stream
// around each launch give its device duration.
// ---------------------------------------------------------------------------
struct LaunchScope {
    LaunchScope(const char* name, cudaStream_t s, double alg_bytes = 0.0);
    ~LaunchScope();
    const char* name;
    cudaStream_t stream;
    bool timed;
    cudaEvent_t ev0, ev1;
};
#define VIE_KLAUNCH(name, stream, ...) \
    do {                                \
        LaunchScope ls_(name, stream);  \
        __VA_ARGS__;                    \
    } while (0)
// same, recording the launch's algorithmic bytes (known on the host)
#define VIE_KLAUNCH_B(name, stream, bytes, ...) \
    do {                                         \
        LaunchScope ls_(name, stream, bytes);    \
        __VA_ARGS__;                             \
    } while (0)
// algorithmic bytes counted on the device by the Gram-Schmidt kernels (solve.cu):
// [0] gs_dots, [1] gs_update, [2] solution_update; optionally reset
int solve_device_bytes(double out[3], bool reset);

// Launches whose right-hand side count is known only on the device (the solver's active list)
// count themselves on the device, per kernel name: ctr[0] += algorithmic bytes and ctr[1] += 1
// when the launch has work (a launch whose list is empty returns at once and is not counted).
// dev_bytes_ptr(name) is the pair's address on the current device (NULL if it cannot be had);
// such launches pass kDevCounted as their host-side bytes, and vie_stats_read adds the counters in.
constexpr double kDevCounted = -1.0;
unsigned long long* dev_bytes_ptr(const char* name);
__device__ __forceinline__ void dev_bytes_add(unsigned long long* ctr, double bytes, bool work) {
    if (ctr && work && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(ctr, (unsigned long long)bytes);
        atomicAdd(ctr + 1, 1ull);
    }
}

// Launch accounting of CUDA graphs.  Between stats_capture_begin and stats_capture_end (on the
// capturing thread) every LaunchScope appends a record to `list` instead of counting, with
// event-record nodes around the launch when timing is on; each replay of the graph is then
// counted by stats_graph_replayed, and its device times are added by stats_graph_harvest
// once the replay has finished.  stats_capture_release destroys the records' events.
struct CapRec {
    std::string name;
    double bytes;
    cudaEvent_t ev0, ev1;
};
void stats_capture_begin(std::vector<CapRec>* list);
void stats_capture_end();
void stats_graph_replayed(const std::vector<CapRec>& list);
void stats_graph_harvest(const std::vector<CapRec>& list);
void stats_capture_release(std::vector<CapRec>& list);

// ---------------------------------------------------------------------------
// Entry points between translation units
// ---------------------------------------------------------------------------
int green_setup(vie_handle* h);                 // green.cu
int green_setup_external(vie_handle* h, const double2* ext);  // green.cu, ext on the device
int green_split_bf16(vie_handle* h);            // zpass_bf16.cu: greenbf from green32t
int twiddle_setup(vie_handle* h);               // matvec.cu
int matvec_device(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, cudaStream_t s);
size_t matvec_workspace_bytes(const vie_handle* h, int nrhs, int precision);
// z-pass autotuner, outside capture (op: the N block, or VIE_OP_K for the K block)
int matvec_tune(vie_handle* h, int nrhs, int precision, cudaStream_t s, int op = VIE_OP_NSCAT);

// Support of a solve: per (z, y) row of the grid the voxel interval [x0, x1) whose
// unknowns are kept and the offset of voxel (x0, y, z) within a component block of ns
// voxels; a vector on the support is laid out [R][12][ns].  rows == NULL: the full
// grid in its natural layout (ns = nx ny nz).
struct Support {
    const int4* rows = nullptr;  // [nz * ny] (x0, x1, offset, 0)
    long long ns = 0;
};
// y = op(x) for vectors on a support.  tmp: scratch of 2 nrhs 12 nx ny nz complex values
// of the precision, used only when the matvec has to run on the full grid (scatter,
// full matvec, gather).
// shift (op PA only, optional): device [nrhs] values, y = op(x) - shift[r] x per right-hand side
// (the shifted operator of the solver's Arnoldi steps).
// conv (optional): full-grid [nrhs][12][nz][ny][nx] output of the convolution (N - G) x at
// every voxel, support or not (the operator's value before its voxel-wise terms).
// rmap, nact (optional, device memory): compute y only for the *nact right-hand sides listed in
// rmap, leaving the others' y untouched; the launches are sized for nrhs and skip the rest on the
// device, so no host round trip is needed (fused xy path; the other paths compute all of them).
int matvec_support(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, const Support& sp,
                   void* tmp, cudaStream_t s, const double2* shift = nullptr, void* conv = nullptr,
                   const int* rmap = nullptr, const int* nact = nullptr);
// full-grid vector <-> vector on a support (values outside the support dropped / set to zero)
int support_gather(const vie_handle* h, int nrhs, const void* full, void* part, int precision, const Support& sp,
                   cudaStream_t s);
int support_scatter(const vie_handle* h, int nrhs, const void* part, void* full, int precision, const Support& sp,
                    cudaStream_t s);
// full 3-D FFT of `batch` complex double volumes [batch][Lz][Ly][Lx] in place (forward, unscaled)
int fft3d_inplace64(vie_handle* h, double2* data, int batch, cudaStream_t s);
// jm: the full JM-VIE system (jmvie.cu; FP64 mode only), vectors [nrhs][2][12][nz][ny][nx]
int solve_device(vie_handle* h, int nrhs, const double2* b, double2* x, double tol, int restart, int maxit,
                 int mode, int flags, vie_solve_info* info, cudaStream_t s, bool jm = false);
int rhs_planewave_device(vie_handle* h, const double pol[3], const double dir[3], double2* e, double2* b,
                         cudaStream_t s);
int rhs_dipoles_device(vie_handle* h, int nrhs, const double* pos, const double* mom, double2* e, double2* b,
                       cudaStream_t s);
int materials_device(vie_handle* h, const double* eps_real, const double* sigma, cudaStream_t s);
// kmatvec.cu: the K octant spectra of a handle, built on first use
int k_octants(vie_handle* h, cudaStream_t s);
// jmvie.cu: the full JM-VIE (Eq. 14-15).  Vectors [R][2][12][nz][ny][nx] (j, then m' = m / eta0);
// the support form runs in FP64 (double2 vectors) or FP32 (float2), the full form in FP64.
int jm_materials(vie_handle* h, const double* mu_real, const double* mu_imag, cudaStream_t s);  // device maps or NULL
int jm_matvec_full(vie_handle* h, int R, const double2* x, double2* y, int op, cudaStream_t s,
                   const double2* shift = nullptr);
int jm_matvec_support(vie_handle* h, int R, const void* x, void* y, int op, const Support& sp, void* tmp,
                      cudaStream_t s, const double2* shift, int precision);
int jm_rhs_device(vie_handle* h, int R, const double2* einc, const double2* hinc, double2* b, cudaStream_t s);
int jm_fields_device(vie_handle* h, int R, const double2* x, const double2* einc, const double2* hinc, double2* eout,
                     double2* hout, double* p_abs, double* P_abs_host, cudaStream_t s);
// tucker.cu: Tucker compression of the handle's Green tensors (vie_green_tucker) and its reconstruction
int green_tucker(vie_handle* h, double tol, bool apply, int* ranks, double* err, size_t* bytes);
int tucker_reconstruct(vie_handle* h, double2* out, cudaStream_t s);
int fields_device(vie_handle* h, int nrhs, const double2* x, const double2* e_inc, double2* e_out, double* p_abs,
                  double* P_abs_host, cudaStream_t s);

// physical constants (SI)
constexpr double VIE_C0 = 299792458.0;
constexpr double VIE_EPS0 = 8.8541878128e-12;
constexpr double VIE_PI = 3.14159265358979323846;
