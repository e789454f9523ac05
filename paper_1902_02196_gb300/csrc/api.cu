// C ABI entry points (include/vie.h): argument checks, host-buffer staging, handle lifetime.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

// green.cu: the 30 Toeplitz tensors of the K operator into device memory
int green_k_toeplitz(vie_handle* h, double2* out, cudaStream_t s);
// kmatvec.cu: the release of a handle's K spectra
void kmatvec_release(vie_handle* h);
// rhs_post.cu: tested incident magnetic field of dipoles; magnetic field, b1+ and W_m from x
int rhs_dipoles_h_device(vie_handle* h, int R, const double* pos, const double* mom, double2* hinc, cudaStream_t s);
int hfields_device(vie_handle* h, int R, const double2* x, const double2* hinc, double2* hout, double2* b1p,
                   double* Wm_host, cudaStream_t s);

namespace {
thread_local std::string g_last_error;

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int next_pow2(int v) {
    int L = 2;
    while (L < v) L *= 2;
    return L;
}

cudaStream_t pick(vie_handle* h, void* s) { return s ? reinterpret_cast<cudaStream_t>(s) : h->stream; }

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// Two-phase staging: declare every buffer, reserve once, then bind.
struct Stager {
    vie_handle* h;
    cudaStream_t st;
    struct Item {
        const void* user;
        size_t bytes;
        bool is_out;
        bool host;
        size_t off;
    };
    std::vector<Item> items;
    bool any_host = false;
    int add(const void* p, size_t bytes, bool is_out) {
        Item it{p, bytes, is_out, p != nullptr && !is_device_ptr(p), 0};
        if (it.host) any_host = true;
        items.push_back(it);
        return (int)items.size() - 1;
    }
    int bind(std::vector<void*>& dev) {
        size_t off = 0;
        for (auto& it : items)
            if (it.host) {
                it.off = off;
                off += a256(it.bytes);
            }
        if (off) VIE_TRY(ws_reserve(h, h->stage_ws, off));
        dev.resize(items.size());
        for (size_t i = 0; i < items.size(); ++i) {
            auto& it = items[i];
            if (!it.user) {
                dev[i] = nullptr;
            } else if (it.host) {
                dev[i] = static_cast<char*>(h->stage_ws.ptr) + it.off;
                if (!it.is_out) VIE_CUDA(cudaMemcpyAsync(dev[i], it.user, it.bytes, cudaMemcpyHostToDevice, st));
            } else {
                dev[i] = const_cast<void*>(it.user);
            }
        }
        return VIE_OK;
    }
    int finish(const std::vector<void*>& dev) {
        for (size_t i = 0; i < items.size(); ++i) {
            auto& it = items[i];
            if (it.user && it.host && it.is_out)
                VIE_CUDA(cudaMemcpyAsync(const_cast<void*>(it.user), dev[i], it.bytes, cudaMemcpyDeviceToHost, st));
        }
        if (any_host) VIE_CUDA(cudaStreamSynchronize(st));
        return VIE_OK;
    }
};

void release(vie_handle* h) {
    if (!h) return;
    kmatvec_release(h);
    dev_free(h, h->eps64);
    dev_free(h, h->chi64);
    dev_free(h, h->tau64);
    dev_free(h, h->ieps64);
    dev_free(h, h->chi32);
    dev_free(h, h->tau32);
    dev_free(h, h->ieps32);
    if (!h->shared_green) {
        cudaFree(h->green64);
        cudaFree(h->green32);
        cudaFree(h->green32t);
        cudaFree(h->green64t);
        cudaFree(h->greenbf);
        cudaFree(h->colmap);
        cudaFree(h->colkx32);
        cudaFree(h->tw64);
        cudaFree(h->tw32);
        cudaFree(h->toeplitz);
    }
    cudaFree(h->tucker);
    dev_free(h, h->fft_ws.ptr);
    dev_free(h, h->stage_ws.ptr);
    dev_free(h, h->solve_ws.ptr);
    dev_free(h, h->support_ws.ptr);
    dev_free(h, h->post_ws.ptr);
    dev_free(h, h->fcache_ws.ptr);
    cudaFree(h->mu64);  // one allocation holds mu64, chim64, imu64 and jmsup64
    dev_free(h, h->jm_ws.ptr);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

#define REQUIRE(cond, msg)           \
    do {                             \
        if (!(cond)) {               \
            set_error(msg);          \
            return VIE_EINVAL;       \
        }                            \
    } while (0)

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

cudaError_t dev_malloc(const vie_handle* h, void** p, size_t bytes) {
    return h->async_alloc ? cudaMallocAsync(p, bytes, h->stream) : cudaMalloc(p, bytes);
}

void dev_free(const vie_handle* h, void* p) {
    if (!p) return;
    if (h->async_alloc)
        cudaFreeAsync(p, h->stream);
    else
        cudaFree(p);
}

namespace {
std::atomic<int> g_inject_oom{0};  // workspace allocations still to fail (vie_fault_inject)
}

int ws_reserve(vie_handle* h, Workspace& w, size_t bytes) {
    if (w.bytes >= bytes) return VIE_OK;
    for (int n = g_inject_oom.load(); n > 0;)
        if (g_inject_oom.compare_exchange_weak(n, n - 1)) {
            set_error("injected allocation failure (vie_fault_inject) of " + std::to_string(bytes) + " bytes");
            return VIE_ENOMEM;
        }
    if (w.ptr) {
        dev_free(h, w.ptr);
        h->bytes_held -= w.bytes;
        w.ptr = nullptr;
        w.bytes = 0;
    }
    if (dev_malloc(h, &w.ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        w.ptr = nullptr;
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
        return VIE_ENOMEM;
    }
    w.bytes = bytes;
    h->bytes_held += bytes;
    return VIE_OK;
}

extern "C" {

const char* vie_strerror(int code) {
    switch (code) {
        case VIE_OK: return "success";
        case VIE_EINVAL: return "invalid argument";
        case VIE_ENOMEM: return "out of memory";
        case VIE_EDEVICE: return "CUDA device error";
        case VIE_ETIMEOUT: return "timed out";
        case VIE_NOT_CONVERGED: return "solver did not reach the tolerance";
    }
    return "unknown error";
}

const char* vie_last_error(void) { return g_last_error.c_str(); }

int vie_fault_inject(int kind, int count) {
    REQUIRE(count >= 0, "count must be >= 0");
    switch (kind) {
        case VIE_INJECT_NONE: g_inject_oom = 0; return VIE_OK;
        case VIE_INJECT_OOM: g_inject_oom = count; return VIE_OK;
    }
    set_error("unknown fault kind");
    return VIE_EINVAL;
}

int vie_setup(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma, int flags,
              vie_handle** out) {
    g_last_error.clear();
    REQUIRE(out, "out is NULL");
    *out = nullptr;
    REQUIRE((flags & ~VIE_SETUP_PWC) == 0, "unknown flags");
    return handle_create(grid, freq_hz, eps_real, sigma, nullptr, out, nullptr, (flags & VIE_SETUP_PWC) ? 3 : 12);
}

int vie_setup_green_external(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma,
                             const void* toeplitz_fp64, vie_handle** out) {
    g_last_error.clear();
    REQUIRE(out, "out is NULL");
    *out = nullptr;
    REQUIRE(toeplitz_fp64, "toeplitz_fp64 is NULL");
    return handle_create(grid, freq_hz, eps_real, sigma, nullptr, out, toeplitz_fp64);
}

}  // extern "C"

size_t handle_green_bytes(const vie_handle* h) {
    const size_t ov = (size_t)h->O[0] * h->O[1] * h->O[2];
    return 60 * ov * (2 * sizeof(double2) + 2 * sizeof(float2) + sizeof(uint2)) + 60 * h->nv * sizeof(double2) +
           2048 * (sizeof(double2) + sizeof(float2)) + 2 * (size_t)h->L[0];
}

int handle_create(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma,
                  const vie_handle* share, vie_handle** out, const void* ext, int nc) {
    *out = nullptr;
    REQUIRE(grid && eps_real && sigma, "NULL argument");
    REQUIRE(grid->nx >= 1 && grid->ny >= 1 && grid->nz >= 1, "grid sizes must be >= 1");
    REQUIRE(grid->nx <= 512 && grid->ny <= 512 && grid->nz <= 512, "grid sizes above 512 are not supported");
    REQUIRE(std::isfinite(grid->dx) && std::isfinite(grid->dy) && std::isfinite(grid->dz) && grid->dx > 0 &&
                grid->dy > 0 && grid->dz > 0,
            "voxel sizes must be finite and positive");
    REQUIRE(std::isfinite(freq_hz) && freq_hz > 0, "frequency must be finite and positive");
    REQUIRE(!share || (share->nx == grid->nx && share->ny == grid->ny && share->nz == grid->nz &&
                       share->dx == grid->dx && share->dy == grid->dy && share->dz == grid->dz &&
                       share->freq == freq_hz),
            "template handle has another grid, voxel size or frequency");
    vie_handle* h = new (std::nothrow) vie_handle();
    if (!h) {
        set_error("host allocation failed");
        return VIE_ENOMEM;
    }
    std::memset(static_cast<void*>(h), 0, sizeof(vie_handle));
    h->nx = grid->nx, h->ny = grid->ny, h->nz = grid->nz;
    h->nc = nc == 3 ? 3 : 12;
    h->dx = grid->dx, h->dy = grid->dy, h->dz = grid->dz;
    h->freq = freq_hz;
    h->omega = 2.0 * VIE_PI * freq_hz;
    h->k0 = h->omega / VIE_C0;
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int i = 0; i < 3; ++i) {
        h->L[i] = next_pow2(2 * n[i] - 1);
        h->O[i] = h->L[i] / 2 + 1;
    }
    h->nv = (size_t)h->nx * h->ny * h->nz;
    int rc = VIE_OK;
    auto fail = [&](int code) {
        release(h);
        return code;
    };
    h->async_alloc = share != nullptr;  // a server request's handle
    if (cudaGetDevice(&h->device) != cudaSuccess || cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("no usable CUDA device");
        return fail(VIE_EDEVICE);
    }
    // validate the material maps on the host
    std::vector<double> er(h->nv), sg(h->nv);
    const bool dev_in = is_device_ptr(eps_real);
    if (dev_in) {
        if (cudaMemcpy(er.data(), eps_real, sizeof(double) * h->nv, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(sg.data(), sigma, sizeof(double) * h->nv, cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("cannot read material maps");
            return fail(VIE_EINVAL);
        }
    } else {
        std::memcpy(er.data(), eps_real, sizeof(double) * h->nv);
        std::memcpy(sg.data(), sigma, sizeof(double) * h->nv);
    }
    for (size_t m = 0; m < h->nv; ++m)
        if (!std::isfinite(er[m]) || !std::isfinite(sg[m]) || er[m] <= 0.0 || sg[m] < 0.0) {
            set_error("material map entry " + std::to_string(m) + " is not finite or out of range");
            return fail(VIE_EINVAL);
        }
    const size_t nv = h->nv;
    if (dev_malloc(h, (void**)&h->eps64, sizeof(double2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->chi64, sizeof(double2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->tau64, sizeof(double2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->ieps64, sizeof(double2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->chi32, sizeof(float2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->tau32, sizeof(float2) * nv) != cudaSuccess ||
        dev_malloc(h, (void**)&h->ieps32, sizeof(float2) * nv) != cudaSuccess) {
        cudaGetLastError();
        set_error("material allocation failed");
        return fail(VIE_ENOMEM);
    }
    h->bytes_held += nv * (4 * sizeof(double2) + 3 * sizeof(float2));
    double* dmat = nullptr;
    if (dev_malloc(h, (void**)&dmat, sizeof(double) * 2 * nv) != cudaSuccess) {
        cudaGetLastError();
        set_error("material staging failed");
        return fail(VIE_ENOMEM);
    }
    cudaMemcpyAsync(dmat, er.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dmat + nv, sg.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, h->stream);
    rc = materials_device(h, dmat, dmat + nv, h->stream);
    dev_free(h, dmat);
    cudaStreamSynchronize(h->stream);  // er and sg are read by the copies above
    if (rc < 0) return fail(rc);
    if (share) {
        h->shared_green = 1;
        h->green64 = share->green64;
        h->green32 = share->green32;
        h->green32t = share->green32t;
        h->green64t = share->green64t;
        h->greenbf = share->greenbf;
        h->colmap = share->colmap;
        h->colkx32 = share->colkx32;
        h->colpos32 = share->colpos32;
        h->tw64 = share->tw64;
        h->tw32 = share->tw32;
        h->toeplitz = share->toeplitz;
        *out = h;
        return VIE_OK;
    }
    if ((rc = twiddle_setup(h)) < 0) return fail(rc);
    if (ext) {
        const size_t ebytes = sizeof(double2) * 144 * (size_t)(2 * h->nx - 1) * (2 * h->ny - 1) * (2 * h->nz - 1);
        const void* dext = ext;
        void* tmp = nullptr;
        if (!is_device_ptr(ext)) {
            if (cudaMalloc(&tmp, ebytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("staging of the external Toeplitz table failed");
                return fail(VIE_ENOMEM);
            }
            if (cudaMemcpy(tmp, ext, ebytes, cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaFree(tmp);
                set_error("cannot read the external Toeplitz table");
                return fail(VIE_EINVAL);
            }
            dext = tmp;
        }
        rc = green_setup_external(h, static_cast<const double2*>(dext));
        cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
        if (rc < 0) return fail(rc);
    } else if ((rc = green_setup(h)) < 0) {
        return fail(rc);
    }
    *out = h;
    return VIE_OK;
}

extern "C" {

void vie_destroy(vie_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
}

int vie_info(vie_handle* h, int* fft_len_xyz, size_t* device_bytes) {
    REQUIRE(h, "NULL handle");
    if (fft_len_xyz)
        for (int i = 0; i < 3; ++i) fft_len_xyz[i] = h->L[i];
    if (device_bytes) *device_bytes = h->bytes_held;
    return VIE_OK;
}

int vie_matvec(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, void* stream) {
    g_last_error.clear();
    REQUIRE(h && x && y, "NULL argument");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    REQUIRE(precision == VIE_FP64 || precision == VIE_FP32 || precision == VIE_BF16X3, "unknown precision");
    REQUIRE(op == VIE_OP_A || op == VIE_OP_PA || op == VIE_OP_NSCAT || op == VIE_OP_K, "unknown operator");
    REQUIRE(op != VIE_OP_K || precision != VIE_BF16X3, "the K operator runs in FP64 or FP32");
    REQUIRE(op != VIE_OP_K || h->nc == 12, "the K operator is built for the PWL system only");
    REQUIRE(x != y, "x and y must not overlap");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * (precision == VIE_FP64 ? sizeof(double2) : sizeof(float2));
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(x, bytes, false);
    sg.add(y, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(matvec_device(h, nrhs, d[0], d[1], precision, op, st));
    return sg.finish(d);
}

int vie_rhs_planewave(vie_handle* h, const double pol[3], const double dir[3], void* e_inc, void* b, void* stream) {
    g_last_error.clear();
    REQUIRE(h && pol && dir, "NULL argument");
    for (int i = 0; i < 3; ++i) REQUIRE(std::isfinite(pol[i]) && std::isfinite(dir[i]), "non-finite source");
    const size_t bytes = (size_t)h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(e_inc, bytes, true);
    sg.add(b, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(rhs_planewave_device(h, pol, dir, (double2*)d[0], (double2*)d[1], st));
    return sg.finish(d);
}

int vie_rhs_dipoles(vie_handle* h, int nrhs, const double* pos, const double* mom, void* e_inc, void* b,
                    void* stream) {
    g_last_error.clear();
    REQUIRE(h && pos && mom, "NULL argument");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    for (int i = 0; i < 3 * nrhs; ++i) REQUIRE(std::isfinite(pos[i]) && std::isfinite(mom[i]), "non-finite source");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(e_inc, bytes, true);
    sg.add(b, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(rhs_dipoles_device(h, nrhs, pos, mom, (double2*)d[0], (double2*)d[1], st));
    return sg.finish(d);
}

int vie_solve(vie_handle* h, int nrhs, const void* b, void* x, double tol, int restart, int maxit, int mode,
              int flags, vie_solve_info* info, void* stream) {
    g_last_error.clear();
    REQUIRE(h && b && x, "NULL argument");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    REQUIRE(std::isfinite(tol) && tol > 0 && tol < 1, "tol must be in (0, 1)");
    REQUIRE(restart >= 1 && restart <= 128, "restart must be in [1, 128]");
    REQUIRE(maxit >= 1, "maxit must be >= 1");
    REQUIRE(mode == VIE_SOLVE_FP64 || mode == VIE_SOLVE_FP32_REFINE || mode == VIE_SOLVE_BF16X3_REFINE,
            "unknown mode");
    REQUIRE(mode != VIE_SOLVE_BF16X3_REFINE || h->nc == 12, "the BF16x3 mode is built for the PWL system only");
    REQUIRE((flags & ~15) == 0, "unknown flags");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(b, bytes, false);
    sg.add(x, bytes, (flags & 1) ? false : true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    sg.items[1].is_out = true;  // x is returned even when it carried the initial guess
    int rc = solve_device(h, nrhs, (const double2*)d[0], (double2*)d[1], tol, restart, maxit, mode, flags, info, st);
    if (rc < 0) return rc;
    VIE_TRY(sg.finish(d));
    VIE_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int vie_fields(vie_handle* h, int nrhs, const void* x, const void* e_inc, void* e_coeff, double* p_abs,
               double* P_abs, void* stream) {
    g_last_error.clear();
    REQUIRE(h && x && e_inc, "NULL argument");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(x, bytes, false);
    sg.add(e_inc, bytes, false);
    sg.add(e_coeff, bytes, true);
    sg.add(p_abs, (size_t)nrhs * h->nv * sizeof(double), true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(fields_device(h, nrhs, (const double2*)d[0], (const double2*)d[1], (double2*)d[2], (double*)d[3], P_abs,
                          st));
    return sg.finish(d);
}

int vie_green_toeplitz(vie_handle* h, void* out) {
    g_last_error.clear();
    REQUIRE(h && out, "NULL argument");
    const size_t bytes = 60 * h->nv * sizeof(double2);
    VIE_CUDA(cudaStreamSynchronize(h->stream));
    if (h->toeplitz) {
        VIE_CUDA(cudaMemcpy(out, h->toeplitz, bytes, cudaMemcpyDefault));
        return VIE_OK;
    }
    // the handle keeps the Tucker form only: reconstruct
    Stager sg{h, h->stream};
    sg.add(out, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(tucker_reconstruct(h, static_cast<double2*>(d[0]), h->stream));
    return sg.finish(d);
}

int vie_green_tucker(vie_handle* h, double tol, int flags, int* ranks, double* rel_err, size_t* compressed_bytes) {
    g_last_error.clear();
    REQUIRE(h, "NULL handle");
    REQUIRE(std::isfinite(tol) && tol >= 1e-7 && tol < 1, "tol must be in [1e-7, 1)");
    REQUIRE((flags & ~VIE_TUCKER_APPLY) == 0, "unknown flags");
    REQUIRE(!h->shared_green, "the handle shares another handle's Green tensors");
    VIE_CUDA(cudaStreamSynchronize(h->stream));
    return green_tucker(h, tol, (flags & VIE_TUCKER_APPLY) != 0, ranks, rel_err, compressed_bytes);
}

int vie_rhs_dipoles_h(vie_handle* h, int nrhs, const double* pos, const double* mom, void* h_inc, void* stream) {
    g_last_error.clear();
    REQUIRE(h && pos && mom && h_inc, "NULL argument");
    REQUIRE(h->nc == 12, "magnetic fields are built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    for (int i = 0; i < 3 * nrhs; ++i) REQUIRE(std::isfinite(pos[i]) && std::isfinite(mom[i]), "non-finite source");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(h_inc, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(rhs_dipoles_h_device(h, nrhs, pos, mom, static_cast<double2*>(d[0]), st));
    return sg.finish(d);
}

int vie_hfields(vie_handle* h, int nrhs, const void* x, const void* h_inc, void* h_coeff, void* b1_plus, double* W_m,
                void* stream) {
    g_last_error.clear();
    REQUIRE(h && x && h_inc, "NULL argument");
    REQUIRE(h->nc == 12, "magnetic fields are built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const size_t bytes = (size_t)nrhs * h->nc * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(x, bytes, false);
    sg.add(h_inc, bytes, false);
    sg.add(h_coeff, bytes, true);
    sg.add(b1_plus, (size_t)nrhs * h->nv * sizeof(double2), true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(hfields_device(h, nrhs, static_cast<const double2*>(d[0]), static_cast<const double2*>(d[1]),
                           static_cast<double2*>(d[2]), static_cast<double2*>(d[3]), W_m, st));
    return sg.finish(d);
}

int vie_set_permeability(vie_handle* h, const double* mu_real, const double* mu_imag) {
    g_last_error.clear();
    REQUIRE(h && mu_real && mu_imag, "NULL argument");
    REQUIRE(h->nc == 12, "the JM-VIE is built for the PWL system only");
    std::vector<double> mr(h->nv), mi(h->nv);
    const bool dev_in = is_device_ptr(mu_real);
    if (dev_in) {
        VIE_CUDA(cudaMemcpy(mr.data(), mu_real, sizeof(double) * h->nv, cudaMemcpyDeviceToHost));
        VIE_CUDA(cudaMemcpy(mi.data(), mu_imag, sizeof(double) * h->nv, cudaMemcpyDefault));
    } else {
        std::memcpy(mr.data(), mu_real, sizeof(double) * h->nv);
        std::memcpy(mi.data(), mu_imag, sizeof(double) * h->nv);
    }
    for (size_t m = 0; m < h->nv; ++m)
        REQUIRE(std::isfinite(mr[m]) && std::isfinite(mi[m]) && mr[m] > 0.0 && mi[m] >= 0.0,
                "permeability entry " + std::to_string(m) + " is not finite or out of range");
    double* d = nullptr;
    VIE_CUDA(cudaMalloc(&d, 2 * sizeof(double) * h->nv));
    int rc = VIE_OK;
    if (cudaMemcpy(d, mr.data(), sizeof(double) * h->nv, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + h->nv, mi.data(), sizeof(double) * h->nv, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot stage the permeability maps");
        rc = VIE_EDEVICE;
    }
    if (rc == VIE_OK) rc = jm_materials(h, d, d + h->nv, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    return rc;
}

int vie_jm_matvec(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, void* stream) {
    g_last_error.clear();
    REQUIRE(h && x && y, "NULL argument");
    REQUIRE(h->nc == 12, "the JM-VIE is built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    REQUIRE(precision == VIE_FP64 || precision == VIE_FP32, "precision must be VIE_FP64 or VIE_FP32");
    REQUIRE(op == VIE_OP_A || op == VIE_OP_PA, "unknown operator (VIE_OP_A or VIE_OP_PA)");
    REQUIRE(x != y, "x and y must not overlap");
    const size_t bytes = (size_t)nrhs * 24 * h->nv * (precision == VIE_FP64 ? sizeof(double2) : sizeof(float2));
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(x, bytes, false);
    sg.add(y, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(jm_matvec_support(h, nrhs, d[0], d[1], op, Support{}, nullptr, st, nullptr, precision));
    return sg.finish(d);
}

int vie_jm_rhs(vie_handle* h, int nrhs, const void* e_inc, const void* h_inc, void* b, void* stream) {
    g_last_error.clear();
    REQUIRE(h && e_inc && h_inc && b, "NULL argument");
    REQUIRE(h->nc == 12, "the JM-VIE is built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const size_t half = (size_t)nrhs * 12 * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(e_inc, half, false);
    sg.add(h_inc, half, false);
    sg.add(b, 2 * half, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(jm_rhs_device(h, nrhs, static_cast<const double2*>(d[0]), static_cast<const double2*>(d[1]),
                          static_cast<double2*>(d[2]), st));
    return sg.finish(d);
}

int vie_jm_solve(vie_handle* h, int nrhs, const void* b, void* x, double tol, int restart, int maxit, int mode,
                 int flags, vie_solve_info* info, void* stream) {
    g_last_error.clear();
    REQUIRE(h && b && x, "NULL argument");
    REQUIRE(h->nc == 12, "the JM-VIE is built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    REQUIRE(std::isfinite(tol) && tol > 0 && tol < 1, "tol must be in (0, 1)");
    REQUIRE(restart >= 1 && restart <= 128, "restart must be in [1, 128]");
    REQUIRE(maxit >= 1, "maxit must be >= 1");
    REQUIRE(mode == VIE_SOLVE_FP64 || mode == VIE_SOLVE_FP32_REFINE, "mode must be VIE_SOLVE_FP64 or VIE_SOLVE_FP32_REFINE");
    REQUIRE((flags & ~11) == 0, "unknown flags");
    const size_t bytes = (size_t)nrhs * 24 * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(b, bytes, false);
    sg.add(x, bytes, (flags & 1) ? false : true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    sg.items[1].is_out = true;
    int rc = solve_device(h, nrhs, (const double2*)d[0], (double2*)d[1], tol, restart, maxit, mode, flags | 4, info,
                          st, true);
    if (rc < 0) return rc;
    VIE_TRY(sg.finish(d));
    VIE_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int vie_jm_fields(vie_handle* h, int nrhs, const void* x, const void* e_inc, const void* h_inc, void* e_coeff,
                  void* h_coeff, double* p_abs, double* P_abs, void* stream) {
    g_last_error.clear();
    REQUIRE(h && x && e_inc && h_inc, "NULL argument");
    REQUIRE(h->nc == 12, "the JM-VIE is built for the PWL system only");
    REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const size_t half = (size_t)nrhs * 12 * h->nv * sizeof(double2);
    cudaStream_t st = pick(h, stream);
    Stager sg{h, st};
    sg.add(x, 2 * half, false);
    sg.add(e_inc, half, false);
    sg.add(h_inc, half, false);
    sg.add(e_coeff, half, true);
    sg.add(h_coeff, half, true);
    sg.add(p_abs, (size_t)nrhs * h->nv * sizeof(double), true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(jm_fields_device(h, nrhs, static_cast<const double2*>(d[0]), static_cast<const double2*>(d[1]),
                             static_cast<const double2*>(d[2]), static_cast<double2*>(d[3]),
                             static_cast<double2*>(d[4]), static_cast<double*>(d[5]), P_abs, st));
    return sg.finish(d);
}

int vie_green_toeplitz_k(vie_handle* h, void* out) {
    g_last_error.clear();
    REQUIRE(h && out, "NULL argument");
    const size_t bytes = 30 * h->nv * sizeof(double2);
    Stager sg{h, h->stream};
    sg.add(out, bytes, true);
    std::vector<void*> d;
    VIE_TRY(sg.bind(d));
    VIE_TRY(green_k_toeplitz(h, static_cast<double2*>(d[0]), h->stream));
    return sg.finish(d);
}

}  // extern "C"
