// Request loop with continuous batching (vie_server_*, vie_submit, vie_poll).
//
// A request is one dielectric solve: a grid, voxel size, frequency and material map,
// nrhs dipole right-hand sides (Eq. 13 with a point current, tested as in
// vie_rhs_dipoles), GMRES to a tolerance (Section IV-B, Section V), then the fields and
// absorbed power (Section IV-C, Eq. 44).  The server runs up to max_concurrent requests
// at once, one host thread and one CUDA stream each, so their kernels overlap on the
// device; a finished request frees its slot and its memory and the next admissible
// request starts at once (continuous batching rather than a queue of fixed batches).
// Admission follows serve_policy.h: the device-memory budget covers every running
// request's working set and the cached Green tensors.  The Green tensors depend only on
// (grid, voxel size, frequency), so each key is built once, kept on the device and
// shared by every request with that key; idle entries are evicted least recently used.
// Every request computes exactly what vie_setup + vie_rhs_dipoles + vie_solve +
// vie_fields compute on its own, on its own stream, so its result does not depend on
// what else runs.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "serve_policy.h"

namespace {

using Clock = std::chrono::steady_clock;

struct GreenKey {
    int nx, ny, nz;
    double dx, dy, dz, freq;
    bool operator<(const GreenKey& o) const {
        return std::tie(nx, ny, nz, dx, dy, dz, freq) < std::tie(o.nx, o.ny, o.nz, o.dx, o.dy, o.dz, o.freq);
    }
};

struct CacheEntry {
    vie_handle* tmpl = nullptr;  // owns the Green tensors
    int users = 0;
    bool building = true;
    bool failed = false;
    unsigned long long last = 0;
    size_t bytes = 0;
};

struct Req {
    unsigned long long id = 0;
    vie_grid grid{};
    double freq = 0, tol = 0;
    int nrhs = 0, restart = 0, maxit = 0, mode = 0;
    std::vector<double> eps, sig, pos, mom;
    void* x_out = nullptr;
    double* p_abs_out = nullptr;
    double* P_abs_out = nullptr;
    size_t work = 0, green = 0;
    int bypassed = 0;
    Clock::time_point t_submit, t_start, t_end;
    float dev_ms[2] = {-1.f, -1.f};  // device span after the server's reference event
    bool done = false;
    vie_result res{};
};

int next_pow2(int v) {
    int L = 2;
    while (L < v) L *= 2;
    return L;
}

// device bytes of one request's working set (material maps, b, e_inc, x, p_abs, solver and
// FFT workspaces), an upper bound: the solver's vectors are sized for the full grid
size_t work_bytes(const vie_grid& g, int R, int restart, int mode) {
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    const size_t n = (size_t)R * 12 * nv;
    const size_t Lx = next_pow2(2 * g.nx - 1), Ly = next_pow2(2 * g.ny - 1);
    const size_t basis = (mode == VIE_SOLVE_FP64 ? 16 : 8) * (size_t)(restart + 1) * n;
    // b, e_inc, x; solver r, bt, t, x; scratch (the solve keeps no point for vie_fields: flags 4)
    const size_t vecs = 16 * n * (3 + 4 + 2) + 8 * (size_t)R * nv;
    const size_t fft = 16 * (size_t)R * 12 * g.nz * (g.ny * Lx + Ly * Lx);
    const size_t mats = nv * (4 * 16 + 3 * 8);
    return basis + vecs + fft + mats + ((size_t)64 << 20);
}

// device bytes of a cache entry: Green tensors (FP64, FP32 and both transposed), Toeplitz
// tensors, twiddles, column map, and the template handle's own material maps
size_t green_bytes(const vie_grid& g) {
    size_t O = 1;
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int i = 0; i < 3; ++i) O *= (size_t)next_pow2(2 * n[i] - 1) / 2 + 1;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    return 60 * O * (16 + 16 + 8 + 8) + 60 * nv * 16 + 2048 * 24 + 8 * 4096 + nv * (4 * 16 + 3 * 8) +
           ((size_t)16 << 20);
}

}  // namespace

struct vie_server {
    int device = 0;
    size_t budget = 0;
    int slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> queue;
    std::map<unsigned long long, std::shared_ptr<Req>> tickets;
    std::map<GreenKey, CacheEntry> cache;
    size_t in_use = 0;
    unsigned long long next_id = 1, clock = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    Clock::time_point t0;          // creation: origin of the host spans
    cudaEvent_t ref = nullptr;     // recorded at creation: origin of the device spans
    cudaMemPool_t pool = nullptr;  // the device's default memory pool, which requests allocate from
    uint64_t pool_keep0 = 0;       // its release threshold before this server set it
};

namespace {

constexpr int kMaxBypass = 4;

GreenKey key_of(const Req& r) {
    return GreenKey{r.grid.nx, r.grid.ny, r.grid.nz, r.grid.dx, r.grid.dy, r.grid.dz, r.freq};
}

// Under the lock: pick the next request by serve::admit, reserve its memory, register it
// with its cache entry (creating the entry, to be built by this worker, when missing).
bool admit_locked(vie_server* s, std::shared_ptr<Req>& out, bool& builder) {
    if (s->queue.empty()) return false;
    std::vector<GreenKey> keys;
    std::vector<serve::CacheView> cv;
    std::map<GreenKey, int> index;
    for (auto& kv : s->cache) {
        index[kv.first] = (int)keys.size();
        keys.push_back(kv.first);
        cv.push_back(serve::CacheView{kv.second.bytes, kv.second.users, kv.second.last});
    }
    std::vector<serve::QueuedView> qv;
    for (auto& r : s->queue) {
        auto it = index.find(key_of(*r));
        qv.push_back(serve::QueuedView{r->work, r->green, it == index.end() ? -1 : it->second, r->bypassed});
    }
    const size_t free_bytes = s->budget > s->in_use ? s->budget - s->in_use : 0;
    const serve::Decision d = serve::admit(qv, cv, free_bytes, kMaxBypass);
    if (d.pick < 0) return false;
    for (int c : d.evict) {
        auto it = s->cache.find(keys[c]);
        if (it->second.tmpl) vie_destroy(it->second.tmpl);
        s->in_use -= it->second.bytes;
        s->cache.erase(it);
    }
    if (d.pick > 0) s->queue.front()->bypassed++;
    out = s->queue[d.pick];
    s->queue.erase(s->queue.begin() + d.pick);
    s->in_use += out->work;
    const GreenKey k = key_of(*out);
    auto it = s->cache.find(k);
    builder = it == s->cache.end();
    if (builder) {
        CacheEntry e;
        e.bytes = out->green;
        s->in_use += e.bytes;
        it = s->cache.emplace(k, e).first;
    }
    it->second.users++;
    it->second.last = ++s->clock;
    out->res.green_cached = builder ? 0 : 1;
    return true;
}

#define SRV_TRY(expr)         \
    do {                      \
        const int rc_ = (expr); \
        if (rc_ < 0) return rc_; \
    } while (0)

// one request on the calling thread (device already selected)
int run_request(vie_server* s, Req& r, bool builder, vie_solve_info* info) {
    const GreenKey k = key_of(r);
    vie_handle* tmpl = nullptr;
    if (builder) {
        vie_handle* t = nullptr;
        const int rc = handle_create(&r.grid, r.freq, r.eps.data(), r.sig.data(), nullptr, &t);
        std::lock_guard<std::mutex> lk(s->mu);
        CacheEntry& e = s->cache[k];
        e.building = false;
        e.failed = rc < 0;
        e.tmpl = t;
        s->cv.notify_all();
        if (rc < 0) return rc;
        tmpl = t;
    } else {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return !s->cache[k].building; });
        if (s->cache[k].failed) {
            set_error("Green tensor setup of this (grid, voxel, frequency) failed");
            return VIE_EDEVICE;
        }
        tmpl = s->cache[k].tmpl;
    }
    vie_handle* h = nullptr;
    SRV_TRY(handle_create(&r.grid, r.freq, r.eps.data(), r.sig.data(), tmpl, &h));
    // the request's buffers come from the device's memory pool in the order of its stream (the
    // handle allocates with cudaMallocAsync), so neither they nor the handle's workspaces
    // synchronise the device when they are allocated or freed
    struct Guard {
        vie_handle* h;
        std::vector<void*> bufs;
        ~Guard() {
            if (h) cudaStreamSynchronize(h->stream);
            for (void* p : bufs) dev_free(h, p);
            vie_destroy(h);
        }
    } g{h, {}};
    const size_t n = (size_t)r.nrhs * 12 * h->nv;
    void *b = nullptr, *e = nullptr, *x = nullptr, *pa = nullptr;
    if (dev_malloc(h, &b, 16 * n) != cudaSuccess || (g.bufs.push_back(b), dev_malloc(h, &e, 16 * n)) != cudaSuccess ||
        (g.bufs.push_back(e), dev_malloc(h, &x, 16 * n)) != cudaSuccess ||
        (g.bufs.push_back(x), dev_malloc(h, &pa, 8 * (size_t)r.nrhs * h->nv)) != cudaSuccess) {
        cudaGetLastError();
        set_error("request buffers: device allocation failed");
        return VIE_ENOMEM;
    }
    g.bufs.push_back(pa);
    void* st = h->stream;
    // device span of the request's work on its stream
    struct Span {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Span() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } sp;
    if (s->ref && (cudaEventCreate(&sp.e0) != cudaSuccess || cudaEventCreate(&sp.e1) != cudaSuccess ||
                   cudaEventRecord(sp.e0, h->stream) != cudaSuccess)) {
        cudaGetLastError();
        if (sp.e0) cudaEventDestroy(sp.e0);
        if (sp.e1) cudaEventDestroy(sp.e1);
        sp.e0 = sp.e1 = nullptr;
    }
    SRV_TRY(vie_rhs_dipoles(h, r.nrhs, r.pos.data(), r.mom.data(), e, b, st));
    // flags 4: the request's vie_fields takes no field map, so the solve keeps no point for it
    const int rc = vie_solve(h, r.nrhs, b, x, r.tol, r.restart, r.maxit, r.mode, 4, info, st);
    if (rc < 0) return rc;
    std::vector<double> P(r.nrhs);
    SRV_TRY(vie_fields(h, r.nrhs, x, e, nullptr, (double*)pa, P.data(), st));
    if (r.x_out) VIE_CUDA(cudaMemcpyAsync(r.x_out, x, 16 * n, cudaMemcpyDeviceToHost, h->stream));
    if (r.p_abs_out)
        VIE_CUDA(cudaMemcpyAsync(r.p_abs_out, pa, 8 * (size_t)r.nrhs * h->nv, cudaMemcpyDeviceToHost, h->stream));
    if (sp.e1 && cudaEventRecord(sp.e1, h->stream) != cudaSuccess) cudaGetLastError();
    VIE_CUDA(cudaStreamSynchronize(h->stream));
    if (sp.e1 && (cudaEventElapsedTime(&r.dev_ms[0], s->ref, sp.e0) != cudaSuccess ||
                  cudaEventElapsedTime(&r.dev_ms[1], s->ref, sp.e1) != cudaSuccess)) {
        cudaGetLastError();
        r.dev_ms[0] = r.dev_ms[1] = -1.f;
    }
    if (r.P_abs_out) std::memcpy(r.P_abs_out, P.data(), sizeof(double) * r.nrhs);
    return rc;  // VIE_OK or VIE_NOT_CONVERGED
}

void worker(vie_server* s) {
    if (cudaSetDevice(s->device) != cudaSuccess) cudaGetLastError();
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        std::shared_ptr<Req> r;
        bool builder = false;
        s->cv.wait(lk, [&] { return s->stop || admit_locked(s, r, builder); });
        if (!r) return;  // stop
        lk.unlock();
        r->t_start = Clock::now();
        std::vector<vie_solve_info> info(r->nrhs);
        const int rc = run_request(s, *r, builder, info.data());
        r->t_end = Clock::now();
        lk.lock();
        r->res.status = rc;
        r->res.nrhs = r->nrhs;
        r->res.iterations = 0;
        r->res.resid = 0.0;
        for (auto& i : info) {
            r->res.iterations = i.iterations > r->res.iterations ? i.iterations : r->res.iterations;
            r->res.resid = i.resid > r->res.resid ? i.resid : r->res.resid;
        }
        r->res.queued_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
        r->res.run_s = std::chrono::duration<double>(r->t_end - r->t_start).count();
        r->res.start_s = std::chrono::duration<double>(r->t_start - s->t0).count();
        r->res.end_s = std::chrono::duration<double>(r->t_end - s->t0).count();
        r->res.dev_start_s = r->dev_ms[0] >= 0.f ? 1e-3 * r->dev_ms[0] : -1.0;
        r->res.dev_end_s = r->dev_ms[1] >= 0.f ? 1e-3 * r->dev_ms[1] : -1.0;
        r->done = true;
        s->in_use -= r->work;
        auto it = s->cache.find(key_of(*r));
        if (it != s->cache.end()) {
            it->second.users--;
            it->second.last = ++s->clock;
            if (it->second.failed && it->second.users == 0) {
                s->in_use -= it->second.bytes;
                s->cache.erase(it);
            }
        }
        s->cv.notify_all();
    }
}

}  // namespace

int vie_server_create(size_t hbm_budget_bytes, int max_concurrent, vie_server** out) {
    if (!out) {
        set_error("out is NULL");
        return VIE_EINVAL;
    }
    *out = nullptr;
    if (max_concurrent < 1 || max_concurrent > 64) {
        set_error("max_concurrent must be in [1, 64]");
        return VIE_EINVAL;
    }
    int dev = 0;
    VIE_CUDA(cudaGetDevice(&dev));
    size_t free_b = 0, total_b = 0;
    VIE_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (hbm_budget_bytes == 0) hbm_budget_bytes = free_b / 100 * 85;
    if (hbm_budget_bytes > free_b) {
        set_error("budget above the free device memory");
        return VIE_EINVAL;
    }
    vie_server* s = new (std::nothrow) vie_server();
    if (!s) {
        set_error("host allocation failed");
        return VIE_ENOMEM;
    }
    s->device = dev;
    s->budget = hbm_budget_bytes;
    // requests allocate from the device's default memory pool in stream order; keep up to the
    // budget in the pool between requests instead of returning it at every synchronisation
    // (a setting of this process's pool, not of the device; vie_server_destroy restores it and
    // returns what the pool holds)
    {
        uint64_t keep = hbm_budget_bytes;
        if (cudaDeviceGetDefaultMemPool(&s->pool, dev) != cudaSuccess ||
            cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &s->pool_keep0) != cudaSuccess ||
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            s->pool = nullptr;
        }
    }
    s->slots = max_concurrent;
    s->t0 = Clock::now();
    // the origin of the device spans: an event that has completed before any request starts
    if (cudaEventCreate(&s->ref) != cudaSuccess || cudaEventRecord(s->ref, cudaStreamPerThread) != cudaSuccess ||
        cudaEventSynchronize(s->ref) != cudaSuccess) {
        cudaGetLastError();
        if (s->ref) cudaEventDestroy(s->ref);
        s->ref = nullptr;
    }
    for (int i = 0; i < max_concurrent; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return VIE_OK;
}

void vie_server_destroy(vie_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
        s->cv.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->cache)
        if (kv.second.tmpl) vie_destroy(kv.second.tmpl);
    if (s->ref) cudaEventDestroy(s->ref);
    if (s->pool) {  // every request's frees have completed (their handles synchronised their streams)
        if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &s->pool_keep0) != cudaSuccess ||
            cudaMemPoolTrimTo(s->pool, 0) != cudaSuccess)
            cudaGetLastError();
    }
    delete s;
}

int vie_submit(vie_server* s, const vie_request* q, unsigned long long* ticket) {
    if (!s || !q || !ticket) {
        set_error("NULL argument");
        return VIE_EINVAL;
    }
    const vie_grid& g = q->grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > 512 || g.ny > 512 || g.nz > 512 || !(g.dx > 0) || !(g.dy > 0) ||
        !(g.dz > 0) || !(q->freq_hz > 0) || !q->eps_real || !q->sigma || q->nrhs < 1 || !q->dip_pos ||
        !q->dip_mom || !(q->tol > 0) || q->restart < 1 || q->restart > 128 || q->maxit < 1 ||
        (q->mode != VIE_SOLVE_FP64 && q->mode != VIE_SOLVE_FP32_REFINE)) {
        set_error("invalid request (grid, frequency, materials, right-hand sides or solver settings)");
        return VIE_EINVAL;
    }
    auto r = std::make_shared<Req>();
    r->grid = g;
    r->freq = q->freq_hz;
    r->tol = q->tol;
    r->nrhs = q->nrhs;
    r->restart = q->restart;
    r->maxit = q->maxit;
    r->mode = q->mode;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    r->eps.assign(q->eps_real, q->eps_real + nv);
    r->sig.assign(q->sigma, q->sigma + nv);
    r->pos.assign(q->dip_pos, q->dip_pos + 3 * (size_t)q->nrhs);
    r->mom.assign(q->dip_mom, q->dip_mom + 3 * (size_t)q->nrhs);
    r->x_out = q->x_out;
    r->p_abs_out = q->p_abs_out;
    r->P_abs_out = q->P_abs_out;
    r->work = work_bytes(g, q->nrhs, q->restart, q->mode);
    r->green = green_bytes(g);
    if (r->work + r->green > s->budget) {
        set_error("request needs " + std::to_string(r->work + r->green) + " device bytes, above the server budget");
        return VIE_ENOMEM;
    }
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->tickets[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
    s->cv.notify_all();
    return VIE_OK;
}

int vie_poll(vie_server* s, unsigned long long ticket, int timeout_us, vie_result* out) {
    if (!s || !out || timeout_us < 0) {
        set_error("NULL argument or negative timeout");
        return VIE_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket (never issued or already collected)");
        return VIE_EINVAL;
    }
    std::shared_ptr<Req> r = it->second;
    if (!s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) return VIE_ETIMEOUT;
    *out = r->res;
    s->tickets.erase(ticket);
    return VIE_OK;
}

int vie_server_stats(vie_server* s, int* queued, int* running, size_t* bytes_in_use, int* cache_entries) {
    if (!s) {
        set_error("NULL server");
        return VIE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    int run = 0;
    for (auto& kv : s->cache) run += kv.second.users;
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = run;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    if (cache_entries) *cache_entries = (int)s->cache.size();
    return VIE_OK;
}
