// Launch counting and optional per-kernel device timing with CUDA events.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {
struct Entry {
    long long launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};
struct Pending {
    std::string name;
    cudaEvent_t start, stop;
};
std::mutex g_mu;
std::map<std::string, Entry> g_entries;
std::vector<Pending> g_pending;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pool;
bool g_timing = false;
long long g_total = 0;
thread_local std::vector<CapRec>* t_cap = nullptr;  // graph capture in progress on this thread

// device byte counters, one per registered kernel name
constexpr int kDevSlots = 16;  // names; two counters each (bytes, launches with work)
constexpr int kMaxDev = 64;
const char* g_dev_names[kDevSlots];
int g_ndev = 0;
unsigned long long* g_dev_addr[kMaxDev];

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess)
            g_entries[p.name].ms += ms;
        else
            cudaGetLastError();
        g_pool.emplace_back(p.start, p.stop);
    }
    g_pending.clear();
}
}  // namespace

__device__ unsigned long long g_dev_bytes[2 * kDevSlots];

unsigned long long* dev_bytes_ptr(const char* name) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    int slot = -1;
    for (int i = 0; i < g_ndev; ++i)
        if (std::strcmp(g_dev_names[i], name) == 0) slot = i;
    if (slot < 0) {
        if (g_ndev >= kDevSlots) return nullptr;
        slot = g_ndev++;
        g_dev_names[slot] = name;  // names are string literals
    }
    if (!g_dev_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dev_bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_dev_addr[dev] = static_cast<unsigned long long*>(p);
    }
    return g_dev_addr[dev] + 2 * slot;
}

namespace {
// adds the device counters into the entries and clears them (current device)
void fold_dev_bytes_locked(bool add) {
    if (g_ndev == 0) return;
    unsigned long long v[2 * kDevSlots] = {};
    if (cudaMemcpyFromSymbol(v, g_dev_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (add)
        for (int i = 0; i < g_ndev; ++i)
            if (v[2 * i + 1]) {
                Entry& e = g_entries[g_dev_names[i]];
                e.bytes += (double)v[2 * i];
                e.launches += (long long)v[2 * i + 1];
            }
    const unsigned long long z[2 * kDevSlots] = {};
    if (cudaMemcpyToSymbol(g_dev_bytes, z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}
}  // namespace

void stats_capture_begin(std::vector<CapRec>* list) { t_cap = list; }
void stats_capture_end() { t_cap = nullptr; }

void stats_graph_replayed(const std::vector<CapRec>& list) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& r : list) {
        ++g_total;  // every launch issued
        if (r.bytes < 0) continue;  // counted on the device when it has work
        Entry& e = g_entries[r.name];
        ++e.launches;
        e.bytes += r.bytes;
    }
}

void stats_graph_harvest(const std::vector<CapRec>& list) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& r : list) {
        if (!r.ev0) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev0, r.ev1) == cudaSuccess)
            g_entries[r.name].ms += ms;
        else
            cudaGetLastError();
    }
}

void stats_capture_release(std::vector<CapRec>& list) {
    for (auto& r : list) {
        if (r.ev0) cudaEventDestroy(r.ev0);
        if (r.ev1) cudaEventDestroy(r.ev1);
    }
    list.clear();
}

LaunchScope::LaunchScope(const char* n, cudaStream_t s, double alg_bytes)
    : name(n), stream(s), timed(false), ev0(nullptr), ev1(nullptr) {
    if (t_cap) {  // captured into a graph: counted per replay; event-record nodes when timing
        CapRec r{name, alg_bytes, nullptr, nullptr};  // alg_bytes < 0: counted on the device
        bool timing;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            timing = g_timing;
        }
        if (timing && cudaEventCreate(&r.ev0) == cudaSuccess && cudaEventCreate(&r.ev1) == cudaSuccess &&
            cudaEventRecordWithFlags(r.ev0, stream, cudaEventRecordExternal) == cudaSuccess) {
            ev0 = r.ev0;
            ev1 = r.ev1;
        } else {
            cudaGetLastError();
            if (r.ev0) cudaEventDestroy(r.ev0);
            if (r.ev1) cudaEventDestroy(r.ev1);
            r.ev0 = r.ev1 = nullptr;
        }
        t_cap->push_back(r);
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    Entry& e = g_entries[name];
    ++g_total;  // every launch issued
    if (alg_bytes >= 0) {  // else counted on the device when it has work
        ++e.launches;
        e.bytes += alg_bytes;
    }
    if (!g_timing) return;
    if (!g_pool.empty()) {
        ev0 = g_pool.back().first;
        ev1 = g_pool.back().second;
        g_pool.pop_back();
    } else if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(ev0, stream);
    timed = true;
}

LaunchScope::~LaunchScope() {
    if (ev0 && !timed) {  // captured launch: the closing event-record node
        if (cudaEventRecordWithFlags(ev1, stream, cudaEventRecordExternal) != cudaSuccess) cudaGetLastError();
        return;
    }
    if (!timed) return;
    cudaEventRecord(ev1, stream);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(Pending{name, ev0, ev1});
    if (g_pending.size() > 200000) drain_locked();
}

extern "C" {

int vie_stats_reset(int enable_timing) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    double dummy[3];
    solve_device_bytes(dummy, true);
    fold_dev_bytes_locked(false);
    g_entries.clear();
    g_total = 0;
    g_timing = enable_timing != 0;
    return VIE_OK;
}

int vie_stats_read(int max_entries, char* names, long long* launches, double* ms, double* bytes, int* n_entries,
                   long long* total_launches) {
    // the device-side counters are complete once the counted work has finished
    if (cudaDeviceSynchronize() != cudaSuccess) cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    double dev[3] = {0, 0, 0};
    if (solve_device_bytes(dev, true) == VIE_OK) {
        const char* nm[3] = {"gs_dots", "gs_update", "solution_update"};
        for (int i = 0; i < 3; ++i)
            if (g_entries.count(nm[i])) g_entries[nm[i]].bytes += dev[i];
    }
    fold_dev_bytes_locked(true);
    int i = 0;
    for (auto& kv : g_entries) {
        if (i >= max_entries) break;
        if (names) {
            std::strncpy(names + 48 * i, kv.first.c_str(), 47);
            names[48 * i + 47] = 0;
        }
        if (launches) launches[i] = kv.second.launches;
        if (ms) ms[i] = kv.second.ms;
        if (bytes) bytes[i] = kv.second.bytes;
        ++i;
    }
    if (n_entries) *n_entries = i;
    if (total_launches) *total_launches = g_total;
    return VIE_OK;
}

}  // extern "C"
