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

LaunchScope::LaunchScope(const char* n, cudaStream_t s, double alg_bytes)
    : name(n), stream(s), timed(false), ev0(nullptr), ev1(nullptr) {
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_total;
    Entry& e = g_entries[name];
    ++e.launches;
    e.bytes += alg_bytes;
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
    g_entries.clear();
    g_total = 0;
    g_timing = enable_timing != 0;
    return VIE_OK;
}

int vie_stats_read(int max_entries, char* names, long long* launches, double* ms, double* bytes, int* n_entries,
                   long long* total_launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    double dev[3] = {0, 0, 0};
    if (solve_device_bytes(dev, true) == VIE_OK) {
        const char* nm[3] = {"gs_dots", "gs_update", "solution_update"};
        for (int i = 0; i < 3; ++i)
            if (g_entries.count(nm[i])) g_entries[nm[i]].bytes += dev[i];
    }
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
