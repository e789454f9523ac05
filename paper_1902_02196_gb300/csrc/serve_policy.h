// Admission and Green-cache eviction policy of the request loop (server.cu).  Plain C++,
// no CUDA: the CPU tests compile this header on its own.
//
// Device memory is accounted in two parts: each admitted request's own working set
// (material maps, right-hand sides, solution, solver and FFT workspaces) and the Green
// tensors of every cache entry, shared by all requests of one (grid, voxel, frequency).
// A request is admitted when its working set, plus its Green tensors if they are not
// cached yet, fits in the free budget, after evicting least-recently-used cache entries
// that no running request holds.  The queue is served in order, except that a request
// behind a head that does not fit may go first; a head can be passed at most max_bypass
// times, after which the loop waits for memory to free up.
#pragma once

#include <cstddef>
#include <vector>

namespace serve {

struct QueuedView {
    size_t work;       // bytes of the request's own working set
    size_t green;      // bytes of its Green tensors when not cached
    int cache_entry;   // index of its key's entry in the cache view, -1 if none
    int bypassed;      // times another request was admitted ahead of it while it was the head
};

struct CacheView {
    size_t bytes;
    int users;                // running requests holding the entry
    unsigned long long last;  // last use (larger = more recent)
};

struct Decision {
    int pick = -1;             // queue index to admit, -1 = none
    std::vector<int> evict;    // cache indices to evict first (LRU order)
};

// free_bytes = budget - in_use (in_use counts admitted working sets and all cache entries)
inline Decision admit(const std::vector<QueuedView>& q, const std::vector<CacheView>& cache, size_t free_bytes,
                      int max_bypass) {
    Decision d;
    for (size_t i = 0; i < q.size(); ++i) {
        const QueuedView& r = q[i];
        const size_t need = r.work + (r.cache_entry >= 0 ? 0 : r.green);
        std::vector<int> ev;
        size_t avail = free_bytes;
        if (need > avail) {
            // evict idle entries, least recently used first, other than the request's own
            std::vector<int> idle;
            for (size_t c = 0; c < cache.size(); ++c)
                if (cache[c].users == 0 && (int)c != r.cache_entry) idle.push_back((int)c);
            for (size_t a = 0; a < idle.size(); ++a)
                for (size_t b = a + 1; b < idle.size(); ++b)
                    if (cache[idle[b]].last < cache[idle[a]].last) {
                        const int t = idle[a];
                        idle[a] = idle[b];
                        idle[b] = t;
                    }
            for (int c : idle) {
                if (avail >= need) break;
                avail += cache[c].bytes;
                ev.push_back(c);
            }
        }
        if (need <= avail) {
            d.pick = (int)i;
            d.evict = ev;
            return d;
        }
        if (i == 0 && r.bypassed >= max_bypass) return d;  // the head waits for memory; nobody passes it
    }
    return d;
}

}  // namespace serve
