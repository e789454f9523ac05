// Launch-configuration autotuner of the z-pass kernels: measures each compiled tile width of a
// kernel once per grid shape and keeps the fastest (see autotune.h).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "autotune.h"

namespace {
const char* const kKinds[] = {"zpass_block_f32", "zpass_block_bf16x3", "zpass_block_k_f32"};

std::mutex g_mu;
std::map<std::array<int, 6>, int> g_pick;
std::vector<std::string> g_report;

// median device time of three launches of configuration c on the scratch spectrum, or a negative
// value when a launch fails
float time_config(int c, cudaStream_t s, const std::function<int(int, cudaStream_t, const ZFArgs&)>& launch,
                  const ZFArgs& zt) {
    cudaEvent_t e[4];
    for (auto& ev : e)
        if (cudaEventCreate(&ev) != cudaSuccess) return -1.f;
    float out = -1.f;
    if (launch(c, s, zt) == VIE_OK) {  // warm-up (kernel attributes, instruction cache)
        float t[3];
        bool ok = true;
        for (int i = 0; i < 3 && ok; ++i) {
            ok = cudaEventRecord(e[0], s) == cudaSuccess && launch(c, s, zt) == VIE_OK &&
                 cudaEventRecord(e[1], s) == cudaSuccess && cudaEventSynchronize(e[1]) == cudaSuccess &&
                 cudaEventElapsedTime(&t[i], e[0], e[1]) == cudaSuccess;
        }
        if (ok) {
            std::sort(t, t + 3);
            out = t[1];
        }
    }
    cudaGetLastError();
    for (auto& ev : e) cudaEventDestroy(ev);
    return out;
}
}  // namespace

int autotune_pick(const int key[5], int n, cudaStream_t s,
                  const std::function<int(int, cudaStream_t, const ZFArgs&)>& launch, const ZFArgs& z,
                  const std::function<std::string(int)>& label) {
    if (n <= 1) return 0;
    // right-hand sides of the measurement: the launch's count rounded up to a power of two, at most 8
    int rt = 1;
    while (rt < z.R && rt < 8) rt *= 2;
    const std::array<int, 6> k{key[0], key[1], key[2], key[3], key[4], rt};
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_pick.find(k);
    if (it != g_pick.end()) return it->second;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 0;
    }
    // scratch spectrum [rt * 12][nz][Ly][Lx] of zeros; the measured kernels work in place on it
    ZFArgs zt = z;
    zt.R = rt;
    zt.nact = nullptr;
    zt.bctr = nullptr;
    const size_t bytes = sizeof(float2) * (size_t)rt * 12 * z.nz * z.Ly * z.Lx;
    float2* w = nullptr;
    int pick = 0;
    std::string line = std::string(kKinds[key[0]]) + " Lz=" + std::to_string(key[1]) + " Lx=" +
                       std::to_string(key[2]) + " Ly=" + std::to_string(key[3]) + " nz=" + std::to_string(key[4]) +
                       " R<=" + std::to_string(rt) + ":";
    if (cudaMalloc(&w, bytes) == cudaSuccess && cudaMemsetAsync(w, 0, bytes, s) == cudaSuccess) {
        zt.w = w;
        float best = -1.f;
        for (int c = 0; c < n; ++c) {
            const float t = time_config(c, s, launch, zt);
            char buf[64];
            std::snprintf(buf, sizeof(buf), " %s %.4f ms", label(c).c_str(), t);
            line += buf;
            if (t > 0.f && (best < 0.f || t < best)) best = t, pick = c;
        }
    } else {
        line += " no scratch memory, default";
    }
    cudaStreamSynchronize(s);
    cudaFree(w);
    cudaGetLastError();
    line += " -> " + label(pick);
    g_pick[k] = pick;
    g_report.push_back(line);
    return pick;
}

extern "C" int vie_tuning(char* out, size_t len) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::string all;
    for (const auto& l : g_report) all += l + "\n";
    if (out && len > 0) {
        const size_t n = std::min(len - 1, all.size());
        std::memcpy(out, all.data(), n);
        out[n] = 0;
    }
    return (int)all.size();
}
