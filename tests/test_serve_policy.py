"""Admission policy of the request loop (csrc/serve_policy.h), compiled with g++ and run on the CPU.

The header is plain C++; each case below is a small program that checks one property:
in-order admission, a later request passing a head that does not fit (and the limit on
that), eviction of idle cached Green tensors in least-recently-used order (never one in
use, never the request's own), and a cached key costing only the working set.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1902_02196_gb300", "csrc", "serve_policy.h")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "serve_policy.h"
using namespace serve;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)
int main() {
    std::vector<CacheView> none;
    // 1. in order: the head fits, it goes first
    {
        std::vector<QueuedView> q = {{10, 5, -1, 0}, {1, 1, -1, 0}};
        Decision d = admit(q, none, 100, 4);
        CHECK(d.pick == 0 && d.evict.empty());
    }
    // 2. the head does not fit, a smaller one behind it does
    {
        std::vector<QueuedView> q = {{80, 30, -1, 0}, {10, 5, -1, 0}};
        Decision d = admit(q, none, 50, 4);
        CHECK(d.pick == 1);
    }
    // 3. ... but not once the head has been passed max_bypass times
    {
        std::vector<QueuedView> q = {{80, 30, -1, 4}, {10, 5, -1, 0}};
        Decision d = admit(q, none, 50, 4);
        CHECK(d.pick == -1);
    }
    // 4. nothing fits: no pick
    {
        std::vector<QueuedView> q = {{80, 30, -1, 0}, {70, 5, -1, 0}};
        Decision d = admit(q, none, 50, 4);
        CHECK(d.pick == -1 && d.evict.empty());
    }
    // 5. a cached key needs only the working set
    {
        std::vector<CacheView> c = {{40, 1, 7}};
        std::vector<QueuedView> q = {{20, 40, 0, 0}};
        Decision d = admit(q, c, 25, 4);
        CHECK(d.pick == 0 && d.evict.empty());
        std::vector<QueuedView> q2 = {{20, 40, -1, 0}};
        CHECK(admit(q2, c, 25, 4).pick == -1);  // same request without the cache entry does not fit
    }
    // 6. eviction: idle entries only, least recently used first, just enough of them
    {
        std::vector<CacheView> c = {{30, 0, 5}, {30, 1, 1}, {30, 0, 2}, {30, 0, 9}};
        std::vector<QueuedView> q = {{40, 20, -1, 0}};  // needs 60, 10 free
        Decision d = admit(q, c, 10, 4);
        CHECK(d.pick == 0);
        CHECK(d.evict.size() == 2 && d.evict[0] == 2 && d.evict[1] == 0);  // last 2, then 5; never entry 1 (in use)
    }
    // 7. a request's own idle entry is not evicted for it
    {
        std::vector<CacheView> c = {{50, 0, 1}, {30, 0, 3}};
        std::vector<QueuedView> q = {{35, 50, 0, 0}};  // needs 35 (cached), 10 free: evict entry 1, keep 0
        Decision d = admit(q, c, 10, 4);
        CHECK(d.pick == 0 && d.evict.size() == 1 && d.evict[0] == 1);
    }
    // 8. eviction cannot make room: the head waits, later requests may pass
    {
        std::vector<CacheView> c = {{30, 1, 1}};
        std::vector<QueuedView> q = {{90, 10, -1, 0}, {5, 5, -1, 0}};
        Decision d = admit(q, c, 20, 4);
        CHECK(d.pick == 1 && d.evict.empty());
    }
    std::printf("OK\n");
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_serve_policy(tmp_path):
    src = tmp_path / "policy_test.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "policy_test"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout
