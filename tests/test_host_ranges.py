"""The library's host-thread helper (host_ranges in csrc/iedd_internal.cuh), which the RS factor's
level planning and the CBD partition run their independent items on (no GPU).

A small C++ program includes the internal header and checks the helper's contract: every index
of [0, n) is visited exactly once, in contiguous ranges; fewer than `grain` items per thread run
on the caller alone; an exception thrown in any range reaches the caller after every thread has
ended.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_12574_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")

PROGRAM = r"""
#include "iedd_internal.cuh"

#include <atomic>
#include <cstdio>
#include <stdexcept>
#include <thread>
#include <vector>

void ie_set_error(const std::string &) {}

int main() {
    // every index exactly once, for sizes around the thread split
    for (long long n : {0LL, 1LL, 7LL, 64LL, 1000LL, 100003LL}) {
        for (long long grain : {1LL, 16LL, 1000LL}) {
            std::vector<std::atomic<int>> hits((size_t)n);
            for (auto &h : hits) h = 0;
            host_ranges(n, grain, [&](long long b0, long long b1) {
                for (long long i = b0; i < b1; ++i) hits[(size_t)i]++;
            });
            for (long long i = 0; i < n; ++i)
                if (hits[(size_t)i] != 1) { std::printf("index %lld of %lld visited %d times\n", i, n, (int)hits[(size_t)i]); return 1; }
        }
    }
    // fewer than `grain` items per thread: one range, on the caller's thread
    {
        const std::thread::id me = std::this_thread::get_id();
        int ranges = 0;
        bool elsewhere = false;
        host_ranges(100, 1000, [&](long long, long long) {
            ++ranges;
            elsewhere = elsewhere || std::this_thread::get_id() != me;
        });
        if (ranges != 1 || elsewhere) { std::printf("small input split: %d ranges\n", ranges); return 2; }
    }
    // an exception in one range reaches the caller once the other ranges have finished
    {
        std::atomic<long long> done{0};
        bool caught = false;
        try {
            host_ranges(1 << 20, 1, [&](long long b0, long long b1) {
                if (b0 == 0) throw std::runtime_error("range 0 failed");
                done += b1 - b0;
            });
        } catch (const std::runtime_error &e) {
            caught = std::string(e.what()) == "range 0 failed";
        }
        const long long hc = std::max(1u, std::thread::hardware_concurrency());
        const long long first = (1LL << 20) / std::min(hc, 1LL << 20);
        if (!caught || done != (1LL << 20) - first) {
            std::printf("exception: caught %d, done %lld of %lld\n", (int)caught, (long long)done, (1LL << 20) - first);
            return 3;
        }
    }
    std::printf("ok\n");
    return 0;
}
"""


def test_host_ranges_contract(tmp_path):
    if not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    src = tmp_path / "ranges.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "ranges"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-pthread", str(src),
                        "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
