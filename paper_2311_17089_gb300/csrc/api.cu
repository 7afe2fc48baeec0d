// Error reporting and small host utilities shared by the entry points.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <set>
#include <string>
#include <tuple>

#include "common.cuh"

namespace msgs {

static thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MS_OK;
    return fail(MS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int num_sms() {
    static std::atomic<int> cached[64];  // zero-initialised (static storage)
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    if (n < 1) n = 1;
    if (dev >= 0 && dev < 64) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

int ensure_smem_attr(const void *func, int bytes) {
    // the attribute belongs to the function on the current device: set once
    // per (device, function, size), from any host thread
    static std::mutex mu;
    static std::set<std::tuple<int, const void *, int>> done;
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    const auto key = std::make_tuple(dev, func, bytes);
    {
        std::lock_guard<std::mutex> g(mu);
        if (done.count(key)) return MS_OK;
    }
    rc = cuda_check(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                    "shared memory attribute");
    if (rc) return rc;
    std::lock_guard<std::mutex> g(mu);
    done.insert(key);
    return MS_OK;
}

static std::atomic<uint32_t> g_bin_spin_limit{0};

uint32_t bin_spin_limit() {
    const uint32_t v = g_bin_spin_limit.load(std::memory_order_relaxed);
    return v ? v : kSpinLimit;
}

}  // namespace msgs

extern "C" int ms_debug_set_spin_limit(uint32_t limit) {
    msgs::g_bin_spin_limit.store(limit, std::memory_order_relaxed);
    return MS_OK;
}

extern "C" const char *ms_last_error(void) { return msgs::g_last_error.c_str(); }

extern "C" int ms_version(void) { return 100; }
