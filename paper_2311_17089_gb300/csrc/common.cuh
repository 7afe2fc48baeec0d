// Internal helpers of libmsgs (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "msgs.h"

namespace msgs {

// ---------------------------------------------------------------- errors
int fail(int code, const std::string &msg);  // records msg, returns code
int cuda_check(cudaError_t e, const char *what);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
bool aligned(const void *p, size_t a);

// ------------------------------------------- single-rounding FP32 operations
// Each is exactly one IEEE-754 round-to-nearest operation; the compiler may
// not fuse or reorder them, which keeps the footprint reproducible
// bit-for-bit by any implementation doing the same operations in order.
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }

// ----------------------------------------------------------- stats layout
// ms_proj_t::stats words
constexpr int kStatSurvivors = 0;  // uint32 listed Gaussians
constexpr int kStatDup = 2;        // uint64 (words 2-3) sum of n_tiles
constexpr int kStatStatus = 4;     // status bits (kStatusTimeout): uint32 of ms_project; words
                                   // 4-5 as a uint64 where ms_sort_depth records its waits
constexpr int kStatHist = 16;      // 4 x 256 uint32 depth-digit histograms
static_assert(kStatHist + 1024 <= MS_STATS_WORDS, "stats layout");

// ms_bins_t::counts words (uint64)
constexpr int kCntDup = 0;
constexpr int kCntSurvivors = 1;
constexpr int kCntStatus = 2;
constexpr uint64_t kStatusOverflow = 1;
constexpr uint64_t kStatusTimeout = 2;
constexpr uint64_t kStatusBounds = 4;  // a debug build's index check failed

// Index checks of the debug build (compiled with -DMS_DEBUG; nothing in the
// release build): a check that fails sets kStatusBounds in the status word
// `status` (an unsigned long long * in device memory) and the kernel goes
// on along the path its release form takes (every such access is guarded
// or clamped there too); ms_bin_counts then returns MS_ERR_BOUNDS.  No
// check traps.
#ifdef MS_DEBUG
#define MS_DCHECK(cond, status) \
    do { \
        if (!(cond)) atomicOr((status), (unsigned long long)kStatusBounds); \
    } while (0)
#else
#define MS_DCHECK(cond, status) \
    do { \
    } while (0)
#endif

// Raster record: three float4 per Gaussian.
//   r0 = (ux, uy, A, B)      A = -log2(e)/2 conic a, B = -log2(e) conic b
//   r1 = (C, opacity, r, g)  C = -log2(e)/2 conic c
//   r2 = (b, thr, ex, ey)   thr = -log2(e) ln(255 opacity): alpha >= 1/255
//                            exactly when power * log2(e) >= thr; (ex, ey)
//                            the half extents of that level set's box
constexpr int kRecFloats = 12;

// Bounded waits: spin iterations before giving up (each ~100 ns).
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Relaxed (non-fencing) accesses for words that carry their own payload:
// polling them costs no ordering, so many can be in flight at once.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Makes data published before a flag (seen by a relaxed load) visible.
__device__ __forceinline__ void fence_acquire() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int num_sms();
// cudaFuncAttributeMaxDynamicSharedMemorySize = bytes for func on the
// current device, once per (device, function, size); thread-safe
int ensure_smem_attr(const void *func, int bytes);
// Polls the binning's look-back waits make before giving up: kSpinLimit,
// unless a test lowered it (ms_debug_set_spin_limit).
uint32_t bin_spin_limit();

}  // namespace msgs
