// Throughput probes of the execution units the blend is bound by: the FP32
// pipe (scalar FFMA and Blackwell's packed fma.rn.f32x2) and the MUFU ex2
// unit.  Each thread runs kChains independent dependency chains so the
// pipes stay full; the result is written out so nothing is dead code.  The
// caller times a launch with CUDA events and divides the operation count
// (ms_alu_probe_ops) by the time: the measured peak the raster roofline
// divides by, at the clock the GPU ran during the launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "f32x2.cuh"

namespace msgs {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) probe_ffma(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_ffma2(float *out, int iters, float a, float b) {
    f32x2 x[kChains];
    const f32x2 a2 = splat2(a), b2 = splat2(b);
#pragma unroll
    for (int c = 0; c < kChains; c++)
        x[c] = pack2((float)(threadIdx.x + c) * 1e-3f, (float)(threadIdx.x - c) * 1e-3f);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma2(x[c], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        float lo, hi;
        unpack2(x[c], lo, hi);
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

// x -> 2^-x maps (0, 1] into [0.5, 1): the chains stay in range.
__global__ void __launch_bounds__(256) probe_ex2(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = a + (float)(threadIdx.x + c) * 1e-4f * b;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = ex2_neg(x[c]);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace msgs

using namespace msgs;

extern "C" double ms_alu_probe_ops(int kind, int blocks, int iters) {
    if (kind < MS_PROBE_FFMA || kind > MS_PROBE_EX2 || blocks < 1 || iters < 1) return 0.0;
    const double per = (double)blocks * 256.0 * iters * kUnroll * kChains;
    return kind == MS_PROBE_FFMA2 ? 2.0 * per : per;
}

extern "C" int ms_alu_probe(int kind, int blocks, int iters, float *out, void *stream) {
    if (kind < MS_PROBE_FFMA || kind > MS_PROBE_EX2)
        return fail(MS_ERR_INVALID_ARG, "unknown probe kind");
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || !out)
        return fail(MS_ERR_INVALID_ARG, "blocks must be 1..2^20, iters >= 1, out non-NULL");
    cudaStream_t st = as_stream(stream);
    if (kind == MS_PROBE_FFMA) probe_ffma<<<blocks, 256, 0, st>>>(out, iters, 0.999f, 1e-3f);
    else if (kind == MS_PROBE_FFMA2) probe_ffma2<<<blocks, 256, 0, st>>>(out, iters, 0.999f, 1e-3f);
    else probe_ex2<<<blocks, 256, 0, st>>>(out, iters, 0.5f, 1.0f);
    return cuda_check(cudaGetLastError(), "probe launch");
}
