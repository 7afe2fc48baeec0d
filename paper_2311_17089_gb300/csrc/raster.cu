// Front-to-back blending per 16x16 tile (Sec. 3.1; Eq. 3 with incremental
// transmittance): one 256-thread CTA per tile, one thread per pixel.
//
// The tile's sorted list is walked in batches of 256 records; each thread
// gathers one record into shared memory (converting the conic to log2
// units so the pixel loop needs one ex2 per evaluation), then every pixel
// thread blends the batch from registers.  A CTA stops early once all its
// pixels have terminated (__syncthreads_count vote at batch boundaries).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace msgs {

constexpr int kRasterThreads = 256;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kRasterThreads)
raster_kernel(const uint32_t *__restrict__ ranges, const uint32_t *__restrict__ gidx,
              const float4 *__restrict__ rec, uint32_t n_rec, int W, int H, int tiles_x,
              float bg0,
              float bg1, float bg2, float *__restrict__ image,
              float *__restrict__ final_t, uint32_t *__restrict__ n_contrib,
              uint32_t *__restrict__ n_eval) {
    __shared__ float4 s_r0[kRasterThreads];
    __shared__ float4 s_r1[kRasterThreads];
    __shared__ float s_b[kRasterThreads];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * 16 + (tid & 15), py = ty * 16 + (tid >> 4);
    const bool inside = px < W && py < H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    bool done = !inside;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0, evals = end - start;
    for (uint32_t b = start; b < end; b += kRasterThreads) {
        if (__syncthreads_count(done) == kRasterThreads) break;
        const uint32_t j = b + tid;
        if (j < end) {
            uint32_t g = gidx[j];
            if (g >= n_rec) g = 0;  // unreachable unless binning reported an error
            float4 r0 = rec[3 * (size_t)g];
            float4 r1 = rec[3 * (size_t)g + 1];
            float rb = reinterpret_cast<const float *>(rec)[12 * (size_t)g + 8];
            // power * log2(e) = A dx^2 + B dx dy + C dy^2
            s_r0[tid] = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
            s_r1[tid] = make_float4(-0.5f * kLog2e * r1.x, r1.y, r1.z, r1.w);
            s_b[tid] = rb;
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kRasterThreads, end - b);
        if (!done) {
            for (int k = 0; k < cnt; k++) {
                const float4 r0 = s_r0[k];
                const float4 r1 = s_r1[k];
                const float dx = fx - r0.x, dy = fy - r0.y;
                const float u = fmaf(r0.w, dy, r0.z * dx);
                const float p = fmaf(r1.x * dy, dy, dx * u);
                if (p > 0.0f) continue;
                const float al = fminf(kAlphaMax, r1.y * ex2_approx(p));
                if (al < kAlphaMin) continue;
                const float Tn = fmaf(-al, T, T);
                if (Tn < kTStop) {
                    done = true;
                    evals = b - start + (uint32_t)k + 1;
                    break;
                }
                const float wgt = al * T;
                C0 = fmaf(wgt, r1.z, C0);
                C1 = fmaf(wgt, r1.w, C1);
                C2 = fmaf(wgt, s_b[k], C2);
                T = Tn;
                last = b - start + (uint32_t)k + 1;
            }
        }
    }
    if (inside) {
        const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
        image[p] = fmaf(T, bg0, C0);
        image[plane + p] = fmaf(T, bg1, C1);
        image[2 * plane + p] = fmaf(T, bg2, C2);
        if (final_t) final_t[p] = T;
        if (n_contrib) n_contrib[p] = last;
        if (n_eval) n_eval[p] = evals;
    }
}

}  // namespace msgs

using namespace msgs;

extern "C" int ms_raster(const ms_proj_t *proj, const ms_bins_t *bins, const ms_camera_t *cam,
                         float *image, float *final_t, uint32_t *n_contrib, uint32_t *n_eval,
                         void *stream) {
    if (!proj || !bins || !cam || !image) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
    if (!proj->rec || !aligned(proj->rec, 16)) return fail(MS_ERR_INVALID_ARG, "rec NULL or misaligned");
    if (!bins->gauss_idx || !bins->ranges) return fail(MS_ERR_INVALID_ARG, "bins buffers NULL");
    if (proj->n < 1 || proj->n > INT32_MAX) return fail(MS_ERR_INVALID_ARG, "ms_proj_t n must be 1..2^31-1");
    const int tiles_x = (cam->width + 15) / 16, tiles_y = (cam->height + 15) / 16;
    raster_kernel<<<tiles_x * tiles_y, kRasterThreads, 0, as_stream(stream)>>>(
        bins->ranges, bins->gauss_idx, reinterpret_cast<const float4 *>(proj->rec),
        (uint32_t)(proj->n > 0 ? proj->n : 0), cam->width,
        cam->height, tiles_x, cam->bg[0], cam->bg[1], cam->bg[2], image, final_t, n_contrib, n_eval);
    return cuda_check(cudaGetLastError(), "raster_kernel launch");
}
