// AggregateGaussians for one coarse level l_m (Alg. 1; Sec. 4.1 "Aggregate
// to Insert Large Gaussians"; supplementary "Details of Gaussian
// Aggregation Algorithm"), on the device:
//   1. agg_cover_kernel, once per training camera (already downsampled by
//      4^(l_m-1)): the FP32 footprint of every Gaussian of levels < l_m;
//      a Gaussian splatted to the camera (valid, touching its image) keeps
//      the smallest coverage S seen.
//   2. agg_key_kernel: small Gaussians (smallest S < S_T = 2 px) get the
//      voxel key of their normalised position (per component x / B inside
//      [-B, B], sign(x) (2 - B / |x|) outside; floor(400 / l_m) voxels per
//      axis over [-2, 2]), computed in FP32 in a fixed operation order, plus
//      the digit histograms of the sort.
//   3. Three onesweep passes sort the small Gaussians by key (the first
//      compacts them; stable, so each voxel's members stay in index order).
//   4. agg_heads_kernel / agg_scan_kernel number the voxels; agg_pool_kernel
//      averages each voxel's members (position, quaternion, log-scale,
//      opacity, colour, coverage) in index order and enlarges the scale by
//      S_T / S_avg (adds ln(S_T / S_avg) to the averaged log-scales).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "footprint.cuh"
#include "sort.cuh"

namespace msgs {

constexpr float kST = 2.0f;             // S_T, the selection threshold (Eq. 6)
constexpr int kAggThreads = 256;
constexpr int kAggPasses = 3;           // keys below 2^24 (R <= 200)

__global__ void agg_init_kernel(int64_t n, float *__restrict__ smin) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        smin[i] = __int_as_float(0x7f800000);
}

__global__ void agg_cover_kernel(SceneK sc, CamK cam, int level_m, float *__restrict__ smin) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sc.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (sc.level[i] >= level_m) continue;
        float m[3] = {sc.mean[3 * i], sc.mean[3 * i + 1], sc.mean[3 * i + 2]};
        float s[3] = {sc.scale[3 * i], sc.scale[3 * i + 1], sc.scale[3 * i + 2]};
        float4 q = reinterpret_cast<const float4 *>(sc.quat)[i];
        Foot f;
        footprint(m, s, q, sc.lnop[i], cam, f);
        if (f.valid && f.ntiles > 0 && f.S < smin[i]) smin[i] = f.S;
    }
}

__device__ __forceinline__ float norm32(float x, float B) {
    const float ax = fabsf(x);
    if (ax <= B) return fdv(x, B);
    const float t = fs(2.0f, fdv(B, ax));
    return x < 0.0f ? -t : t;
}

__device__ __forceinline__ uint32_t vox32(float xn, int R) {
    const float t = fm(fa(xn, 2.0f), (float)R * 0.25f);
    int v = (int)floorf(t);
    v = v < 0 ? 0 : (v > R - 1 ? R - 1 : v);
    return (uint32_t)v;
}

__global__ void __launch_bounds__(kAggThreads)
agg_key_kernel(SceneK sc, int level_m, float B, const float *__restrict__ smin,
               uint32_t *__restrict__ flag, uint32_t *__restrict__ keys,
               uint32_t *__restrict__ hist, uint32_t *__restrict__ n_small) {
    __shared__ uint32_t s_hist[kAggPasses][256];
    __shared__ uint32_t s_count;
    for (int i = threadIdx.x; i < kAggPasses * 256; i += kAggThreads) (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int R = 400 / level_m;
    uint32_t local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sc.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool small = sc.level[i] < level_m && smin[i] < kST;
        flag[i] = small ? 1u : 0u;
        if (!small) continue;
        const uint32_t vx = vox32(norm32(sc.mean[3 * i], B), R);
        const uint32_t vy = vox32(norm32(sc.mean[3 * i + 1], B), R);
        const uint32_t vz = vox32(norm32(sc.mean[3 * i + 2], B), R);
        const uint32_t key = (vz * (uint32_t)R + vy) * (uint32_t)R + vx;
        keys[i] = key;
        for (int p = 0; p < kAggPasses; p++) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
        local++;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&s_count, local);
    __syncthreads();
    for (int i = threadIdx.x; i < kAggPasses * 256; i += kAggThreads) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
    if (threadIdx.x == 0 && s_count) atomicAdd(n_small, s_count);
}

// Voxel heads per block of kAggThreads sorted items.
__global__ void __launch_bounds__(kAggThreads)
agg_heads_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ n_small,
                 uint32_t *__restrict__ block_heads) {
    const uint32_t m = *n_small;
    const uint64_t j = (uint64_t)blockIdx.x * kAggThreads + threadIdx.x;
    const bool head = j < m && (j == 0 || keys[j] != keys[j - 1]);
    const uint32_t c = __syncthreads_count(head);
    if (threadIdx.x == 0) block_heads[blockIdx.x] = c;
}

// Exclusive scan of the per-block head counts (one block); total voxels
// to *groups.
__global__ void __launch_bounds__(1024)
agg_scan_kernel(uint32_t *__restrict__ block_heads, int nblocks,
                const unsigned long long *__restrict__ err,
                unsigned long long *__restrict__ groups) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? block_heads[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const uint32_t excl = s_carry + (warp ? s_warp[warp - 1] : 0u) + x - v;
        if (i < nblocks) block_heads[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        groups[0] = s_carry;
        groups[1] = *err;  // status bits of the sort passes
    }
}

struct AggOut {
    float *mean, *log_scale, *quat, *opacity, *color, *s_max, *s_min;
    uint8_t *level;
    int64_t capacity;
};

// One thread per voxel head: average the voxel's members in sorted (index)
// order and write the new Gaussian at the voxel's ordinal.
template <int K>
__global__ void __launch_bounds__(kAggThreads)
agg_pool_kernel(SceneK sc, const float *__restrict__ log_scale, int level_m,
                const float *__restrict__ smin, const uint32_t *__restrict__ keys,
                const uint32_t *__restrict__ idx, const uint32_t *__restrict__ n_small,
                const uint32_t *__restrict__ block_base, AggOut out) {
    __shared__ uint32_t s_warp[kAggThreads / 32];
    const uint32_t m = *n_small;
    const uint64_t j = (uint64_t)blockIdx.x * kAggThreads + threadIdx.x;
    const bool head = j < m && (j == 0 || keys[j] != keys[j - 1]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, head);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; w++) before += s_warp[w];
    if (!head) return;
    const uint64_t g = (uint64_t)block_base[blockIdx.x] + before +
                       __popc(bal & ((1u << lane) - 1u));
    if ((int64_t)g >= out.capacity) return;
    float sm[3] = {0, 0, 0}, sl[3] = {0, 0, 0}, sq[4] = {0, 0, 0, 0}, so = 0.0f, ss = 0.0f;
    float scol[3 * K];
#pragma unroll
    for (int k = 0; k < 3 * K; k++) scol[k] = 0.0f;
    const uint32_t key = keys[j];
    uint32_t cnt = 0;
    for (uint64_t t = j; t < m && keys[t] == key; t++, cnt++) {
        const uint64_t i = idx[t];
        for (int k = 0; k < 3; k++) {
            sm[k] += sc.mean[3 * i + k];
            sl[k] += log_scale[3 * i + k];
        }
        const float4 q = reinterpret_cast<const float4 *>(sc.quat)[i];
        sq[0] += q.x;
        sq[1] += q.y;
        sq[2] += q.z;
        sq[3] += q.w;
        so += sc.opacity[i];
        ss += smin[i];
#pragma unroll
        for (int k = 0; k < 3 * K; k++) scol[k] += sc.color[(size_t)3 * K * i + k];
    }
    const float inv = 1.0f / (float)cnt;
    const float grow = logf(kST / (ss * inv));
    for (int k = 0; k < 3; k++) {
        out.mean[3 * g + k] = sm[k] * inv;
        out.log_scale[3 * g + k] = sl[k] * inv + grow;
    }
    for (int k = 0; k < 4; k++) out.quat[4 * g + k] = sq[k] * inv;
    out.opacity[g] = so * inv;
#pragma unroll
    for (int k = 0; k < 3 * K; k++) out.color[(size_t)3 * K * g + k] = scol[k] * inv;
    out.level[g] = (uint8_t)level_m;
    out.s_max[g] = 0.0f;
    out.s_min[g] = __int_as_float(0x7f800000);
}

struct AggLayout {
    size_t smin, flag, keys, ka, va, kb, vb, hist, status, tickets, n_small, err, heads, total,
        zero_begin;
    int64_t parts, hblocks;
};

static bool agg_layout(int64_t n, AggLayout &L) {
    if (n < 0 || n > kMaxSortItems) return false;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    L.parts = sort_parts((uint64_t)nn);
    L.hblocks = ceil_div((int64_t)nn, kAggThreads);
    size_t o = 0;
    L.smin = o;
    o = up(o + nn * 4);
    L.flag = o;
    o = up(o + nn * 4);
    L.keys = o;
    o = up(o + nn * 4);
    L.ka = o;
    o = up(o + nn * 4);
    L.va = o;
    o = up(o + nn * 4);
    L.kb = o;
    o = up(o + nn * 4);
    L.vb = o;
    o = up(o + nn * 4);
    L.heads = o;
    o = up(o + (size_t)L.hblocks * 4);
    L.zero_begin = o;
    L.hist = o;
    o = up(o + kAggPasses * 256 * 4);
    L.status = o;
    o = up(o + (size_t)kAggPasses * L.parts * 256 * 4);
    L.tickets = o;
    o = up(o + kAggPasses * 4);
    L.n_small = o;
    o = up(o + 8);
    L.err = o;
    o = up(o + 8);
    L.total = o;
    return true;
}

}  // namespace msgs

using namespace msgs;

extern "C" size_t ms_aggregate_workspace_bytes(int64_t n) {
    AggLayout L;
    return agg_layout(n, L) ? L.total : 0;
}

extern "C" int ms_aggregate(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_cams,
                            int32_t level_m, float extent, ms_scene_t *out, int64_t capacity,
                            int64_t *n_out, void *ws, size_t ws_bytes, void *stream) {
    int rc;
    if ((rc = check_scene(scene, true))) return rc;
    if (!out || !n_out) return fail(MS_ERR_INVALID_ARG, "out or n_out is NULL");
    if (n_cams < 0 || (n_cams > 0 && !cams)) return fail(MS_ERR_INVALID_ARG, "bad camera list");
    for (int32_t c = 0; c < n_cams; c++)
        if ((rc = check_cam(cams + c))) return rc;
    if (level_m < 2 || level_m > 255 || level_m > scene->n_levels)
        return fail(MS_ERR_INVALID_ARG, "level_m must be in 2..n_levels");
    if (!(extent > 0.0f) || !isfinite(extent)) return fail(MS_ERR_INVALID_ARG, "extent must be > 0");
    if (capacity < 0) return fail(MS_ERR_INVALID_ARG, "capacity must be >= 0");
    if (capacity > 0 && (!out->mean || !out->log_scale || !out->quat || !out->opacity ||
                         !out->color || !out->level || !out->s_max || !out->s_min))
        return fail(MS_ERR_INVALID_ARG, "out has a NULL array");
    if (capacity > 0 && !aligned(out->quat, 16))
        return fail(MS_ERR_INVALID_ARG, "out quat must be 16-byte aligned");
    if (out->sh_degree != scene->sh_degree)
        return fail(MS_ERR_INVALID_ARG, "out sh_degree differs from the scene's");
    if (!scene->log_scale) return fail(MS_ERR_INVALID_ARG, "scene log_scale is NULL");
    AggLayout L;
    if (!agg_layout(scene->n, L)) return fail(MS_ERR_INVALID_ARG, "scene n out of range");
    if (!ws || ws_bytes < L.total || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "aggregate workspace missing, too small or misaligned");
    cudaStream_t st = as_stream(stream);
    char *w = static_cast<char *>(ws);
    if ((rc = cuda_check(cudaMemsetAsync(w + L.zero_begin, 0, L.total - L.zero_begin, st),
                         "aggregate workspace memset")))
        return rc;
    if ((rc = cuda_check(cudaMemsetAsync(n_out, 0, 2 * sizeof(int64_t), st), "n_out memset")))
        return rc;
    const int64_t n = scene->n;
    if (n == 0) return MS_OK;
    const SceneK sk = make_scene(*scene);
    float *smin = reinterpret_cast<float *>(w + L.smin);
    uint32_t *flag = reinterpret_cast<uint32_t *>(w + L.flag);
    uint32_t *keys = reinterpret_cast<uint32_t *>(w + L.keys);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    uint32_t *n_small = reinterpret_cast<uint32_t *>(w + L.n_small);
    uint32_t *heads = reinterpret_cast<uint32_t *>(w + L.heads);
    const int grid = grid_for(n, kAggThreads, 8);
    agg_init_kernel<<<grid, kAggThreads, 0, st>>>(n, smin);
    for (int32_t c = 0; c < n_cams; c++)
        agg_cover_kernel<<<grid, kAggThreads, 0, st>>>(sk, make_cam(cams[c]), level_m, smin);
    agg_key_kernel<<<grid, kAggThreads, 0, st>>>(sk, level_m, extent, smin, flag, keys, hist,
                                                 n_small);
    uint32_t *bufs_k[2] = {reinterpret_cast<uint32_t *>(w + L.ka),
                           reinterpret_cast<uint32_t *>(w + L.kb)};
    uint32_t *bufs_v[2] = {reinterpret_cast<uint32_t *>(w + L.va),
                           reinterpret_cast<uint32_t *>(w + L.vb)};
    for (int p = 0; p < kAggPasses; p++) {
        PassArgs a;
        a.keys_in = p == 0 ? keys : bufs_k[(p - 1) & 1];
        a.vals_in = p == 0 ? nullptr : bufs_v[(p - 1) & 1];
        a.filter = p == 0 ? flag : nullptr;
        a.keys_out = bufs_k[p & 1];
        a.vals_out = bufs_v[p & 1];
        a.n32 = p == 0 ? nullptr : n_small;
        a.n64 = nullptr;
        a.n_cap = (uint64_t)n;
        a.shift = 8 * p;
        a.hist = hist + 256 * p;
        a.status = reinterpret_cast<uint32_t *>(w + L.status) + (size_t)p * L.parts * 256;
        a.ticket = reinterpret_cast<uint32_t *>(w + L.tickets) + p;
        a.err = reinterpret_cast<unsigned long long *>(w + L.err);
        if ((rc = launch_onesweep(a, (uint64_t)n, st))) return rc;
    }
    const uint32_t *skeys = bufs_k[(kAggPasses - 1) & 1];
    const uint32_t *sidx = bufs_v[(kAggPasses - 1) & 1];
    agg_heads_kernel<<<(int)L.hblocks, kAggThreads, 0, st>>>(skeys, n_small, heads);
    agg_scan_kernel<<<1, 1024, 0, st>>>(heads, (int)L.hblocks,
                                         reinterpret_cast<unsigned long long *>(w + L.err),
                                         reinterpret_cast<unsigned long long *>(n_out));
    // `out` describes arrays this call writes (ms_scene_t declares scene
    // arrays const because every other entry point only reads them)
    AggOut o = {const_cast<float *>(out->mean), const_cast<float *>(out->log_scale),
                const_cast<float *>(out->quat), const_cast<float *>(out->opacity),
                const_cast<float *>(out->color), const_cast<float *>(out->s_max),
                const_cast<float *>(out->s_min), const_cast<uint8_t *>(out->level), capacity};
    switch (scene->sh_degree) {
    case 0: agg_pool_kernel<1><<<(int)L.hblocks, kAggThreads, 0, st>>>(sk, scene->log_scale, level_m, smin, skeys, sidx, n_small, heads, o); break;
    case 1: agg_pool_kernel<4><<<(int)L.hblocks, kAggThreads, 0, st>>>(sk, scene->log_scale, level_m, smin, skeys, sidx, n_small, heads, o); break;
    case 2: agg_pool_kernel<9><<<(int)L.hblocks, kAggThreads, 0, st>>>(sk, scene->log_scale, level_m, smin, skeys, sidx, n_small, heads, o); break;
    case 3: agg_pool_kernel<16><<<(int)L.hblocks, kAggThreads, 0, st>>>(sk, scene->log_scale, level_m, smin, skeys, sidx, n_small, heads, o); break;
    default: agg_pool_kernel<1><<<(int)L.hblocks, kAggThreads, 0, st>>>(sk, scene->log_scale, level_m, smin, skeys, sidx, n_small, heads, o);
    }
    return cuda_check(cudaGetLastError(), "aggregate launches");
}
