// Tile binning (Sec. 3.1: every 2D Gaussian touching a 16x16 tile is listed
// for it, and each list is sorted by the Gaussians' view-space depth).
//
// Design: instead of one radix sort of D 64-bit (tile, depth) keys, the
// listed Gaussians are first sorted by their 32-bit depth bits (4 onesweep
// passes over the N_s survivors; the first pass also compacts them out of
// the N-long footprint arrays), then expanded to one (tile, index) entry per
// covered tile in depth order, then stably sorted by tile id (1-2 passes
// over D entries).  Stability gives every tile's list in (depth, index)
// order, exactly the order of a (tile, depth, index) sort.
//
// Onesweep pass (single-pass LSD radix step): each CTA takes a 2048-item
// partition by atomic ticket, ranks its items stably per 8-bit digit with
// warp match, publishes its per-digit counts and obtains the counts of all
// earlier partitions by decoupled look-back, then scatters through shared
// memory.  A look-back word carries its own count, so it is published and
// polled with relaxed accesses (no fences; many polls in flight at once).  Every wait on another CTA is bounded; a wait that gives up sets
// a status bit and the CTA carries on, so a kernel can never hang.
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "sort.cuh"

namespace msgs {

constexpr int kDupThreads = 256;
constexpr int kDupIPT = 4;
constexpr int kDupPart = kDupThreads * kDupIPT;
constexpr int kDupRun = 8;                      // entries one thread emits per window
constexpr int kDupWin = kDupThreads * kDupRun;  // entries staged per window
constexpr unsigned long long kDupFlagAgg = 1ull << 62;
constexpr unsigned long long kDupFlagPre = 2ull << 62;
constexpr unsigned long long kDupValMask = (1ull << 62) - 1;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over the first 256 threads of the
// block (the other threads pass 0 and get their result ignored); every
// thread of the block must call it.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t *s_warp,
                                                       uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31 && warp < kScanWarps) s_warp[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kScanWarps; w++) {
        uint32_t t = s_warp[w];
        if (w < warp) wpre += t;
        total += t;
    }
    __syncthreads();
    return wpre + x - v;
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t pass_count(const PassArgs &a) {
    uint64_t n = a.n_cap;
    if (a.n32) n = umin64(n, *a.n32);
    if (a.n64) n = umin64(n, *a.n64);
    return n;
}


template <int IPT>
__global__ void __launch_bounds__(kSortThreads)
onesweep_pass(PassArgs a) {
    constexpr int kPart = SortCfg<IPT>::kPart;
    extern __shared__ __align__(16) uint32_t sort_smem[];
    uint32_t(*s_whist)[kDigits] = reinterpret_cast<uint32_t(*)[kDigits]>(sort_smem);
    uint32_t *s_keys = sort_smem + kSortWarps * kDigits;
    uint32_t *s_vals = s_keys + kPart;
    __shared__ uint32_t s_base[kDigits];
    __shared__ uint32_t s_excl[kDigits];
    __shared__ uint32_t s_prefix[kDigits];
    __shared__ uint32_t s_gofs[kDigits];
    __shared__ uint32_t s_warp[kScanWarps];
    __shared__ uint32_t s_part;
    __shared__ uint32_t s_total;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a pass holds fewer than 2^30 items (kMaxSortItems), so item indices
    // and scatter positions are 32-bit and digit counts fit the look-back
    // words' 30 bits
    const uint32_t n = (uint32_t)pass_count(a);
    const uint32_t parts = (n + kPart - 1) / kPart;
    {
        uint32_t tot;
        uint32_t b = block_excl_scan256(tid < kDigits ? a.hist[tid] : 0u, s_warp, tot);
        if (tid < kDigits) s_base[tid] = b;
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) s_part = atomicAdd(a.ticket, 1u);
        for (int i = tid; i < kSortWarps * kDigits; i += kSortThreads) (&s_whist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t p = s_part;
        if (p >= parts) break;
        // ---- load every item first (all loads in flight together), then
        // rank (warp-striped, rounds in item order)
        uint32_t key[IPT], val[IPT], rank[IPT];
        bool ok[IPT];
        const uint32_t wbase = p * (uint32_t)kPart + (uint32_t)warp * 32u * IPT;
#pragma unroll
        for (int r = 0; r < IPT; r++) {
            const uint32_t i = wbase + (uint32_t)r * 32u + lane;
            ok[r] = i < n;
            if (a.filter && ok[r]) ok[r] = __ldg(a.filter + i) > 0;
        }
#pragma unroll
        for (int r = 0; r < IPT; r++) {
            const uint32_t i = wbase + (uint32_t)r * 32u + lane;
            key[r] = ok[r] ? a.keys_in[i] : 0u;
            val[r] = ok[r] ? (a.vals_in ? a.vals_in[i] : (uint32_t)i) : 0u;
        }
#pragma unroll
        for (int r = 0; r < IPT; r++) {
            const bool valid = ok[r];
            const uint32_t d = (key[r] >> a.shift) & 255u;
            const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u);
            uint32_t before = 0;
            if (valid) before = s_whist[warp][d] + __popc(peers & lanemask_lt());
            __syncwarp();
            if (valid && lane == 31 - __clz(peers)) s_whist[warp][d] += __popc(peers);
            __syncwarp();
            rank[r] = valid ? ((d << 16) | before) : 0xffffffffu;
        }
        __syncthreads();
        // ---- per digit (threads 0..255): warp prefix, partition count,
        // publish, look back
        const uint32_t d = tid;
        uint32_t local = 0;
        if (tid < kDigits) {
            uint32_t run = 0;
#pragma unroll 8
            for (int w = 0; w < kSortWarps; w++) {
                uint32_t c = s_whist[w][d];
                s_whist[w][d] = run;
                run += c;
            }
            local = run;
            uint32_t *st = a.status + (uint64_t)p * kDigits + d;
            if (p == 0) {
                st_relaxed(st, kFlagPre | local);
                s_prefix[d] = 0;
            } else {
                st_relaxed(st, kFlagAgg | local);
                // batched look-back: poll up to kLookback predecessors at
                // once, add aggregates until the nearest inclusive prefix
                uint32_t excl = 0;
                int64_t k = (int64_t)p - 1;
                uint32_t spins = 0;
                while (k >= 0) {
                    uint32_t v[kLookback];
#pragma unroll
                    for (int i = 0; i < kLookback; i++)
                        v[i] = (k - i >= 0) ? ld_relaxed(a.status + (uint64_t)(k - i) * kDigits + d)
                                            : kFlagPre;
                    int i = 0;
                    bool stop = false;
                    for (; i < kLookback; i++) {
                        if ((v[i] & kFlagMask) == 0) break;  // not published yet: poll again
                        excl += v[i] & kValMask;
                        if (v[i] & kFlagPre) {
                            stop = true;
                            break;
                        }
                    }
                    if (stop) break;
                    k -= i;
                    if (i == 0) {
                        if (++spins > a.spin_limit) {
                            atomicOr(a.err, (unsigned long long)kStatusTimeout);
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                st_relaxed(st, kFlagPre | ((excl + local) & kValMask));
                s_prefix[d] = excl;
            }
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan256(local, s_warp, tot);
        if (tid < kDigits) {
            s_excl[d] = ex;
            // output position of the partition's j-th staged item of digit d
            // is s_gofs[d] + j (modulo 2^32)
            s_gofs[d] = s_base[d] + s_prefix[d] - ex;
        }
        if (tid == 0) s_total = tot;
        __syncthreads();
        // ---- stage digit-sorted in shared memory
#pragma unroll
        for (int r = 0; r < IPT; r++) {
            if (rank[r] == 0xffffffffu) continue;
            uint32_t dd = rank[r] >> 16;
            uint32_t pos = s_excl[dd] + s_whist[warp][dd] + (rank[r] & 0xffffu);
            MS_DCHECK(pos < (uint32_t)kPart, a.err);
            s_keys[pos] = key[r];
            s_vals[pos] = val[r];
        }
        __syncthreads();
        // ---- coalesced scatter
        const uint32_t total = s_total;
        for (uint32_t j = tid; j < total; j += kSortThreads) {
            const uint32_t k = s_keys[j];
            const uint32_t g = s_gofs[(k >> a.shift) & 255u] + j;
            if (g >= n) {  // only reachable after a wait gave up
                MS_DCHECK(false, a.err);
                atomicOr(a.err, (unsigned long long)kStatusTimeout);
                continue;
            }
            if (a.keys_out) a.keys_out[g] = k;
            a.vals_out[g] = s_vals[j];
        }
    }
}

// Duplication: exclusive scan of n_tiles in depth order (decoupled look-back
// across partitions), then one (tile id, Gaussian index) entry per covered
// tile, emitted with a block-wide load-balanced search so writes are
// contiguous.  Also accumulates the tile-id digit histograms of the
// following radix passes.
struct DupArgs {
    const uint32_t *order;       // Gaussian indices in depth order
    const uint32_t *n_tiles;
    const uint2 *rect;
    const uint32_t *n32;         // survivors (device)
    uint64_t n_max;              // length of n_tiles / rect
    int tiles_x;
    uint32_t tiles;
    uint64_t cap;
    uint32_t *keys_out, *vals_out;
    uint32_t *hist;              // [2][256]
    unsigned long long *status;  // [partitions]
    uint32_t *ticket;
    unsigned long long *err;
    const unsigned long long *dup;  // duplicates D (device)
    uint32_t *tstatus;           // tile-pass look-back words, zeroed here
    uint64_t tstride;            // words per tile pass in tstatus
    uint32_t tpart;              // partition size of the tile passes
    uint32_t spin_limit;         // look-back polls before a wait gives up
};

// kSparse: the order may hold Gaussians without tiles in this frame (a depth
// order shared by several frames); their rectangles are not loaded.
template <bool kSparse>
__global__ void __launch_bounds__(kDupThreads)
duplicate_kernel(DupArgs a) {
    __shared__ uint32_t s_off[kDupPart + 1];
    __shared__ uint32_t s_idx[kDupPart];
    __shared__ uint2 s_rect[kDupPart];
    __shared__ uint32_t s_hist[2][256];
    __shared__ uint2 s_emit[kDupWin];
    __shared__ uint32_t s_warp[kSortWarps];
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x;
    const uint64_t n = umin64(*a.n32, a.n_max);
    const uint64_t parts = (n + kDupPart - 1) / kDupPart;
    for (int i = tid; i < 512; i += kDupThreads) (&s_hist[0][0])[i] = 0;
    {
        // clear the look-back words the tile passes will use (only as many
        // partitions as D needs; the passes start after this kernel ends)
        const uint64_t words = ((umin64(*a.dup, a.cap) + a.tpart - 1) / a.tpart) * 256;
        for (uint64_t w = blockIdx.x * (uint64_t)kDupThreads + tid; w < words;
             w += (uint64_t)gridDim.x * kDupThreads) {
            a.tstatus[w] = 0u;
            a.tstatus[a.tstride + w] = 0u;
        }
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) s_part = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t p = s_part;
        if (p >= parts) break;
        uint32_t nt[kDupIPT], gi[kDupIPT];
        uint32_t sum = 0;
#pragma unroll
        for (int r = 0; r < kDupIPT; r++) {
            const uint64_t j = (uint64_t)p * kDupPart + tid * kDupIPT + r;
            gi[r] = j < n ? a.order[j] : 0xffffffffu;
        }
#pragma unroll
        for (int r = 0; r < kDupIPT; r++) {
            const uint32_t g = gi[r];
            uint32_t c = 0;
            uint2 rc = make_uint2(0, 0);
            if (g != 0xffffffffu) {
                if (g < a.n_max) {
                    c = a.n_tiles[g];
                    if (!kSparse || c) rc = a.rect[g];
                } else {
                    MS_DCHECK(false, a.err);
                    atomicOr(a.err, (unsigned long long)kStatusTimeout);
                }
            }
            s_idx[tid * kDupIPT + r] = g;
            s_rect[tid * kDupIPT + r] = rc;
            nt[r] = c;
            sum += c;
        }
        uint32_t total;
        uint32_t excl = block_excl_scan256(sum, s_warp, total);
#pragma unroll
        for (int r = 0; r < kDupIPT; r++) {
            s_off[tid * kDupIPT + r] = excl;
            excl += nt[r];
        }
        if (tid == 0) {
            s_off[kDupPart] = total;
            unsigned long long *st = a.status + p;
            unsigned long long pre = 0;
            if (p == 0) {
                st_relaxed64(st, kDupFlagPre | total);
            } else {
                st_relaxed64(st, kDupFlagAgg | total);
                // batched look-back over up to kLookback predecessors
                int64_t k = (int64_t)p - 1;
                uint32_t spins = 0;
                while (k >= 0) {
                    unsigned long long v[kLookback];
#pragma unroll
                    for (int i = 0; i < kLookback; i++)
                        v[i] = (k - i >= 0) ? ld_relaxed64(a.status + (k - i)) : kDupFlagPre;
                    int i = 0;
                    bool stop = false;
                    for (; i < kLookback; i++) {
                        if ((v[i] >> 62) == 0) break;
                        pre += v[i] & kDupValMask;
                        if (v[i] & kDupFlagPre) {
                            stop = true;
                            break;
                        }
                    }
                    if (stop) break;
                    k -= i;
                    if (i == 0) {
                        if (++spins > a.spin_limit) {
                            atomicOr(a.err, (unsigned long long)kStatusTimeout);
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                st_relaxed64(st, kDupFlagPre | ((pre + total) & kDupValMask));
            }
            s_prefix = pre;
        }
        __syncthreads();
        const uint64_t base = s_prefix;
        // emission in windows of kDupWin entries: each thread builds a run of
        // kDupRun consecutive entries (one search for the run's first item,
        // then it steps through the items' tile rectangles), the window is
        // staged in shared memory and written out coalesced
        for (uint32_t w0 = 0; w0 < total; w0 += kDupWin) {
            const uint32_t k0 = w0 + (uint32_t)tid * kDupRun;
            if (k0 < total) {
                // last item whose offset is <= k0
                int lo = 0, hi = kDupPart;  // invariant s_off[lo] <= k0 < s_off[hi]
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (s_off[mid] <= k0) lo = mid;
                    else hi = mid;
                }
                uint2 rc = s_rect[lo];
                uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16;
                uint32_t w = (rc.y & 0xffffu) - x0 + 1;
                const uint32_t m = k0 - s_off[lo];
                uint32_t xx = m % w, yy = m / w;
                uint32_t hb = 0xffffffffu, hc = 0;  // run of equal high bytes
#pragma unroll 4
                for (int r = 0; r < kDupRun; r++) {
                    const uint32_t k = k0 + r;
                    if (k >= total) break;
                    while (k >= s_off[lo + 1]) {  // next item with tiles
                        lo++;
                        rc = s_rect[lo];
                        x0 = rc.x & 0xffffu;
                        y0 = rc.x >> 16;
                        w = (rc.y & 0xffffu) - x0 + 1;
                        xx = 0;
                        yy = 0;
                    }
                    uint32_t tile = (y0 + yy) * (uint32_t)a.tiles_x + x0 + xx;
                    if (++xx == w) {
                        xx = 0;
                        yy++;
                    }
                    if (tile >= a.tiles) {
                        MS_DCHECK(false, a.err);
                        atomicOr(a.err, (unsigned long long)kStatusTimeout);
                        tile = 0xffffffffu;  // not written
                    } else if (base + k < a.cap) {  // the entries the tile passes sort
                        atomicAdd(&s_hist[0][tile & 255u], 1u);
                        const uint32_t h = (tile >> 8) & 255u;
                        if (h != hb) {
                            if (hc) atomicAdd(&s_hist[1][hb], hc);
                            hb = h;
                            hc = 0;
                        }
                        hc++;
                    }
                    s_emit[tid * kDupRun + r] = make_uint2(tile, s_idx[lo]);
                }
                if (hc) atomicAdd(&s_hist[1][hb], hc);
            }
            __syncthreads();
            const uint32_t cnt = min(total - w0, (uint32_t)kDupWin);
            for (uint32_t j = tid; j < cnt; j += kDupThreads) {
                const uint2 e = s_emit[j];
                const uint64_t g = base + w0 + j;
                if (e.x == 0xffffffffu) continue;  // reported above
                if (g < a.cap) {
                    a.keys_out[g] = e.x;
                    a.vals_out[g] = e.y;
                } else {
                    atomicOr(a.err, (unsigned long long)kStatusOverflow);
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int i = tid; i < 512; i += kDupThreads) {
        uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(&a.hist[i], v);
    }
}

// [start, end) of every tile's run in the tile-sorted keys.  Each thread
// takes 8 consecutive keys (two 16-byte loads when the keys are 16-byte
// aligned) and the key on either side, all loaded before any is compared,
// so a thread has several loads in flight instead of one per key.
constexpr uint32_t kNoTile = 0xffffffffu;
__global__ void ranges_kernel(const uint32_t *__restrict__ keys,
                              const unsigned long long *__restrict__ dup, uint64_t cap,
                              uint32_t tiles, uint32_t *__restrict__ ranges) {
    const uint64_t n = umin64(*dup, cap);
    const uint64_t chunks = (n + 7) / 8;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = c * 8;
        uint32_t k[8];
        if (vec && base + 8 <= n) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(keys + base));
            const uint4 b = __ldg(reinterpret_cast<const uint4 *>(keys + base) + 1);
            k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
            k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) k[j] = base + j < n ? __ldg(keys + base + j) : kNoTile;
        }
        const uint32_t prev = base > 0 ? __ldg(keys + base - 1) : kNoTile;
        const uint32_t next = base + 8 < n ? __ldg(keys + base + 8) : kNoTile;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint32_t kk = k[j];
            if (kk >= tiles) continue;  // also the positions past n
            const uint32_t left = j == 0 ? prev : k[j - 1];
            const uint32_t right = j == 7 ? next : k[j + 1];
            const uint32_t i = (uint32_t)(base + j);
            if (left != kk) ranges[2 * (uint64_t)kk] = i;
            if (right != kk) ranges[2 * (uint64_t)kk + 1] = i + 1;
        }
    }
}

// The first kernel of ms_bin: zeroes the workspace's look-back words,
// tickets and histograms and the caller's tile ranges (grid-stride, 16-byte
// stores where aligned), and thread 0 writes the counts: D and the survivors
// from the projection's stats, the status word with the overflow bit, the
// projection's own status and (ms_bin_ordered) the status of the depth sort
// it takes its order from.  Every later kernel of the call only ORs into
// the status word, after this one.
__global__ void bin_start_kernel(const uint32_t *__restrict__ stats,
                                 const uint32_t *__restrict__ order_stats,
                                 unsigned long long *__restrict__ counts, uint64_t cap,
                                 uint4 *__restrict__ zero16, uint64_t n16,
                                 uint32_t *__restrict__ ranges, uint64_t n_ranges) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = t; i < n16; i += stride) zero16[i] = make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t i = t; i < n_ranges; i += stride) ranges[i] = 0u;
    if (t == 0) {
        const unsigned long long d = *reinterpret_cast<const unsigned long long *>(stats + kStatDup);
        unsigned long long st = stats[kStatStatus];
        if (order_stats) st |= order_stats[kStatStatus];  // the shared depth sort's waits
        if (d > cap) st |= kStatusOverflow;
        counts[kCntDup] = d;
        counts[kCntSurvivors] = stats[kStatSurvivors];
        counts[kCntStatus] = st;
        counts[3] = 0ull;
    }
}

// ------------------------------------------------------------ launcher

template <int IPT>
static int launch_pass(const PassArgs &a, uint64_t bound, cudaStream_t st) {
    int rc = ensure_smem_attr(reinterpret_cast<const void *>(onesweep_pass<IPT>),
                              SortCfg<IPT>::kSmem);
    if (rc) return rc;
    const int64_t parts = (int64_t)((bound + SortCfg<IPT>::kPart - 1) / SortCfg<IPT>::kPart);
    const int per_sm = a.ctas_per_sm > 0 ? a.ctas_per_sm
                       : bound <= kSmallPassItems ? kSmallPassCtasPerSm : kLargePassCtasPerSm;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(parts, (int64_t)num_sms() * per_sm));
    onesweep_pass<IPT><<<grid, kSortThreads, SortCfg<IPT>::kSmem, st>>>(a);
    return MS_OK;
}

int launch_onesweep(const PassArgs &a, uint64_t bound, cudaStream_t st) {
    return bound <= kSmallPassItems ? launch_pass<kSmallIPT>(a, bound, st)
                                    : launch_pass<kLargeIPT>(a, bound, st);
}

// ------------------------------------------------------------ split

// The shared depth order restricted to each view (ms_split_order): one pass
// over the union's order in partitions of kSplitPart positions (8
// consecutive ones per thread, so a thread's items stay in order), each item
// appended to the order of every view whose bit its mask holds.  Per view,
// the partition's count is found by a block scan of per-thread counts
// (four views per 64-bit word, 16 bits each) and its offset by a decoupled
// look-back over the earlier partitions' counts (thread v for view v).
constexpr int kSplitThreads = 256;
constexpr int kSplitIPT = 8;
constexpr int kSplitPart = kSplitThreads * kSplitIPT;

struct SplitArgs {
    const uint32_t *order;   // union order (Gaussian indices)
    const uint32_t *flags;   // per Gaussian: bit v set if listed in view v
    const uint32_t *n32;     // union count (device)
    uint64_t n_max;          // length of flags and order
    int n_views;
    uint32_t *out[MS_MAX_PROJ_VIEWS];         // per-view orders
    uint32_t *view_stats[MS_MAX_PROJ_VIEWS];  // per-view count and status
    uint32_t *status;        // [partitions][MS_MAX_PROJ_VIEWS] look-back words, zeroed
    uint32_t *ticket;        // [2] zeroed: partitions taken, CTAs finished
    unsigned long long *err;  // the union's status word (the sort's waits and this pass's)
    uint32_t spin_limit;
};

__device__ __forceinline__ uint64_t block_excl_scan256_u64(uint64_t v, uint64_t *s_warp,
                                                           uint64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint64_t wpre = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kSplitThreads / 32; w++) {
        const uint64_t t = s_warp[w];
        if (w < warp) wpre += t;
        total += t;
    }
    __syncthreads();
    return wpre + x - v;
}

__global__ void __launch_bounds__(kSplitThreads) split_kernel(SplitArgs a) {
    __shared__ uint64_t s_warp[kSplitThreads / 32];
    __shared__ uint32_t s_prefix[MS_MAX_PROJ_VIEWS];
    __shared__ uint32_t s_part;
    const int tid = threadIdx.x;
    const uint32_t n = (uint32_t)umin64(*a.n32, a.n_max);
    const uint32_t parts = (n + kSplitPart - 1) / kSplitPart;
    if (blockIdx.x == 0 && tid < a.n_views && n == 0) a.view_stats[tid][kStatSurvivors] = 0u;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_part = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t p = s_part;
        if (p >= parts) break;
        uint32_t g[kSplitIPT], m[kSplitIPT];
        const uint32_t j0 = p * (uint32_t)kSplitPart + (uint32_t)tid * kSplitIPT;
#pragma unroll
        for (int r = 0; r < kSplitIPT; r++) g[r] = j0 + r < n ? a.order[j0 + r] : 0xffffffffu;
#pragma unroll
        for (int r = 0; r < kSplitIPT; r++) {
            m[r] = 0u;
            if (g[r] < a.n_max) m[r] = a.flags[g[r]];
            else if (g[r] != 0xffffffffu) {
                MS_DCHECK(false, a.err);
                atomicOr(a.err, (unsigned long long)kStatusTimeout);
            }
        }
        // per-thread counts of views 0-3 and 4-7, 16 bits each
        uint64_t c_lo = 0, c_hi = 0;
#pragma unroll
        for (int r = 0; r < kSplitIPT; r++)
#pragma unroll
            for (int v = 0; v < 4; v++) {
                c_lo += (uint64_t)((m[r] >> v) & 1u) << (16 * v);
                c_hi += (uint64_t)((m[r] >> (v + 4)) & 1u) << (16 * v);
            }
        uint64_t t_lo, t_hi;
        const uint64_t e_lo = block_excl_scan256_u64(c_lo, s_warp, t_lo);
        const uint64_t e_hi = block_excl_scan256_u64(c_hi, s_warp, t_hi);
        if (tid < a.n_views) {
            const int v = tid;
            const uint32_t local =
                (uint32_t)(((v < 4 ? t_lo : t_hi) >> (16 * (v & 3))) & 0xffffu);
            uint32_t *st = a.status + (uint64_t)p * MS_MAX_PROJ_VIEWS + v;
            uint32_t excl = 0;
            if (p == 0) {
                st_relaxed(st, kFlagPre | local);
            } else {
                st_relaxed(st, kFlagAgg | local);
                int64_t k = (int64_t)p - 1;
                uint32_t spins = 0;
                while (k >= 0) {
                    const uint32_t w = ld_relaxed(a.status + (uint64_t)k * MS_MAX_PROJ_VIEWS + v);
                    if ((w & kFlagMask) == 0) {  // not published yet: poll again
                        if (++spins > a.spin_limit) {
                            atomicOr(a.err, (unsigned long long)kStatusTimeout);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    excl += w & kValMask;
                    if (w & kFlagPre) break;
                    k--;
                }
                st_relaxed(st, kFlagPre | ((excl + local) & kValMask));
            }
            s_prefix[v] = excl;
            if (p + 1 == parts) a.view_stats[v][kStatSurvivors] = excl + local;
        }
        __syncthreads();
        // append each item to the order of every view it is listed in
        uint32_t pos[MS_MAX_PROJ_VIEWS];
#pragma unroll
        for (int v = 0; v < MS_MAX_PROJ_VIEWS; v++)
            pos[v] = (v < a.n_views ? s_prefix[v] : 0u) +
                     (uint32_t)(((v < 4 ? e_lo : e_hi) >> (16 * (v & 3))) & 0xffffu);
#pragma unroll
        for (int r = 0; r < kSplitIPT; r++) {
            const uint32_t mr = m[r];
#pragma unroll
            for (int v = 0; v < MS_MAX_PROJ_VIEWS; v++)
                if (v < a.n_views && ((mr >> v) & 1u)) {
                    const uint32_t q = pos[v]++;
                    if (q < a.n_max) a.out[v][q] = g[r];
                    else atomicOr(a.err, (unsigned long long)kStatusTimeout);
                }
        }
    }
    // the last CTA to finish copies the union's status (the sort's waits and
    // this pass's) to every view
    __shared__ bool s_last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.ticket + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && tid < a.n_views) {
        __threadfence();
        const uint32_t st = (uint32_t)ld_relaxed64(a.err);
        a.view_stats[tid][kStatStatus] = st;
        a.view_stats[tid][kStatStatus + 1] = 0u;
    }
}

// ------------------------------------------------------------ workspace

struct BinLayout {
    size_t dkeys_a, dvals_a, dkeys_b, dvals_b;
    size_t tkeys_a, tvals_a, tkeys_b, tvals_b;
    size_t zero_begin;  // everything from here to total is zeroed per call
    size_t tickets, thist, dup_status, dstatus, tstatus;
    size_t total;
    int64_t dparts, tparts, dupparts;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool layout(int64_t n, int64_t cap, BinLayout &L) {
    if (n < 0 || n > kMaxSortItems || cap < 1 || cap > kMaxSortItems) return false;
    int64_t nn = n > 0 ? n : 1;
    L.dparts = sort_parts((uint64_t)nn);
    L.tparts = sort_parts((uint64_t)cap);
    L.dupparts = ceil_div(nn, kDupPart);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.dkeys_a = take(nn * 4);
    L.dvals_a = take(nn * 4);
    L.dkeys_b = take(nn * 4);
    L.dvals_b = take(nn * 4);
    L.tkeys_a = take(cap * 4);
    L.tvals_a = take(cap * 4);
    L.tkeys_b = take(cap * 4);
    L.tvals_b = take(cap * 4);
    L.tstatus = take((size_t)2 * L.tparts * 256 * 4);  // cleared by duplicate_kernel
    L.zero_begin = o;
    L.tickets = take(16 * 4);
    L.thist = take(512 * 4);
    L.dup_status = take(L.dupparts * 8);
    L.dstatus = take((size_t)4 * L.dparts * 256 * 4);
    L.total = o;
    return true;
}

}  // namespace msgs

using namespace msgs;

extern "C" size_t ms_bin_workspace_bytes(int64_t n, int64_t tiles, int64_t dup_capacity) {
    BinLayout L;
    if (tiles < 1 || tiles > 65536 || !layout(n, dup_capacity, L)) return 0;
    return L.total;
}

namespace msgs {
namespace {

// The four stable depth passes over proj's listed Gaussians (pass 0 takes
// the items with n_tiles > 0, compacting them in index order); the depth
// order's indices end in vals_final.
int depth_passes(const ms_proj_t *proj, int64_t n, const BinLayout &L, char *w,
                 uint32_t *vals_final, unsigned long long *err, uint32_t spin_limit,
                 cudaStream_t st, int ctas_per_sm = 0) {
    auto U32 = [&](size_t off) { return reinterpret_cast<uint32_t *>(w + off); };
    uint32_t *tickets = U32(L.tickets);
    const uint32_t *survivors = proj->stats + kStatSurvivors;
    uint32_t *dk[2] = {U32(L.dkeys_a), U32(L.dkeys_b)};
    uint32_t *dv[2] = {U32(L.dvals_a), U32(L.dvals_b)};
    int rc;
    for (int pass = 0; pass < 4; pass++) {
        PassArgs a;
        a.keys_in = pass == 0 ? proj->depth : dk[(pass - 1) & 1];
        a.vals_in = pass == 0 ? nullptr : dv[(pass - 1) & 1];
        a.filter = pass == 0 ? proj->n_tiles : nullptr;
        a.keys_out = pass == 3 ? nullptr : dk[pass & 1];
        a.vals_out = pass == 3 ? vals_final : dv[pass & 1];
        a.n32 = pass == 0 ? nullptr : survivors;
        a.n64 = nullptr;
        a.n_cap = (uint64_t)n;
        a.shift = 8 * pass;
        a.hist = proj->stats + kStatHist + 256 * pass;
        a.status = U32(L.dstatus) + (size_t)pass * L.dparts * 256;
        a.ticket = tickets + pass;
        a.err = err;
        a.spin_limit = spin_limit;
        a.ctas_per_sm = ctas_per_sm;
        if ((rc = launch_onesweep(a, (uint64_t)n, st))) return rc;
    }
    return MS_OK;
}

int check_bin_args(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam, const ms_bins_t *out,
                   void *ws, size_t ws_bytes, BinLayout &L, int64_t &tiles, int &tiles_x) {
    if (!proj || !out || !cam) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
    tiles_x = (cam->width + 15) / 16;
    const int tiles_y = (cam->height + 15) / 16;
    tiles = (int64_t)tiles_x * tiles_y;
    if (tiles > 65536) return fail(MS_ERR_INVALID_ARG, "more than 65536 tiles");
    if (!layout(n, out->dup_capacity, L))
        return fail(MS_ERR_INVALID_ARG, "n or dup_capacity out of range");
    if (!ws || ws_bytes < L.total || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "workspace missing, too small or misaligned");
    if (!out->gauss_idx || !out->ranges || !out->counts || !aligned(out->counts, 8))
        return fail(MS_ERR_INVALID_ARG, "ms_bins_t has a NULL or misaligned buffer");
    if (n > 0 && (!proj->n_tiles || !proj->depth || !proj->rect || !proj->stats))
        return fail(MS_ERR_INVALID_ARG, "ms_proj_t has a NULL buffer");
    if (proj->n < n) return fail(MS_ERR_INVALID_ARG, "ms_proj_t holds fewer Gaussians than n");
    return MS_OK;
}

// ms_bin, or with `order` (a depth order of a superset of proj's listed
// Gaussians; its count and the sort's status in order_stats) the same
// without the depth passes.
int bin_impl(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam, const ms_bins_t *out,
             const uint32_t *order, const uint32_t *order_stats, void *ws, size_t ws_bytes,
             void *stream) {
    BinLayout L;
    int64_t tiles = 0;
    int tiles_x = 0;
    int rc = check_bin_args(proj, n, cam, out, ws, ws_bytes, L, tiles, tiles_x);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    char *w = static_cast<char *>(ws);
    const int sms = num_sms();
    if (n == 0) {
        if ((rc = cuda_check(cudaMemsetAsync(out->ranges, 0, (size_t)tiles * 2 * sizeof(uint32_t), st),
                             "ranges memset")))
            return rc;
        return cuda_check(cudaMemsetAsync(out->counts, 0, 4 * sizeof(uint64_t), st), "counts memset");
    }
    auto U32 = [&](size_t off) { return reinterpret_cast<uint32_t *>(w + off); };
    uint32_t *tickets = U32(L.tickets);
    unsigned long long *err = reinterpret_cast<unsigned long long *>(out->counts) + kCntStatus;
    const uint32_t spin_limit = bin_spin_limit();

    // the zeroed region starts and ends on 256-byte boundaries (layout)
    const uint64_t n16 = (L.total - L.zero_begin) / 16;
    bin_start_kernel<<<std::max(1, std::min(sms * 2, (int)ceil_div((int64_t)n16, 256))), 256, 0,
                       st>>>(proj->stats, order ? order_stats : nullptr,
                             reinterpret_cast<unsigned long long *>(out->counts),
                             (uint64_t)out->dup_capacity,
                             reinterpret_cast<uint4 *>(w + L.zero_begin), n16, out->ranges,
                             (uint64_t)tiles * 2);
    const uint32_t *survivors = proj->stats + kStatSurvivors;
    const unsigned long long *dup64 =
        reinterpret_cast<const unsigned long long *>(proj->stats + kStatDup);
    const uint32_t *order_n = order ? order_stats + kStatSurvivors : survivors;
    if (!order) {
        // ---- depth sort: 4 passes over the listed Gaussians; after them
        // (out: a, b, a, b) the depth-ordered indices are in dvals_b
        if ((rc = depth_passes(proj, n, L, w, U32(L.dvals_b), err, spin_limit, st))) return rc;
        order = U32(L.dvals_b);
    }
    // ---- duplicate into (tile, index) entries
    DupArgs da;
    da.order = order;
    da.n_tiles = proj->n_tiles;
    da.rect = reinterpret_cast<const uint2 *>(proj->rect);
    da.n32 = order_n;
    da.n_max = (uint64_t)n;
    da.tiles_x = tiles_x;
    da.tiles = (uint32_t)tiles;
    da.cap = (uint64_t)out->dup_capacity;
    da.keys_out = U32(L.tkeys_a);
    da.vals_out = U32(L.tvals_a);
    da.hist = U32(L.thist);
    da.status = reinterpret_cast<unsigned long long *>(w + L.dup_status);
    da.ticket = tickets + 4;
    da.err = err;
    da.dup = dup64;
    da.tstatus = U32(L.tstatus);
    da.tstride = (uint64_t)L.tparts * 256;
    da.tpart = (uint32_t)sort_part((uint64_t)out->dup_capacity);
    da.spin_limit = spin_limit;
    int dupgrid = (int)std::min<int64_t>(L.dupparts, (int64_t)sms * 4);
    if (order_stats) duplicate_kernel<true><<<dupgrid, kDupThreads, 0, st>>>(da);
    else duplicate_kernel<false><<<dupgrid, kDupThreads, 0, st>>>(da);
    // ---- stable sort by tile id
    const int tpasses = tiles <= 256 ? 1 : 2;
    uint32_t *final_keys = U32(L.tkeys_b);
    for (int pass = 0; pass < tpasses; pass++) {
        PassArgs a;
        a.keys_in = pass == 0 ? U32(L.tkeys_a) : U32(L.tkeys_b);
        a.vals_in = pass == 0 ? U32(L.tvals_a) : U32(L.tvals_b);
        a.filter = nullptr;
        bool last = pass == tpasses - 1;
        a.keys_out = pass == 0 ? U32(L.tkeys_b) : U32(L.tkeys_a);
        a.vals_out = last ? out->gauss_idx : U32(L.tvals_b);
        final_keys = a.keys_out;
        a.n32 = nullptr;
        a.n64 = dup64;
        a.n_cap = (uint64_t)out->dup_capacity;
        a.shift = 8 * pass;
        a.hist = U32(L.thist) + 256 * pass;
        a.status = U32(L.tstatus) + (size_t)pass * L.tparts * 256;
        a.ticket = tickets + 5 + pass;
        a.err = err;
        a.spin_limit = spin_limit;
        if ((rc = launch_onesweep(a, (uint64_t)out->dup_capacity, st))) return rc;
    }
    ranges_kernel<<<sms * 4, 256, 0, st>>>(final_keys, dup64, (uint64_t)out->dup_capacity,
                                           (uint32_t)tiles, out->ranges);
    return cuda_check(cudaGetLastError(), "ms_bin launches");
}

}  // namespace
}  // namespace msgs

extern "C" int ms_bin(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
                      const ms_bins_t *out, void *ws, size_t ws_bytes, void *stream) {
    return bin_impl(proj, n, cam, out, nullptr, nullptr, ws, ws_bytes, stream);
}

extern "C" int ms_bin_ordered(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
                              const ms_bins_t *out, const uint32_t *order,
                              const uint32_t *order_stats, void *ws, size_t ws_bytes,
                              void *stream) {
    if (!order || !order_stats) return fail(MS_ERR_INVALID_ARG, "order / order_stats is NULL");
    return bin_impl(proj, n, cam, out, order, order_stats, ws, ws_bytes, stream);
}

extern "C" size_t ms_sort_depth_workspace_bytes(int64_t n) {
    BinLayout L;
    if (!layout(n, 1, L)) return 0;
    return L.total;
}

extern "C" int ms_sort_depth(const ms_proj_t *proj, int64_t n, uint32_t *order, void *ws,
                             size_t ws_bytes, void *stream) {
    BinLayout L;
    if (!proj || !order) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!layout(n, 1, L)) return fail(MS_ERR_INVALID_ARG, "n out of range");
    if (!ws || ws_bytes < L.total || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "workspace missing, too small or misaligned");
    if (n > 0 && (!proj->n_tiles || !proj->depth || !proj->stats))
        return fail(MS_ERR_INVALID_ARG, "ms_proj_t has a NULL buffer");
    if (proj->n < n) return fail(MS_ERR_INVALID_ARG, "ms_proj_t holds fewer Gaussians than n");
    if (n == 0) return MS_OK;
    cudaStream_t st = as_stream(stream);
    char *w = static_cast<char *>(ws);
    int rc;
    if ((rc = cuda_check(cudaMemsetAsync(w + L.zero_begin, 0, L.total - L.zero_begin, st),
                         "workspace memset")))
        return rc;
    // a wait that gives up is recorded in the sorted projection's status
    // word (stats words 4-5), where ms_bin_ordered picks it up
    unsigned long long *err = reinterpret_cast<unsigned long long *>(proj->stats + kStatStatus);
    // the shared sort runs ahead of every frame that takes its order: its
    // passes take every CTA the SMs hold (a frame's own sort leaves room for
    // the frames sorting beside it)
    if ((rc = depth_passes(proj, n, L, w, order, err, bin_spin_limit(), st, kLargePassCtasPerSm)))
        return rc;
    return cuda_check(cudaGetLastError(), "ms_sort_depth launches");
}

extern "C" size_t ms_split_order_workspace_bytes(int64_t n) {
    if (n < 0 || n > kMaxSortItems) return 0;
    const int64_t parts = ceil_div(n > 0 ? n : 1, (int64_t)kSplitPart);
    return 256 + (size_t)parts * MS_MAX_PROJ_VIEWS * 4;
}

extern "C" int ms_split_order(const ms_proj_t *union_proj, int64_t n, const uint32_t *order,
                              int32_t n_views, uint32_t *const *orders,
                              uint32_t *const *view_stats, void *ws, size_t ws_bytes,
                              void *stream) {
    if (!union_proj || !order || !orders || !view_stats)
        return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (n_views < 1 || n_views > MS_MAX_PROJ_VIEWS)
        return fail(MS_ERR_INVALID_ARG, "n_views must be 1..MS_MAX_PROJ_VIEWS");
    if (n < 0 || n > kMaxSortItems) return fail(MS_ERR_INVALID_ARG, "n out of range");
    const size_t need = ms_split_order_workspace_bytes(n);
    if (!ws || ws_bytes < need || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "workspace missing, too small or misaligned");
    if (!union_proj->n_tiles || !union_proj->stats || !aligned(union_proj->stats, 16))
        return fail(MS_ERR_INVALID_ARG, "union flags / stats NULL or stats misaligned");
    if (union_proj->n < n) return fail(MS_ERR_INVALID_ARG, "the union holds fewer Gaussians than n");
    SplitArgs a;
    for (int v = 0; v < MS_MAX_PROJ_VIEWS; v++) {
        a.out[v] = nullptr;
        a.view_stats[v] = nullptr;
    }
    for (int v = 0; v < n_views; v++) {
        if (!orders[v] || !view_stats[v] || !aligned(view_stats[v], 16))
            return fail(MS_ERR_INVALID_ARG, "orders[v] / view_stats[v] NULL or stats misaligned");
        a.out[v] = orders[v];
        a.view_stats[v] = view_stats[v];
    }
    cudaStream_t st = as_stream(stream);
    int rc;
    if ((rc = cuda_check(cudaMemsetAsync(ws, 0, need, st), "split workspace memset"))) return rc;
    char *w = static_cast<char *>(ws);
    a.order = order;
    a.flags = union_proj->n_tiles;
    a.n32 = union_proj->stats + kStatSurvivors;
    a.n_max = (uint64_t)n;
    a.n_views = n_views;
    a.ticket = reinterpret_cast<uint32_t *>(w);
    a.status = reinterpret_cast<uint32_t *>(w + 256);
    a.err = reinterpret_cast<unsigned long long *>(union_proj->stats + kStatStatus);
    a.spin_limit = bin_spin_limit();
    const int64_t parts = ceil_div(n > 0 ? n : 1, (int64_t)kSplitPart);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(parts, (int64_t)num_sms() * 4));
    split_kernel<<<grid, kSplitThreads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "split_kernel launch");
}

extern "C" int ms_bin_counts(const ms_bins_t *bins, int64_t *d_needed, int64_t *survivors,
                             void *stream) {
    if (!bins || !bins->counts) return fail(MS_ERR_INVALID_ARG, "NULL bins");
    uint64_t h[4];
    cudaStream_t st = as_stream(stream);
    int rc;
    if ((rc = cuda_check(cudaMemcpyAsync(h, bins->counts, sizeof(h), cudaMemcpyDeviceToHost, st),
                         "counts copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(st), "stream sync"))) return rc;
    if (d_needed) *d_needed = (int64_t)h[kCntDup];
    if (survivors) *survivors = (int64_t)h[kCntSurvivors];
    if (h[kCntStatus] & kStatusBounds)
        return fail(MS_ERR_BOUNDS, "an index check of the debug build failed");
    if (h[kCntStatus] & kStatusTimeout)
        return fail(MS_ERR_TIMEOUT, "a bounded device wait gave up during ms_bin");
    if (h[kCntStatus] & kStatusOverflow)
        return fail(MS_ERR_CAPACITY, "tile duplicates exceed dup_capacity");
    return MS_OK;
}

// ------------------------------------------------ binning without allocation
//
// For callers that cannot allocate device memory: an engine plugin whose
// host application owns every device allocation, a render loop that runs
// under a fixed memory budget or a no-allocation rule on its frame thread,
// or a runtime that hands the library only the buffers it must fill.  They
// still pass the projection and the output buffers; the scratch space of the
// binning lives in this library's own static device array.

namespace msgs {

constexpr size_t kStaticScratchBytes = 16u << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_bin_scratch[kStaticScratchBytes];

}  // namespace msgs

extern "C" int ms_bin_noalloc(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
                              const ms_bins_t *out, void *stream) {
    // one cached device address per device; host threads making a first
    // call at once store the same value, so an atomic is all that is needed
    static std::atomic<void *> addr[64];
    if (!cam || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
    const int64_t tiles = (int64_t)((cam->width + 15) / 16) * ((cam->height + 15) / 16);
    const size_t need = ms_bin_workspace_bytes(n, tiles, out->dup_capacity);
    if (need == 0) return fail(MS_ERR_INVALID_ARG, "n, tiles or dup_capacity out of range");
    if (need > kStaticScratchBytes)
        return fail(MS_ERR_INVALID_ARG,
                    "ms_bin_noalloc: n / tiles / dup_capacity need " + std::to_string(need) +
                        " bytes of scratch, more than the static " +
                        std::to_string(kStaticScratchBytes) + " (use ms_bin with a workspace)");
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return fail(MS_ERR_INVALID_ARG, "device index beyond 63");
    void *p = addr[dev].load(std::memory_order_acquire);
    if (!p) {
        // first call on this device: the array's device address (the host
        // symbol is only a stand-in and must never reach a kernel)
        if ((rc = cuda_check(cudaGetSymbolAddress(&p, g_bin_scratch), "cudaGetSymbolAddress")))
            return rc;
        addr[dev].store(p, std::memory_order_release);
    }
    return ms_bin(proj, n, cam, out, p, kStaticScratchBytes, stream);
}
