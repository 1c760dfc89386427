// Device-wide primitives: a single-pass exclusive scan and a stable LSD radix
// sort, both with decoupled look-back (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016; Adinets & Merrill, "Onesweep",
// 2022).  Logical block ids come from an atomic ticket, so a block only ever
// waits on blocks that started before it.  Every wait is bounded (LookBack's
// spin_limit, by default kSpinLimit); running out records VPGS_ERR_TIMEOUT and
// the kernel carries on with a partial prefix, whose scatter positions are
// still bounds-checked.
#pragma once

#include "common.cuh"
#include "profiler.h"

namespace vpgs {

VPGS_D unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
VPGS_D void st_volatile_u64(unsigned long long *p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}
VPGS_D uint32_t ld_volatile_u32(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
VPGS_D void st_volatile_u32(uint32_t *p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}
VPGS_D uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// exclusive scan of n uint32 values: out prefix handed to a store functor
//   Load:  __device__ uint32_t operator()(int64_t i) const         (i < n)
//   Store: __device__ void operator()(int64_t i, uint32_t excl, uint32_t v) const
// The scan total is written to *total (when total != nullptr).
// n = min(n_cap, *n_dev) if n_dev else n_cap.
// Status word layout (64 bit): [63:62] flag 1 = aggregate, 2 = inclusive prefix.
// ---------------------------------------------------------------------------
// How a look-back kernel waits: polls before it gives up (VPGS_ERR_TIMEOUT), and
// whether it returns at entry when the status word already holds an error (the
// render's binning chain, whose later kernels index with earlier outputs).
struct LookBack {
    int spin_limit = kSpinLimit;
    bool stop_on_error = false;
};

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

template <class Load, class Store, int ITEMS>
__global__ void __launch_bounds__(kScanThreads)
scan_kernel(Load load, Store store, int64_t n_cap, const uint32_t *n_dev, uint32_t *ticket,
            unsigned long long *look, uint32_t *total, uint32_t *status, LookBack lb) {
    constexpr int kTile = kScanThreads * ITEMS;
    grid_dep_enter();
    if (lb.stop_on_error && *status != 0u) return;
    __shared__ uint32_t s_items[kTile + kTile / 32];
    __shared__ uint32_t s_warp[kScanThreads / kWarp];
    __shared__ uint32_t s_bid, s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t n = n_cap;
    if (n_dev) n = min(n, (int64_t)*n_dev);
    // tiles in ticket order until they run out (the grid is sized to what fits
    // on the GPU at once, not to the capacity)
    for (;;) {
    if (tid == 0) s_bid = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t bid = s_bid;
    const int64_t base = bid * kTile;
    if (base >= n) {
        if (bid == 0 && tid == 0 && total) *total = 0;
        return;
    }
    // striped, coalesced loads into a padded shared tile
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int idx = j * kScanThreads + tid;
        int64_t gi = base + idx;
        s_items[idx + (idx >> 5)] = gi < n ? load(gi) : 0u;
    }
    __syncthreads();
    // blocked: thread t owns items t*ITEMS .. t*ITEMS+ITEMS-1
    uint32_t v[ITEMS];
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int idx = tid * ITEMS + i;
        v[i] = s_items[idx + (idx >> 5)];
        tsum += v[i];
    }
    // block exclusive scan of the thread sums
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / kWarp ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / kWarp) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t block_agg = s_warp[kScanThreads / kWarp - 1];
    uint32_t texcl = x - tsum + (warp > 0 ? s_warp[warp - 1] : 0u);
    // decoupled look-back, one warp: 32 predecessors per step
    if (warp == 0) {
        unsigned long long excl = 0;
        if (bid == 0) {
            if (lane == 0) st_volatile_u64(look, kFlagPre | block_agg);
        } else {
            if (lane == 0) st_volatile_u64(look + bid, kFlagAgg | block_agg);
            int64_t j0 = bid - 1;
            for (;;) {
                const int64_t j = j0 - lane;
                unsigned long long w = j >= 0 ? ld_volatile_u64(look + j) : kFlagPre;
                int spins = 0;
                bool timed_out = false;
                while (!__all_sync(0xffffffffu, (w >> 62) != 0)) {
                    if (++spins > lb.spin_limit) {
                        timed_out = true;
                        break;
                    }
                    __nanosleep(64);
                    if ((w >> 62) == 0) w = ld_volatile_u64(look + j);
                }
                if (timed_out) {
                    if (lane == 0) set_status(status, VPGS_ERR_TIMEOUT);
                    break;
                }
                const uint32_t pre = __ballot_sync(0xffffffffu, (w >> 62) == 2);
                const int last = pre ? __ffs(pre) - 1 : 31;  // nearest inclusive prefix
                unsigned long long v = lane <= last ? (w & kValMask) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                excl += v;
                if (pre) break;
                j0 -= 32;
            }
            if (lane == 0) st_volatile_u64(look + bid, kFlagPre | (excl + block_agg));
        }
        if (lane == 0) {
            s_excl = (uint32_t)excl;
            if (base + kTile >= n && total) *total = (uint32_t)excl + block_agg;
        }
    }
    __syncthreads();
    uint32_t run = s_excl + texcl;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int64_t gi = base + (int64_t)tid * ITEMS + i;
        if (gi < n) store(gi, run, v[i]);
        run += v[i];
    }
    __syncthreads();  // the next tile reuses the shared arrays
    }
}

// Blocks of a kernel that fit on the current GPU at once.
inline int resident_grid(const void *kernel, int threads, size_t smem, int64_t cap_blocks) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) occ = 1;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t g = (int64_t)occ * std::max(sms, 1);
    return (int)std::max<int64_t>(1, std::min(g, cap_blocks));
}

inline int64_t scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// A ticket-loop grid: what is resident, or at most per_sm blocks per SM (per_sm
// > 0; for passes whose item count is usually far below its capacity, where
// blocks past the last tile only launch, take a ticket and leave).
int device_sm_count();
inline int grid_cap(int resident, int per_sm) {
    return per_sm > 0 ? std::max(1, std::min(resident, per_sm * device_sm_count())) : resident;
}

template <class Load, class Store, int ITEMS>
cudaError_t launch_scan_as(const char *name, Load load, Store store, int64_t n_cap, const uint32_t *n_dev,
                           uint32_t *ticket, unsigned long long *look, uint32_t *total, uint32_t *status,
                           cudaStream_t stream, LookBack lb, int per_sm) {
    const int64_t tile = (int64_t)kScanThreads * ITEMS;
    int64_t nb = (n_cap + tile - 1) / tile;
    if (nb == 0) nb = 1;
    static std::atomic<int> grid_cache[kDeviceCache];  // per <Load, Store, ITEMS> and device
    const int grid_res = per_device(grid_cache, [] {
        return resident_grid((const void *)scan_kernel<Load, Store, ITEMS>, kScanThreads, 0, int64_t(1) << 30);
    });
    const int grid = (int)std::min<int64_t>(grid_cap(grid_res, per_sm), nb);
    VPGS_LAUNCH(name, stream,
                launch_k(scan_kernel<Load, Store, ITEMS>, (unsigned)grid, kScanThreads, 0, stream, load, store, n_cap,
                         n_dev, ticket, look, total, status, lb));
    return cudaGetLastError();
}

// Launch a scan over at most n_cap items.  *ticket and the scan_blocks(n_cap)
// look-back words must be zero on entry (the render's prepare kernel clears them).
// wide: tiles of kScanItemsWide items per thread (fewer tiles in the look-back
// chain, for scans of many millions of items) instead of kScanItems.
template <class Load, class Store>
cudaError_t launch_scan(const char *name, Load load, Store store, int64_t n_cap, const uint32_t *n_dev,
                        uint32_t *ticket, unsigned long long *look, uint32_t *total,
                        uint32_t *status, cudaStream_t stream, LookBack lb = LookBack{}, int per_sm = 0,
                        bool wide = false) {
    if (wide)
        return launch_scan_as<Load, Store, kScanItemsWide>(name, load, store, n_cap, n_dev, ticket, look, total,
                                                           status, stream, lb, per_sm);
    return launch_scan_as<Load, Store, kScanItems>(name, load, store, n_cap, n_dev, ticket, look, total, status,
                                                   stream, lb, per_sm);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value) pairs.
// One kernel computes the global histograms of every pass; then one kernel per
// pass ranks and scatters ("one sweep") with per-digit decoupled look-back.
// ---------------------------------------------------------------------------
struct SortPass {
    int shift, bits;
};

// Lanes of the warp holding the same digit: one ballot per digit bit (a lane
// keeps the lanes that agree with it on every bit), which is cheaper than the
// hardware match for digits of up to 8 bits.  Items past the end (valid =
// false) match only themselves.
VPGS_D uint32_t match_digit(uint32_t d, bool valid, int bits, int lane) {
    uint32_t m = __ballot_sync(0xffffffffu, valid);
    if (!valid) m = 1u << lane;
    for (int b = 0; b < bits; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit != 0u);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// predecessor tiles read per look-back step of a one-sweep pass
#ifndef VPGS_LOOK_DEPTH
#define VPGS_LOOK_DEPTH 16
#endif

// one-sweep look-back word: [31:30] flag (1 = block aggregate, 2 = inclusive
// prefix), [29:0] count
constexpr uint32_t kSFlagAgg = 1u << 30;
constexpr uint32_t kSFlagPre = 2u << 30;
constexpr uint32_t kSValMask = (1u << 30) - 1u;

template <int ITEMS>
static __global__ void __launch_bounds__(kSortThreads)
radix_onesweep_kernel(const uint32_t *__restrict__ key_in, const uint32_t *__restrict__ val_in,
                      uint32_t *__restrict__ key_out, uint32_t *__restrict__ val_out,
                      int64_t n_cap, const uint32_t *n_dev, SortPass pass,
                      const uint32_t *__restrict__ pass_hist, uint32_t *ticket, uint32_t *look,
                      uint32_t *next_look, uint32_t *status, LookBack lb) {
    grid_dep_enter();
    if (lb.stop_on_error && *status != 0u) return;
    constexpr int kWarps = kSortThreads / kWarp;
    constexpr int kSeg = kWarp * ITEMS;  // contiguous items per warp
    constexpr int kTile = kSortThreads * ITEMS;
    static_assert(kSortThreads == kRadix, "one thread per digit");
    __shared__ uint32_t s_cnt[kWarps][kRadix];
    __shared__ uint32_t s_glob[kRadix];
    __shared__ uint32_t s_dstart[kRadix], s_gbase[kRadix], s_wsum[kWarps];
    __shared__ uint32_t s_key[kTile], s_val[kTile];
    __shared__ uint32_t s_bid;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t n = n_cap;
    if (n_dev) n = min(n, (int64_t)*n_dev);
    if (n == 0) return;
    const uint32_t mask = (1u << pass.bits) - 1u;

    // global exclusive digit offsets of this pass (every block recomputes them)
    if (tid < kRadix) {
        // 256 threads: inclusive scan via shared memory in two levels of warps
        uint32_t h = pass_hist[tid];
        uint32_t x = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        s_glob[tid] = x;  // inclusive within warp
    }
    __syncthreads();
    uint32_t glob_excl = 0;
    if (tid < kRadix) {
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += s_glob[w * 32 + 31];
        glob_excl = s_glob[tid] - pass_hist[tid] + add;
    }

    // tiles in ticket order until they run out (the grid is sized to what fits
    // on the GPU at once; a tile only waits on lower tickets, held by running blocks)
    for (;;) {
    if (tid == 0) s_bid = atomicAdd(ticket, 1u);
    for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t bid = s_bid;
    const int64_t base = bid * (int64_t)(kSortThreads * ITEMS);
    if (base >= n) return;

    // load this warp's contiguous segment, 32 consecutive keys per step
    uint32_t k[ITEMS], v[ITEMS], d[ITEMS];
    const int64_t seg = base + (int64_t)warp * kSeg;
#pragma unroll
    for (int s = 0; s < ITEMS; ++s) {
        int64_t i = seg + s * kWarp + lane;
        bool ok = i < n;
        k[s] = ok ? key_in[i] : 0u;
        v[s] = ok ? val_in[i] : 0u;
        d[s] = ok ? ((k[s] >> pass.shift) & mask) : (kRadix + lane);  // sentinel never matches
    }
    // per-warp digit counts
#pragma unroll
    for (int s = 0; s < ITEMS; ++s) {
        const uint32_t m = match_digit(d[s], d[s] < kRadix, pass.bits, lane);
        if (d[s] < kRadix && (m & lanemask_lt()) == 0) s_cnt[warp][d[s]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    // block count per digit and its block-local exclusive start (kRadix == threads)
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) c += s_cnt[w][tid];
    {
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += s_wsum[w];
        s_dstart[tid] = x - c + add;
    }
    // publish, look back over earlier blocks
    {
        uint32_t excl = 0;
        uint32_t *my = look + bid * kRadix + tid;
        if (bid == 0) {
            st_volatile_u32(my, kSFlagPre | c);
        } else {
            st_volatile_u32(my, kSFlagAgg | c);
            // kLookDepth independent loads per step shorten the dependent chain
            constexpr int kLookDepth = VPGS_LOOK_DEPTH;
            int64_t j0 = bid - 1;
            bool done = false;
            while (!done) {
                uint32_t w[kLookDepth];
#pragma unroll
                for (int i = 0; i < kLookDepth; ++i) {
                    const int64_t j = j0 - i;
                    w[i] = j >= 0 ? ld_volatile_u32(look + j * kRadix + tid) : kSFlagPre;
                }
#pragma unroll
                for (int i = 0; i < kLookDepth; ++i) {
                    if (done) break;
                    const int64_t j = j0 - i;
                    uint32_t x = w[i];
                    int spins = 0;
                    while ((x >> 30) == 0) {
                        if (++spins > lb.spin_limit) {
                            set_status(status, VPGS_ERR_TIMEOUT);
                            x = kSFlagPre;
                            break;
                        }
                        __nanosleep(32);
                        x = ld_volatile_u32(look + j * kRadix + tid);
                    }
                    excl += x & kSValMask;
                    if ((x >> 30) == 2) done = true;
                }
                j0 -= kLookDepth;
            }
            st_volatile_u32(my, kSFlagPre | (excl + c));
        }
        s_gbase[tid] = glob_excl + excl;  // global slot of this block's first key with digit tid
        // per-warp bases inside the block (block-local digit order)
        uint32_t run = s_dstart[tid];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = s_cnt[w][tid];
            s_cnt[w][tid] = run;
            run += t;
        }
    }
    __syncthreads();
    // stable ranking into shared memory: order inside a step by lane, steps in
    // order, warps in order
#pragma unroll
    for (int s = 0; s < ITEMS; ++s) {
        const uint32_t m = match_digit(d[s], d[s] < kRadix, pass.bits, lane);
        const uint32_t rank = __popc(m & lanemask_lt());
        if (d[s] < kRadix) {
            const uint32_t lp = s_cnt[warp][d[s]] + rank;
            s_key[lp] = k[s];
            s_val[lp] = v[s];
        }
        __syncwarp();
        if (d[s] < kRadix && rank == 0) s_cnt[warp][d[s]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    // coalesced write-out: consecutive threads write consecutive slots of each digit run
    const int nb = (int)min((int64_t)kTile, n - base);
    for (int i = tid; i < nb; i += kSortThreads) {
        const uint32_t key = s_key[i];
        const uint32_t dg = (key >> pass.shift) & mask;
        const uint32_t pos = s_gbase[dg] + ((uint32_t)i - s_dstart[dg]);
        if ((int64_t)pos < n) {  // always true unless a look-back wait timed out
            key_out[pos] = key;
            val_out[pos] = s_val[i];
        }
    }
    if (next_look) next_look[bid * kRadix + tid] = 0u;  // the next pass starts from zero
    __syncthreads();  // the next tile reuses the shared arrays
    }
}

// Split `bits` low key bits starting at `lo` into balanced passes of <= 8 bits.
inline int plan_passes(int lo, int bits, SortPass *out) {
    int np = (bits + kRadixBits - 1) / kRadixBits;
    if (np == 0) return 0;
    int base = bits / np, extra = bits % np, s = lo;
    for (int p = 0; p < np; ++p) {
        int b = base + (p < extra ? 1 : 0);
        out[p] = {s, b};
        s += b;
    }
    return np;
}

inline int64_t sort_blocks(int64_t n, int items) {
    const int64_t tile = (int64_t)kSortThreads * items;
    return (n + tile - 1) / tile;
}

// Sort n (<= n_cap, or *n_dev) pairs from (k0, v0) using (k1, v1) as the other
// buffer.  Returns in *result_in_1 whether the sorted data ended in buffer 1.
// On entry (the producers of the keys and the render's prepare kernel see to it):
//   hist   [passes][256] global digit histograms of the n keys;
//   ticket [passes] zero;
//   look   [passes][sort_blocks(n_cap)][256], pass 0's words zero for the tiles
//          that hold keys (each pass clears the next pass's words of its tiles).
inline cudaError_t radix_sort_pairs(const char *name, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                                    int64_t n_cap, const uint32_t *n_dev, int lo_bit, int bits,
                                    const uint32_t *hist, uint32_t *ticket, uint32_t *look,
                                    uint32_t *status, cudaStream_t stream, bool *result_in_1, int items,
                                    LookBack lb = LookBack{}, int per_sm = 0) {
    SortPass ps[kMaxSortPasses];
    int np = plan_passes(lo_bit, bits, ps);
    *result_in_1 = (np & 1) != 0;
    if (np == 0 || n_cap == 0) return cudaSuccess;
    if (np > 4) return cudaErrorInvalidValue;
    if (items != 4 && items != 8 && items != 16 && items != 32) return cudaErrorInvalidValue;
    const int64_t nb = sort_blocks(n_cap, items);
    const void *kern = items == 4 ? (const void *)radix_onesweep_kernel<4>
                     : items == 8 ? (const void *)radix_onesweep_kernel<8>
                     : items == 32 ? (const void *)radix_onesweep_kernel<32>
                                   : (const void *)radix_onesweep_kernel<16>;
    static std::atomic<int> grids[4][kDeviceCache];  // by items (4, 8, 16, 32) and device
    const int gi = items == 4 ? 0 : items == 8 ? 1 : items == 16 ? 2 : 3;
    const int grid_res = per_device(grids[gi], [kern] { return resident_grid(kern, kSortThreads, 0, int64_t(1) << 30); });
    const unsigned grid = (unsigned)std::min<int64_t>(grid_cap(grid_res, per_sm), nb);
    cudaError_t e;
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int p = 0; p < np; ++p) {
        uint32_t *lk = look + (size_t)p * nb * kRadix;
        uint32_t *nl = p + 1 < np ? lk + (size_t)nb * kRadix : nullptr;
        const uint32_t *h = hist + p * kRadix;
        if (items == 4)
            VPGS_LAUNCH(name, stream, launch_k(radix_onesweep_kernel<4>, grid, kSortThreads, 0, stream,
                                          ki, vi, ko, vo, n_cap, n_dev, ps[p], h, ticket + p, lk, nl, status, lb));
        else if (items == 8)
            VPGS_LAUNCH(name, stream, launch_k(radix_onesweep_kernel<8>, grid, kSortThreads, 0, stream,
                                          ki, vi, ko, vo, n_cap, n_dev, ps[p], h, ticket + p, lk, nl, status, lb));
        else if (items == 32)
            VPGS_LAUNCH(name, stream, launch_k(radix_onesweep_kernel<32>, grid, kSortThreads, 0, stream,
                                          ki, vi, ko, vo, n_cap, n_dev, ps[p], h, ticket + p, lk, nl, status, lb));
        else
            VPGS_LAUNCH(name, stream, launch_k(radix_onesweep_kernel<16>, grid, kSortThreads, 0, stream,
                                          ki, vi, ko, vo, n_cap, n_dev, ps[p], h, ticket + p, lk, nl, status, lb));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t *tk = ki, *tv = vi;
        ki = ko; vi = vo; ko = tk; vo = tv;
    }
    return cudaSuccess;
}

// Adds the digits of key k to block-shared histograms of every pass (s_h [passes][256]).
VPGS_D void add_digits(uint32_t (*s_h)[kRadix], const SortPass *ps, int np, uint32_t k) {
    for (int p = 0; p < np; ++p) atomicAdd(&s_h[p][(k >> ps[p].shift) & ((1u << ps[p].bits) - 1u)], 1u);
}

// Adds block-shared histograms into the global ones (non-zero bins only).
VPGS_D void flush_digits(const uint32_t (*s_h)[kRadix], int np, uint32_t *hist) {
    for (int i = threadIdx.x; i < np * kRadix; i += blockDim.x) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

}  // namespace vpgs
