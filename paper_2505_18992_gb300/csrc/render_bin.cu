// Tile binning: which Gaussians touch which tile, in depth order.
//
//   1. scan of the visibility flags (tile count > 0) -> compacted (z bits, id)
//   2. stable radix sort of the visible pairs by the FP32 bit pattern of the
//      camera depth (positive floats order like their bits); ties keep index
//      order, i.e. (view, Gaussian) order
//   3. scan of the tile counts in depth order, then a block-cooperative emit
//      of each Gaussian's (global tile id, id) instances at its offset; the
//      tiles are those of the row-wise tile cover counted by the projection
//   4. stable radix sort of the instances by global tile id (only the bits a
//      tile id needs); instances stay in depth order inside each tile
//   5. [start, end) of every tile from the sorted keys
//   6. the compositing launch order: tiles by descending instance count
//
// Sorting the visible Gaussians once by depth and then the instances by tile
// id only moves 32-bit depth keys over N_visible items and a 12-14 bit tile key
// over the instances, instead of a 44+ bit (tile, depth) key over all instances.
#include "internal.h"
#include "prims.cuh"
#include "profiler.h"

namespace vpgs {

struct VisLoad {
    const uint32_t *tcount;
    __device__ uint32_t operator()(int64_t i) const { return tcount[i] > 0u ? 1u : 0u; }
};

struct VisStore {
    const Rec *rec;
    uint32_t *dkey, *dval, *vis_idx;
    int64_t cap;
    __device__ void operator()(int64_t i, uint32_t pos, uint32_t v) const {
        if (v && (int64_t)pos < cap) {
            dkey[pos] = __float_as_uint(rec[i].r2.y);  // camera z > near_z > 0
            dval[pos] = (uint32_t)i;
            vis_idx[pos] = (uint32_t)i;  // kept in index order (the sort reuses dval)
        }
    }
};

struct CountLoad {
    const uint32_t *tcount, *dval;
    __device__ uint32_t operator()(int64_t r) const { return tcount[dval[r]]; }
};

struct OffsetStore {
    uint32_t *inst_off;
    __device__ void operator()(int64_t r, uint32_t off, uint32_t) const { inst_off[r] = off; }
};

// Emits the (global tile id, record) instances of 256 consecutive depth-ranked
// Gaussians per block.  The instances of Gaussians spanning at most kCoverRows
// tile rows are spread evenly over the block's threads; each finds its Gaussian
// by binary search over the block's local offsets, so a Gaussian covering many
// tiles does not serialise, and then its tile from the row spans the counting
// pass stored.  A Gaussian spanning more rows takes one warp: one row per lane,
// its span from the same row-span function that counted it, a warp prefix of
// the rows' counts, and each lane writing its row's run of tiles.
constexpr int kEmitThreads = 256;

// 6 blocks per SM (40 registers): the instance loop is latency-bound and wants them
__global__ void __launch_bounds__(kEmitThreads, 6)
emit_kernel(const uint32_t *__restrict__ dval, const uint32_t *__restrict__ inst_off,
            const BinRec *__restrict__ bin, const uint32_t *n_vis, const uint32_t *n_inst, int64_t N,
            int64_t M_cap, CamParams cam, uint32_t *__restrict__ ikey, uint32_t *__restrict__ ival,
            uint32_t *status, int n_pass, SortPass p0, SortPass p1, SortPass p2, SortPass p3,
            uint32_t *hist, uint32_t *look0) {
    grid_dep_enter();
    if (*status != 0u) return;  // an earlier kernel failed: dval may hold stale entries
    {
        // the tile sort's first-pass look-back words, for the tiles that will hold
        // instances (the instance count is known from here on)
        const int64_t ni = min((int64_t)*n_inst, M_cap);
        const int64_t tile = (int64_t)kSortThreads * kTileSortItems;
        const int64_t nw = (ni + tile - 1) / tile * kRadix;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x)
            look0[i] = 0u;
    }
    // digit histograms of the emitted tile ids, for the tile sort
    __shared__ uint32_t s_h[4][kRadix];
    const SortPass tps[4] = {p0, p1, p2, p3};
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0u;
    __shared__ uint32_t s_start[kEmitThreads], s_id[kEmitThreads], s_vb[kEmitThreads];
    __shared__ uint32_t s_sstart[kEmitThreads];  // starts counting only the small Gaussians' instances
    __shared__ uint16_t s_large[kEmitThreads];   // chunk positions of the large Gaussians
    __shared__ uint32_t s_wsum[kEmitThreads / 32][2];
    __shared__ uint2 s_rect[kEmitThreads];
    __shared__ float4 s_uv[kEmitThreads];
    __shared__ Cover s_cv[kEmitThreads];
    __shared__ uint32_t s_total, s_small, s_nlarge;
    const int64_t nv = *n_vis;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bool overflow = false;
    // chunks of kEmitThreads depth-ranked Gaussians, grid-strided (the grid is
    // sized to what fits on the GPU, not to the capacity)
    for (int64_t r0 = (int64_t)blockIdx.x * kEmitThreads; r0 < nv && !overflow;
         r0 += (int64_t)gridDim.x * kEmitThreads) {
    const int nb = (int)min((int64_t)kEmitThreads, nv - r0);
    const uint32_t base = inst_off[r0];
    if (tid < nb) {
        const int64_t r = r0 + tid;
        const uint32_t id = dval[r];
        const BinRec br = bin[id];
        s_start[tid] = inst_off[r] - base;
        s_id[tid] = id;
        s_rect[tid] = br.rect;
        s_uv[tid] = br.uv;
        s_cv[tid] = br.cv;
        s_vb[tid] = (uint32_t)(id / N) * (uint32_t)cam.T;
        // the block's end offset: the next block's start, or the total
        if (tid == nb - 1) s_total = (r0 + nb < nv ? inst_off[r0 + nb] : *n_inst) - base;
    }
    __syncthreads();
    const uint32_t total = s_total;
    if ((int64_t)base + total > M_cap) {
        if (tid == 0) set_status(status, VPGS_ERR_CAPACITY);
        overflow = true;  // block-uniform
        continue;
    }
    // Gaussians spanning more than kCoverRows tile rows are emitted row-parallel
    // below; the instance loop covers the others, through a prefix of their counts
    // (the chunk's own offsets when it has no large Gaussian, the common case)
    bool large = false;
    uint32_t cnt = 0u;
    if (tid < nb) {
        const uint2 rc = s_rect[tid];
        large = (int)(rc.y >> 16) - (int)(rc.y & 0xffffu) + 1 > kCoverRows;
        cnt = (tid + 1 < nb ? s_start[tid + 1] : total) - s_start[tid];
    }
    const bool any_large = __syncthreads_or(large) != 0;
    if (any_large) {
        uint32_t xs = large ? 0u : cnt, xl = large ? 1u : 0u;  // inclusive scans
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ys = __shfl_up_sync(0xffffffffu, xs, o), yl = __shfl_up_sync(0xffffffffu, xl, o);
            if (lane >= o) {
                xs += ys;
                xl += yl;
            }
        }
        if (lane == 31) {
            s_wsum[warp][0] = xs;
            s_wsum[warp][1] = xl;
        }
        __syncthreads();
        uint32_t ps = 0u, pl = 0u, ts = 0u, tl = 0u;
#pragma unroll
        for (int w = 0; w < kEmitThreads / 32; ++w) {
            if (w < warp) {
                ps += s_wsum[w][0];
                pl += s_wsum[w][1];
            }
            ts += s_wsum[w][0];
            tl += s_wsum[w][1];
        }
        s_sstart[tid] = ps + xs - (large ? 0u : cnt);
        if (large) s_large[pl + xl - 1u] = (uint16_t)tid;
        if (tid == 0) {
            s_small = ts;
            s_nlarge = tl;
        }
        __syncthreads();
    }
    const uint32_t *pref = any_large ? s_sstart : s_start;
    const uint32_t total_small = any_large ? s_small : total;
    for (uint32_t e = tid; e < total_small; e += kEmitThreads) {
        int lo = 0, hi = nb - 1;  // last Gaussian whose (small-instance) start is <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pref[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        uint32_t local = e - pref[lo];
        const uint32_t at = s_start[lo] + local;
        const uint2 rc = s_rect[lo];
        const Cover cv = s_cv[lo];
        const int ty_lo = (int)(rc.y & 0xffffu), ty_hi = (int)(rc.y >> 16);
        uint32_t key = 0xffffffffu;
        // spans stored by the counting pass
        const uint32_t pk[kCoverRows] = {__float_as_uint(cv.a.x), __float_as_uint(cv.a.y),
                                         __float_as_uint(cv.a.z), __float_as_uint(cv.a.w),
                                         __float_as_uint(cv.b.x), __float_as_uint(cv.b.y),
                                         __float_as_uint(cv.b.z), __float_as_uint(cv.b.w)};
#pragma unroll
        for (int r = 0; r < kCoverRows; ++r) {
            const uint32_t t0 = pk[r] & 0xffffu, t1 = pk[r] >> 16;
            const uint32_t n = t0 <= t1 ? t1 - t0 + 1u : 0u;
            if (key == 0xffffffffu && r <= ty_hi - ty_lo) {
                if (local < n)
                    key = s_vb[lo] + (uint32_t)(ty_lo + r) * (uint32_t)cam.tiles_x + t0 + local;
                else
                    local -= n;
            }
        }
        if (key == 0xffffffffu) {  // the rows hold fewer tiles than were counted: never in a sound build
            set_status(status, VPGS_ERR_INTERNAL);
            key = 0u;
        }
        ikey[base + at] = key;
        ival[base + at] = s_id[lo];
        add_digits(s_h, tps, n_pass, key);
    }
    // large Gaussians: one warp each, one tile row per lane, a warp prefix of the
    // rows' counts, each lane writing its row's run of tiles
    const uint32_t n_large = any_large ? s_nlarge : 0u;
    for (uint32_t j = warp; j < n_large; j += kEmitThreads / 32) {
        const int t = s_large[j];
        const uint2 rc = s_rect[t];
        const Cover cv = s_cv[t];
        const float4 uv = s_uv[t];
        const int tx_lo = (int)(rc.x & 0xffffu), tx_hi = (int)(rc.x >> 16);
        const int ty_lo = (int)(rc.y & 0xffffu), ty_hi = (int)(rc.y >> 16);
        const uint32_t start = s_start[t], end = (t + 1 < nb ? s_start[t + 1] : total);
        const uint32_t vb = s_vb[t], id = s_id[t];
        uint32_t running = start;
        for (int ty0 = ty_lo; ty0 <= ty_hi; ty0 += 32) {  // warp-uniform
            const int ty = ty0 + lane;
            int2 sp = make_int2(1, 0);
            if (ty <= ty_hi)
                sp = cover_row(cv, uv.x, uv.z, uv.y, uv.w, ty, tx_lo, tx_hi, cam.tw_shift, cam.tile_h, cam.W, cam.H);
            const uint32_t n = sp.x <= sp.y ? (uint32_t)(sp.y - sp.x + 1) : 0u;
            uint32_t x = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const uint32_t at = running + x - n;
            for (uint32_t k = 0; k < n; ++k) {
                if (at + k >= end) {  // more tiles than were counted: never in a sound build
                    set_status(status, VPGS_ERR_INTERNAL);
                    break;
                }
                const uint32_t key = vb + (uint32_t)ty * (uint32_t)cam.tiles_x + (uint32_t)sp.x + k;
                ikey[base + at + k] = key;
                ival[base + at + k] = id;
                add_digits(s_h, tps, n_pass, key);
            }
            running += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0 && running != end) set_status(status, VPGS_ERR_INTERNAL);
    }
    __syncthreads();  // the next chunk reuses the shared arrays
    }
    __syncthreads();
    flush_digits(s_h, n_pass, hist);
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys, int64_t cap, const uint32_t *n_dev,
                                   uint32_t n_tiles, uint2 *ranges) {
    grid_dep_enter();
    int64_t n = min(cap, (int64_t)*n_dev);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= n_tiles) continue;  // only after a capacity overflow (status already set)
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

// Launch order of the compositing kernels: global tile ids by descending
// instance count, so the longest tiles start first and the short ones fill the
// tail of the grid (tiles are independent: the order changes no pixel).  One
// block: tiles are bucketed by count / 4 (the last bucket takes every count
// beyond), buckets are laid out from the heaviest down, and each tile takes a
// slot in its bucket by a shared-memory atomic.  Up to kOrderPer tiles per
// thread (8, or 32 past 8,192 tiles) are loaded at once and kept in registers
// (packed) between the passes.
constexpr int kOrderThreads = 1024;
constexpr int kOrderBins = 1024;

// work of tile i: its step count if given, else its instance count
VPGS_D uint32_t order_bucket(const uint2 *ranges, const uint32_t *work, int i) {
    uint32_t c;
    if (work) {
        c = work[i];
    } else {
        const uint2 r = ranges[i];
        c = r.y > r.x ? r.y - r.x : 0u;
    }
    return min(c >> 2, (uint32_t)kOrderBins - 1u);
}

template <int kOrderPer>
__global__ void __launch_bounds__(kOrderThreads)
tile_order_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ work, int n_tiles,
                  uint32_t *__restrict__ order) {
    grid_dep_enter();
    __shared__ uint32_t s_bin[kOrderBins];
    __shared__ uint32_t s_warp[kOrderThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool fits = n_tiles <= kOrderThreads * kOrderPer;  // block-uniform
    // bucket of tile tid + k * kOrderThreads (kOrderBins: none), two 16-bit buckets
    // per register (a 1,024-thread block has 64 registers per thread)
    uint32_t bk[kOrderPer / 2];
    auto bucket_of = [&](int k) { return (bk[k >> 1] >> (16 * (k & 1))) & 0xffffu; };
    if (fits) {
#pragma unroll
        for (int k = 0; k < kOrderPer; ++k) {
            const int i = tid + k * kOrderThreads;
            const uint32_t b = i < n_tiles ? order_bucket(ranges, work, i) : (uint32_t)kOrderBins;
            if (k & 1) bk[k >> 1] |= b << 16;
            else bk[k >> 1] = b;
        }
    }
    for (int i = tid; i < kOrderBins; i += kOrderThreads) s_bin[i] = 0u;
    __syncthreads();
    if (fits) {
#pragma unroll
        for (int k = 0; k < kOrderPer; ++k)
            if (bucket_of(k) < (uint32_t)kOrderBins) atomicAdd(&s_bin[bucket_of(k)], 1u);
    } else {
        for (int i = tid; i < n_tiles; i += kOrderThreads) atomicAdd(&s_bin[order_bucket(ranges, work, i)], 1u);
    }
    __syncthreads();
    // exclusive scan over the buckets from the heaviest (thread j holds bucket kOrderBins-1-j)
    const int b = kOrderBins - 1 - tid;
    const uint32_t c = s_bin[b];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive totals of warps 0..lane
    }
    __syncthreads();
    s_bin[b] = x - c + (warp > 0 ? s_warp[warp - 1] : 0u);  // every thread read its count before the barrier
    __syncthreads();
    if (fits) {
#pragma unroll
        for (int k = 0; k < kOrderPer; ++k)
            if (bucket_of(k) < (uint32_t)kOrderBins)
                order[atomicAdd(&s_bin[bucket_of(k)], 1u)] = (uint32_t)(tid + k * kOrderThreads);
    } else {
        for (int i = tid; i < n_tiles; i += kOrderThreads)
            order[atomicAdd(&s_bin[order_bucket(ranges, work, i)], 1u)] = (uint32_t)i;
    }
}

// The backward's steps per tile: the largest n_iter (list position of the last
// Gaussian a pixel blended, from the forward) over the tile's pixels.  One warp
// per tile.
constexpr int kWorkThreads = 256;

__global__ void __launch_bounds__(kWorkThreads)
tile_work_kernel(const int32_t *__restrict__ n_iter, CamParams cam, int n_tiles, uint32_t *__restrict__ work) {
    grid_dep_enter();
    const int t = (int)((blockIdx.x * (unsigned)kWorkThreads + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= n_tiles) return;  // whole warps
    const int v = t / cam.T, lt = t - v * cam.T;
    const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
    const int64_t base = (int64_t)v * cam.H * cam.W;
    int m = 0;
    for (int i = lane; i < cam.tile_w * cam.tile_h; i += 32) {
        const int px = tx * cam.tile_w + i % cam.tile_w, py = ty * cam.tile_h + i / cam.tile_w;
        if (px < cam.W && py < cam.H) m = max(m, n_iter[base + (int64_t)py * cam.W + px]);
    }
    m = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(m, 0));
    if (lane == 0) work[t] = (uint32_t)m;
}

cudaError_t order_tiles_by_steps(const RenderWs &ws, const int32_t *n_iter, int V, const CamParams &cam,
                                 cudaStream_t s) {
    const int n_tiles = V * cam.T;
    if (n_tiles == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((int64_t)n_tiles * 32 + kWorkThreads - 1) / kWorkThreads);
    VPGS_LAUNCH("tile_work", s, launch_k(tile_work_kernel, blocks, kWorkThreads, 0, s, n_iter, cam, n_tiles,
                                         ws.tile_work));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_tiles <= kOrderThreads * 8)
        VPGS_LAUNCH("tile_order", s, launch_k(tile_order_kernel<8>, 1, kOrderThreads, 0, s,
                                              (const uint2 *)ws.ranges, (const uint32_t *)ws.tile_work, n_tiles,
                                              ws.tile_order));
    else
        VPGS_LAUNCH("tile_order", s, launch_k(tile_order_kernel<32>, 1, kOrderThreads, 0, s,
                                              (const uint2 *)ws.ranges, (const uint32_t *)ws.tile_work, n_tiles,
                                              ws.tile_order));
    return cudaGetLastError();
}

int tile_list_buffer(const RenderLayout &L) {
    SortPass ps[kMaxSortPasses];
    return (plan_passes(0, L.tile_bits, ps) & 1) != 0 ? 1 : 0;
}

// SM count of the current device, looked up once per device ordinal.
int device_sm_count() {
    static std::atomic<int> cache[kDeviceCache];
    return per_device(cache, [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
        return sms;
    });
}

cudaError_t build_tile_lists(const GaussIn &g, int V, const CamParams &cam, const OptParams &o, const RenderWs &ws,
                             const RenderLayout &L, int *sorted_buf, cudaStream_t s, bool order_by_count) {
    // every binning kernel stops at entry once a predecessor recorded an error: after
    // a timed-out look-back the compacted and sorted arrays hold holes whose stale
    // contents must not be used as indices
    const LookBack lb{o.spin_limit, true};
    cudaError_t e;
    const int sms = device_sm_count();
    (void)sms;
    uint32_t *n_vis = ws.counters + CNT_VISIBLE;
    uint32_t *n_inst = ws.counters + CNT_INSTANCES;
    // calls of many views (above 4M pairs): wider scan tiles and depth-sort tiles,
    // the offset scan on the resident grid (the visible pairs then fill it)
    const bool many = L.VN > (int64_t(4) << 20);
    // 1. compaction of visible (view, Gaussian) pairs
    e = launch_scan("scan_visible", VisLoad{ws.tcount}, VisStore{ws.rec, ws.dkey[0], ws.dval[0], ws.vis_idx, L.VN},
                    L.VN, nullptr, ws.counters + CNT_TICKET_A, ws.scan_look[0], n_vis, ws.status, s, lb, 0, many);
    if (e != cudaSuccess) return e;
    // 2. depth sort
    bool in1 = false;
    // (digit histograms from the projection kernel)
    // keys per thread: few for a frame's worth of visible Gaussians (short tiles
    // start the look-back chain sooner), more for many views' worth (fewer tiles
    // in the chain); the look-back space is sized for kDepthSortItems, the most tiles
    const int depth_items = many ? 16 : kDepthSortItems;
    e = radix_sort_pairs("sort_depth_pass", ws.dkey[0], ws.dval[0], ws.dkey[1], ws.dval[1], L.VN, n_vis,
                         0, 32, ws.sort_hist[0], ws.counters + CNT_TICKET_D, ws.sort_look[0], ws.status, s,
                         &in1, depth_items, lb, VPGS_DEPTH_SORT_GRID);
    if (e != cudaSuccess) return e;
    const uint32_t *dval = in1 ? ws.dval[1] : ws.dval[0];  // visible records in depth order
    uint32_t *inst_off = in1 ? ws.dkey[0] : ws.dkey[1];  // the depth-sort buffer not holding the result
    SortPass tps[kMaxSortPasses] = {};
    const int np_tile = plan_passes(0, L.tile_bits, tps);
    if (np_tile > 4) return cudaErrorInvalidValue;
    // 3. instance offsets, then emission
    e = launch_scan("scan_offsets", CountLoad{ws.tcount, dval}, OffsetStore{inst_off}, L.VN, n_vis,
                    ws.counters + CNT_TICKET_O, ws.scan_look[1], n_inst, ws.status, s, lb,
                    many ? 0 : VPGS_OFFSET_SCAN_GRID, many);
    if (e != cudaSuccess) return e;
    static std::atomic<int> emit_cache[kDeviceCache];
    const int emit_grid = per_device(emit_cache, [] {
        return resident_grid((const void *)emit_kernel, kEmitThreads, 0, int64_t(1) << 30);
    });
    VPGS_LAUNCH("emit_instances", s,
                launch_k(emit_kernel, (unsigned)std::min<int64_t>(std::max<int64_t>((L.VN + kEmitThreads - 1) / kEmitThreads, 1),
                                                          emit_grid),
                              kEmitThreads, 0, s, dval, inst_off, ws.bin, n_vis, n_inst, L.N, L.M_cap,
                                                    cam, ws.ikey[0], ws.ival[0], ws.status, np_tile, tps[0],
                                                    tps[1], tps[2], tps[3], ws.sort_hist[1], ws.sort_look[1]));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // 4. stable sort by tile id
    // (digit histograms from the emit kernel)
    e = radix_sort_pairs("sort_tile_pass", ws.ikey[0], ws.ival[0], ws.ikey[1], ws.ival[1], L.M_cap, n_inst, 0,
                         L.tile_bits, ws.sort_hist[1], ws.counters + CNT_TICKET_T, ws.sort_look[1],
                         ws.status, s, &in1, kTileSortItems, lb);
    if (e != cudaSuccess) return e;
    *sorted_buf = in1 ? 1 : 0;
    if (*sorted_buf != tile_list_buffer(L)) return cudaErrorUnknown;  // never: same pass plan
    // 5. tile ranges
    const int n_tiles = V * cam.T;  // (ranges zeroed by the prepare kernel)
    const int64_t rb = std::min<int64_t>((L.M_cap + 255) / 256, (int64_t)sms * 16);
    VPGS_LAUNCH("tile_ranges", s,
                launch_k(tile_ranges_kernel, (unsigned)std::max<int64_t>(rb, 1), 256, 0, s,
                    in1 ? ws.ikey[1] : ws.ikey[0], L.M_cap, n_inst, (uint32_t)n_tiles, ws.ranges));
    e = cudaGetLastError();
    if (e != cudaSuccess || !VPGS_TILE_ORDER || !order_by_count) return e;
    // 6. compositing launch order
    if (n_tiles <= kOrderThreads * 8)
        VPGS_LAUNCH("tile_order", s, launch_k(tile_order_kernel<8>, 1, kOrderThreads, 0, s, (const uint2 *)ws.ranges,
                                              (const uint32_t *)nullptr, n_tiles, ws.tile_order));
    else
        VPGS_LAUNCH("tile_order", s, launch_k(tile_order_kernel<32>, 1, kOrderThreads, 0, s, (const uint2 *)ws.ranges,
                                              (const uint32_t *)nullptr, n_tiles, ws.tile_order));
    return cudaGetLastError();
}

}  // namespace vpgs
