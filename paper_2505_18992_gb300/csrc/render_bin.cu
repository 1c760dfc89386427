// Tile binning: which Gaussians touch which tile, in depth order.
//
//   1. scan of the visibility flags (tile count > 0) -> compacted (z bits, id)
//   2. stable radix sort of the visible pairs by the FP32 bit pattern of the
//      camera depth (positive floats order like their bits); ties keep index
//      order, i.e. (view, Gaussian) order
//   3. scan of the tile counts in depth order, then a block-cooperative emit
//      of each Gaussian's (global tile id, id) instances at its offset
//   4. stable radix sort of the instances by global tile id (only the bits a
//      tile id needs); instances stay in depth order inside each tile
//   5. [start, end) of every tile from the sorted keys
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
    uint32_t *dkey, *dval;
    int64_t cap;
    __device__ void operator()(int64_t i, uint32_t pos, uint32_t v) const {
        if (v && (int64_t)pos < cap) {
            dkey[pos] = __float_as_uint(rec[i].r2.y);  // camera z > near_z > 0
            dval[pos] = (uint32_t)i;
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
// Gaussians per block.  The block's instances are spread evenly over its
// threads; each finds its Gaussian by binary search over the block's local
// offsets, so a Gaussian covering thousands of tiles does not serialise.
constexpr int kEmitThreads = 256;

__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const uint32_t *__restrict__ dval, const uint32_t *__restrict__ tcount,
            const uint32_t *__restrict__ inst_off, const uint2 *__restrict__ rect,
            const uint32_t *n_vis, int64_t N, int64_t M_cap, int T, int tiles_x,
            uint32_t *__restrict__ ikey, uint32_t *__restrict__ ival, uint32_t *status) {
    __shared__ uint32_t s_start[kEmitThreads], s_id[kEmitThreads], s_w[kEmitThreads];
    __shared__ uint32_t s_tx0[kEmitThreads], s_ty0[kEmitThreads], s_vb[kEmitThreads];
    __shared__ uint32_t s_total;
    const int64_t nv = *n_vis;
    const int64_t r0 = (int64_t)blockIdx.x * kEmitThreads;
    if (r0 >= nv) return;
    const int tid = threadIdx.x;
    const int nb = (int)min((int64_t)kEmitThreads, nv - r0);
    const uint32_t base = inst_off[r0];
    if (tid < nb) {
        const int64_t r = r0 + tid;
        const uint32_t id = dval[r];
        const uint32_t cnt = tcount[id];
        const uint32_t off = inst_off[r] - base;
        const uint2 rc = rect[id];
        s_start[tid] = off;
        s_id[tid] = id;
        s_tx0[tid] = rc.x & 0xffffu;
        s_w[tid] = (rc.x >> 16) - (rc.x & 0xffffu) + 1u;
        s_ty0[tid] = rc.y & 0xffffu;
        s_vb[tid] = (uint32_t)(id / N) * (uint32_t)T;
        if (tid == nb - 1) s_total = off + cnt;
    }
    __syncthreads();
    const uint32_t total = s_total;
    if ((int64_t)base + total > M_cap) {
        if (tid == 0) set_status(status, VPGS_ERR_CAPACITY);
        return;
    }
    for (uint32_t e = tid; e < total; e += kEmitThreads) {
        int lo = 0, hi = nb - 1;  // last Gaussian whose local start is <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t local = e - s_start[lo];
        const uint32_t w = s_w[lo];
        const uint32_t ty = s_ty0[lo] + local / w, tx = s_tx0[lo] + local % w;
        ikey[base + e] = s_vb[lo] + ty * (uint32_t)tiles_x + tx;
        ival[base + e] = s_id[lo];
    }
}

// ---------------------------------------------------------------------------
// Direct binning: the visible Gaussians are already in depth order, so tile
// lists in depth order are a stable counting sort by tile id over that order.
//   bin_count: per block of kBinRanks ranks, instances per tile (shared-memory
//              counters), written tile-major: bins[t * nbk + b]
//   scan:      exclusive scan of bins -> global slot of (tile t, block b)
//   bin_place: one warp per block walks its instances in (rank, tile) order and
//              places each at its tile's slot + its stable rank (match-any on
//              the tile id); blocks also write the [start, end) of a slice of tiles
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBinRanks)
bin_count_kernel(const uint32_t *__restrict__ dval, const uint2 *__restrict__ rect, const uint32_t *n_vis,
                 int64_t N, int T, int tiles_x, int n_tiles, uint32_t *__restrict__ bins, uint32_t *bin_n) {
    extern __shared__ uint32_t s_h[];
    const int64_t nv = *n_vis;
    const int64_t nbk = (nv + kBinRanks - 1) / kBinRanks;
    const int64_t b = blockIdx.x;
    const int tid = threadIdx.x;
    if (b == 0 && tid == 0) *bin_n = (uint32_t)(nbk * n_tiles);
    if (b >= nbk) return;
    for (int t = tid; t < n_tiles; t += kBinRanks) s_h[t] = 0u;
    __syncthreads();
    const int64_t r = b * kBinRanks + tid;
    if (r < nv) {
        const uint32_t i = dval[r];
        const uint32_t vb = (uint32_t)(i / N) * (uint32_t)T;
        const uint2 rc = rect[i];
        for (uint32_t ty = rc.y & 0xffffu; ty <= (rc.y >> 16); ++ty)
            for (uint32_t tx = rc.x & 0xffffu; tx <= (rc.x >> 16); ++tx)
                atomicAdd(&s_h[vb + ty * (uint32_t)tiles_x + tx], 1u);
    }
    __syncthreads();
    for (int t = tid; t < n_tiles; t += kBinRanks) bins[(int64_t)t * nbk + b] = s_h[t];
}

__global__ void __launch_bounds__(32)
bin_place_kernel(const uint32_t *__restrict__ dval, const uint32_t *__restrict__ tcount,
                 const uint2 *__restrict__ rect, const uint32_t *n_vis, const uint32_t *n_inst, int64_t N,
                 int T, int tiles_x, int n_tiles, const uint32_t *__restrict__ bins, int64_t M_cap,
                 uint32_t *__restrict__ ival, uint2 *__restrict__ ranges, uint32_t *status) {
    extern __shared__ uint32_t s_pos[];
    __shared__ uint32_t s_off[kBinRanks + 1], s_id[kBinRanks], s_tx0[kBinRanks], s_w[kBinRanks],
        s_ty0[kBinRanks], s_vb[kBinRanks];
    const int64_t nv = *n_vis;
    const int64_t nbk = (nv + kBinRanks - 1) / kBinRanks;
    const int64_t b = blockIdx.x;
    const int lane = threadIdx.x;
    if (b >= nbk) return;
    const uint32_t total = *n_inst;
    if ((int64_t)total > M_cap) {
        if (b == 0 && lane == 0) set_status(status, VPGS_ERR_CAPACITY);
        return;
    }
    // [start, end) of this block's slice of tiles
    const int64_t chunk = (n_tiles + nbk - 1) / nbk;
    for (int64_t t = b * chunk + lane; t < min((int64_t)n_tiles, (b + 1) * chunk); t += 32) {
        const uint32_t st = bins[t * nbk];
        const uint32_t en = t + 1 < n_tiles ? bins[(t + 1) * nbk] : total;
        ranges[t] = make_uint2(st, en);
    }
    // a tile's global slot is read on first touch (most tiles are never touched by a block)
    constexpr uint32_t kUnread = 0xffffffffu;
    for (int t = lane; t < n_tiles; t += 32) s_pos[t] = kUnread;
    const int nb = (int)min((int64_t)kBinRanks, nv - b * kBinRanks);
    // the block's ranks and their local instance offsets (warp scan, 8 per lane)
    uint32_t run = 0;
    uint32_t cnt8[kBinRanks / 32];  // ranks per lane: kBinRanks / 32
#pragma unroll
    for (int q = 0; q < kBinRanks / 32; ++q) {
        const int i = lane * (kBinRanks / 32) + q;
        uint32_t c = 0;
        if (i < nb) {
            const uint32_t id = dval[b * kBinRanks + i];
            const uint2 rc = rect[id];
            c = tcount[id];
            s_id[i] = id;
            s_tx0[i] = rc.x & 0xffffu;
            s_w[i] = (rc.x >> 16) - (rc.x & 0xffffu) + 1u;
            s_ty0[i] = rc.y & 0xffffu;
            s_vb[i] = (uint32_t)(id / N) * (uint32_t)T;
        }
        cnt8[q] = c;
        run += c;
    }
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t acc = x - run;
#pragma unroll
    for (int q = 0; q < kBinRanks / 32; ++q) {
        s_off[lane * (kBinRanks / 32) + q] = acc;
        acc += cnt8[q];
    }
    const uint32_t blk_total = __shfl_sync(0xffffffffu, x, 31);
    __syncwarp();
    // stable placement in (rank, tile) order
    for (uint32_t e0 = 0; e0 < blk_total; e0 += 32) {
        const uint32_t e = e0 + lane;
        const bool valid = e < blk_total;
        uint32_t t = 0xffffffe0u + lane;  // unique, never a tile id
        uint32_t id = 0;
        if (valid) {
            int lo = 0, hi = nb - 1;  // last rank whose local start is <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const uint32_t local = e - s_off[lo];
            const uint32_t w = s_w[lo];
            t = s_vb[lo] + (s_ty0[lo] + local / w) * (uint32_t)tiles_x + s_tx0[lo] + local % w;
            id = s_id[lo];
        }
        const uint32_t m = __match_any_sync(0xffffffffu, t);
        const uint32_t rk = __popc(m & lanemask_lt());
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (valid && rk == 0) {
            base = s_pos[t];
            if (base == kUnread) base = bins[(int64_t)t * nbk + b];
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        __syncwarp();
        if (valid) {
            const uint32_t pos = base + rk;
            if ((int64_t)pos < M_cap) ival[pos] = id;
            if (rk == 0) s_pos[t] = base + __popc(m);
        }
        __syncwarp();
    }
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys, int64_t cap, const uint32_t *n_dev,
                                   uint32_t n_tiles, uint2 *ranges) {
    int64_t n = min(cap, (int64_t)*n_dev);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= n_tiles) continue;  // only after a capacity overflow (status already set)
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

int device_sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

cudaError_t build_tile_lists(const GaussIn &g, int V, const CamParams &cam, const RenderWs &ws,
                             const RenderLayout &L, int *sorted_buf, cudaStream_t s) {
    cudaError_t e;
    const int sms = device_sm_count();
    uint32_t *n_vis = ws.counters + CNT_VISIBLE;
    uint32_t *n_inst = ws.counters + CNT_INSTANCES;
    // 1. compaction of visible (view, Gaussian) pairs
    e = launch_scan("scan_visible", VisLoad{ws.tcount}, VisStore{ws.rec, ws.dkey[0], ws.dval[0], L.VN},
                    L.VN, nullptr, ws.counters + CNT_TICKET_A, ws.scan_look, n_vis, ws.status, s);
    if (e != cudaSuccess) return e;
    // 2. depth sort
    bool in1 = false;
    e = radix_sort_pairs("sort_depth_pass", ws.dkey[0], ws.dval[0], ws.dkey[1], ws.dval[1], L.VN, n_vis,
                         0, 32, ws.sort_hist, ws.counters + CNT_TICKET_B, ws.sort_look, ws.status, sms, s,
                         &in1, kDepthSortItems, VPGS_DEPTH_LOOKBACK != 0, ws.counters + CNT_TICKET_A,
                         ws.scan_look);
    if (e != cudaSuccess) return e;
    const uint32_t *dval = in1 ? ws.dval[1] : ws.dval[0];
    const int n_tiles = V * cam.T;
    if (L.direct_bins) {
        // 3. + 4. + 5. direct binning (count, scan, stable placement + tile ranges)
        e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
        if (e != cudaSuccess) return e;
        const size_t hsm = sizeof(uint32_t) * (size_t)n_tiles;
        if (hsm > 48 * 1024) {  // per device and call: cheap, and right on every GPU of the process
            cudaFuncSetAttribute((const void *)bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            cudaFuncSetAttribute((const void *)bin_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        }
        uint32_t *bin_n = ws.counters + CNT_BIN_N;
        VPGS_LAUNCH("bin_count", s,
                    bin_count_kernel<<<(unsigned)L.bin_blocks, kBinRanks, hsm, s>>>(
                        dval, ws.rect, n_vis, L.N, cam.T, cam.tiles_x, n_tiles, ws.bins, bin_n));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_scan("scan_bins", CountsLoad{ws.bins}, CountsStore{ws.bins}, (int64_t)n_tiles * L.bin_blocks,
                        bin_n, ws.counters + CNT_TICKET_A, ws.scan_look, n_inst, ws.status, s);
        if (e != cudaSuccess) return e;
        VPGS_LAUNCH("bin_place", s,
                    bin_place_kernel<<<(unsigned)L.bin_blocks, 32, hsm, s>>>(
                        dval, ws.tcount, ws.rect, n_vis, n_inst, L.N, cam.T, cam.tiles_x, n_tiles, ws.bins,
                        L.M_cap, ws.ival[0], ws.ranges, ws.status));
        *sorted_buf = 0;
        return cudaGetLastError();
    }
    uint32_t *inst_off = in1 ? ws.dkey[0] : ws.dkey[1];  // the depth-sort buffer not holding the result
    // 3. instance offsets, then emission
    e = launch_scan("scan_offsets", CountLoad{ws.tcount, dval}, OffsetStore{inst_off}, L.VN, n_vis,
                    ws.counters + CNT_TICKET_A, ws.scan_look, n_inst, ws.status, s);
    if (e != cudaSuccess) return e;
    VPGS_LAUNCH("emit_instances", s,
                emit_kernel<<<(unsigned)std::max<int64_t>((L.VN + kEmitThreads - 1) / kEmitThreads, 1),
                              kEmitThreads, 0, s>>>(dval, ws.tcount, inst_off, ws.rect, n_vis, L.N, L.M_cap,
                                                    cam.T, cam.tiles_x, ws.ikey[0], ws.ival[0], ws.status));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // 4. stable sort by tile id
    e = radix_sort_pairs("sort_tile_pass", ws.ikey[0], ws.ival[0], ws.ikey[1], ws.ival[1], L.M_cap, n_inst, 0,
                         L.tile_bits, ws.sort_hist, ws.counters + CNT_TICKET_B, ws.sort_look,
                         ws.status, sms, s, &in1, kTileSortItems, VPGS_TILE_LOOKBACK != 0,
                         ws.counters + CNT_TICKET_A, ws.scan_look);
    if (e != cudaSuccess) return e;
    *sorted_buf = in1 ? 1 : 0;
    // 5. tile ranges
    e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * (size_t)V * cam.T, s);
    if (e != cudaSuccess) return e;
    const int64_t rb = std::min<int64_t>((L.M_cap + 255) / 256, (int64_t)sms * 16);
    VPGS_LAUNCH("tile_ranges", s,
                tile_ranges_kernel<<<(unsigned)std::max<int64_t>(rb, 1), 256, 0, s>>>(
                    in1 ? ws.ikey[1] : ws.ikey[0], L.M_cap, n_inst, (uint32_t)(V * cam.T), ws.ranges));
    return cudaGetLastError();
}

}  // namespace vpgs
