// Tile binning: which Gaussians touch which tile, in depth order.
//
//   1. scan of the visibility flags (tile count > 0) -> compacted (z bits, id)
//   2. stable radix sort of the visible pairs by the FP32 bit pattern of the
//      camera depth (positive floats order like their bits); ties keep index
//      order, i.e. (view, Gaussian) order
//   3. scan of the tile counts in depth order; the store step of that scan
//      writes each Gaussian's (global tile id, id) instances at its offset
//   4. stable radix sort of the instances by global tile id (only the bits a
//      tile id needs); instances stay in depth order inside each tile
//   5. [start, end) of every tile from the sorted keys
//
// Sorting the visible Gaussians once by depth and then the instances by tile
// id only moves 32-bit depth keys over N_visible items and a 12-14 bit tile key
// over the instances, instead of a 44+ bit (tile, depth) key over all instances.
#include "internal.h"
#include "prims.cuh"

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

struct EmitStore {
    const uint32_t *dval;
    const uint2 *rect;
    uint32_t *ikey, *ival;
    int64_t N, M_cap;
    int T, tiles_x;
    uint32_t *status;
    __device__ void operator()(int64_t r, uint32_t off, uint32_t cnt) const {
        if (cnt == 0) return;
        if ((int64_t)off + cnt > M_cap) {
            set_status(status, VPGS_ERR_CAPACITY);
            return;
        }
        const uint32_t i = dval[r];
        const uint32_t v = (uint32_t)(i / N);
        const uint2 rc = rect[i];
        const uint32_t tx0 = rc.x & 0xffffu, tx1 = rc.x >> 16, ty0 = rc.y & 0xffffu, ty1 = rc.y >> 16;
        uint32_t o = off;
        const uint32_t base = v * (uint32_t)T;
        for (uint32_t ty = ty0; ty <= ty1; ++ty) {
            const uint32_t row = base + ty * (uint32_t)tiles_x;
            for (uint32_t tx = tx0; tx <= tx1; ++tx) {
                ikey[o] = row + tx;
                ival[o] = i;
                ++o;
            }
        }
    }
};

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
    e = launch_scan(VisLoad{ws.tcount}, VisStore{ws.rec, ws.dkey[0], ws.dval[0], L.VN}, L.VN, nullptr,
                    ws.counters + CNT_TICKET_A, ws.scan_look, n_vis, ws.status, s);
    if (e != cudaSuccess) return e;
    // 2. depth sort
    bool in1 = false;
    e = radix_sort_pairs(ws.dkey[0], ws.dval[0], ws.dkey[1], ws.dval[1], L.VN, n_vis, 0, 32,
                         ws.sort_hist, ws.counters + CNT_TICKET_B, ws.sort_look, ws.status, sms, s,
                         &in1);
    if (e != cudaSuccess) return e;
    const uint32_t *dval = in1 ? ws.dval[1] : ws.dval[0];
    // 3. instance offsets and emission
    EmitStore em{dval, ws.rect, ws.ikey[0], ws.ival[0], L.N, L.M_cap, cam.T, cam.tiles_x, ws.status};
    e = launch_scan(CountLoad{ws.tcount, dval}, em, L.VN, n_vis, ws.counters + CNT_TICKET_A,
                    ws.scan_look, n_inst, ws.status, s);
    if (e != cudaSuccess) return e;
    // 4. stable sort by tile id
    e = radix_sort_pairs(ws.ikey[0], ws.ival[0], ws.ikey[1], ws.ival[1], L.M_cap, n_inst, 0,
                         L.tile_bits, ws.sort_hist, ws.counters + CNT_TICKET_B, ws.sort_look,
                         ws.status, sms, s, &in1);
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
