// Front-to-back alpha compositing per tile, and its backward pass.
//
// One CTA renders one tile (tile_w x tile_h threads, one pixel each), or, in
// persistent mode, a fixed number of CTAs per SM pull tiles from a work queue.
// The tile's depth-ordered Gaussian list is staged through shared memory in
// batches of one record per thread; each pixel walks the batch in order:
//   alpha = min(alpha_max, o exp(-((w1.d)^2 + (w2.d)^2)/2)), d = pixel - mean
//   skip alpha < alpha_min; stop before T (1 - alpha) < t_min
//   C += alpha T c, D += alpha T z, T *= 1 - alpha
// Means are made tile-local when staged ((u_hi - x0) + u_lo), so d keeps
// ~1e-7 px accuracy anywhere in the image.
//
// The backward pass walks the same list from the back, recovering T_i as
// T_{i+1} / (1 - alpha_i), and keeps the colour/depth "behind" each Gaussian,
//   B <- alpha c + (1 - alpha) B   (B starts at the background),
// giving dC/dalpha_i = T_i (c_i - B_i), dA/dalpha_i = T_final / (1 - alpha_i).
// Per-Gaussian 2D gradients (u, v, conic a b c, opacity, rgb, z) of a warp are
// summed by a transpose reduction (16 shuffles for 10 values) and added with
// one atomic per value per warp.
#include "internal.h"
#include "profiler.h"

namespace vpgs {

struct TileCoord {
    int v, tx, ty;
};

VPGS_D TileCoord tile_coord(int t, const CamParams &cam) {
    TileCoord c;
    c.v = t / cam.T;
    const int lt = t - c.v * cam.T;
    c.ty = lt / cam.tiles_x;
    c.tx = lt - c.ty * cam.tiles_x;
    return c;
}

__global__ void __launch_bounds__(1024)
composite_fwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, int n_tiles, CamParams cam, OptParams o,
                     vpgs_images out, const uint32_t *status, uint32_t *work) {
    extern __shared__ float4 smem[];
    const int B = blockDim.x;
    float4 *s0 = smem, *s1 = smem + B, *s2 = smem + 2 * B;
    __shared__ int s_tile;
    if (*status != 0u) return;
    const int tid = threadIdx.x;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f, pyl = (float)ly + 0.5f;
    int t = blockIdx.x;
    for (;;) {
        if (work) {
            if (tid == 0) s_tile = (int)atomicAdd(work, 1u);
            __syncthreads();
            t = s_tile;
            __syncthreads();
        }
        if (t >= n_tiles) return;
        const TileCoord tc = tile_coord(t, cam);
        const int px = tc.tx * cam.tile_w + lx, py = tc.ty * cam.tile_h + ly;
        const bool inside = px < cam.W && py < cam.H;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const uint2 rg = ranges[t];
        const int start = (int)rg.x, end = (int)rg.y;
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
        int cnt = 0, last = 0;
        bool done = !inside;
        for (int b0 = start; b0 < end; b0 += B) {
            if (__syncthreads_count(done) == B) break;
            const int j = b0 + tid;
            if (j < end) {
                const Rec r = rec[ival[j]];
                s0[tid] = make_float4((r.r0.x - ox) + r.r0.z, (r.r0.y - oy) + r.r0.w, r.r1.x, r.r1.y);
                s1[tid] = make_float4(r.r1.z, r.r1.w, r.r2.x, r.r2.y);
                s2[tid] = make_float4(r.r2.z, r.r2.w, r.r3.x, 0.f);
            }
            __syncthreads();
            if (!done) {
                const int nb = min(B, end - b0);
                for (int k = 0; k < nb; ++k) {
                    const float4 a = s0[k], b = s1[k];
                    const PairEval e = eval_pair(pxl - a.x, pyl - a.y, a.z, a.w, b.x, b.y, b.z, o.alpha_max);
                    if (e.alpha < o.alpha_min) continue;
                    const float nt = T * (1.f - e.alpha);
                    if (nt < o.t_min) {
                        done = true;
                        break;
                    }
                    const float w = e.alpha * T;
                    const float4 c = s2[k];
                    C0 = fmaf(w, c.x, C0);
                    C1 = fmaf(w, c.y, C1);
                    C2 = fmaf(w, c.z, C2);
                    D = fmaf(w, b.w, D);
                    T = nt;
                    ++cnt;
                    last = b0 + k - start + 1;
                }
            }
        }
        if (inside) {
            const int64_t HW = (int64_t)cam.H * cam.W;
            const int64_t pix = (int64_t)tc.v * HW + (int64_t)py * cam.W + px;
            if (out.rgb) {
                float *rgb = out.rgb + (int64_t)tc.v * 3 * HW + (int64_t)py * cam.W + px;
                rgb[0] = fmaf(T, o.bg0, C0);
                rgb[HW] = fmaf(T, o.bg1, C1);
                rgb[2 * HW] = fmaf(T, o.bg2, C2);
            }
            if (out.depth) out.depth[pix] = D;
            if (out.alpha) out.alpha[pix] = 1.f - T;
            out.t_final[pix] = T;
            if (out.n_contrib) out.n_contrib[pix] = cnt;
            out.n_iter[pix] = last;
        }
        if (!work) return;
        __syncthreads();
    }
}

// one reduction step of the transpose reduction: C live values -> C/2
template <int C, int O>
VPGS_D void tr_step(float (&v)[16], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        const float send = up ? v[i] : v[i + C / 2];
        const float keep = up ? v[i + C / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// sum v[0..9] over the warp and add the 10 totals to dst[0..9]
VPGS_D void warp_reduce_add10(float (&v)[16], float *dst, int lane) {
    tr_step<16, 16>(v, lane);
    tr_step<8, 8>(v, lane);
    tr_step<4, 4>(v, lane);
    tr_step<2, 2>(v, lane);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int slot = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    if (!(lane & 1) && slot < 10 && v[0] != 0.f) atomicAdd(dst + slot, v[0]);
}

__global__ void __launch_bounds__(1024)
composite_bwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, int n_tiles, CamParams cam, OptParams o,
                     const float *__restrict__ t_final, const int32_t *__restrict__ n_iter,
                     const float *__restrict__ dL_drgb, const float *__restrict__ dL_ddepth,
                     const float *__restrict__ dL_dalpha, float *__restrict__ g2d,
                     const uint32_t *status, uint32_t *work) {
    extern __shared__ float4 smem[];
    const int B = blockDim.x;
    float4 *s0 = smem, *s1 = smem + B, *s2 = smem + 2 * B;
    uint32_t *s_id = reinterpret_cast<uint32_t *>(smem + 3 * B);
    __shared__ int s_tile;
    __shared__ int s_max;
    if (*status != 0u) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f, pyl = (float)ly + 0.5f;
    int t = blockIdx.x;
    for (;;) {
        if (work) {
            if (tid == 0) s_tile = (int)atomicAdd(work, 1u);
            __syncthreads();
            t = s_tile;
        }
        if (tid == 0) s_max = 0;
        __syncthreads();
        if (t >= n_tiles) return;
        const TileCoord tc = tile_coord(t, cam);
        const int px = tc.tx * cam.tile_w + lx, py = tc.ty * cam.tile_h + ly;
        const bool inside = px < cam.W && py < cam.H;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const uint2 rg = ranges[t];
        const int start = (int)rg.x;
        const int64_t HW = (int64_t)cam.H * cam.W;
        const int64_t pix = (int64_t)tc.v * HW + (int64_t)py * cam.W + px;
        float T = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f;
        int last = 0;
        if (inside) {
            T = t_final[pix];
            last = n_iter[pix];
            if (dL_drgb) {
                const float *gp = dL_drgb + (int64_t)tc.v * 3 * HW + (int64_t)py * cam.W + px;
                gC0 = gp[0]; gC1 = gp[HW]; gC2 = gp[2 * HW];
            }
            if (dL_ddepth) gD = dL_ddepth[pix];
            if (dL_dalpha) gA = dL_dalpha[pix];
        }
        const float T_fin = T;
        float B0 = o.bg0, B1 = o.bg1, B2 = o.bg2, BD = 0.f;
        {
            int m = __reduce_max_sync(0xffffffffu, (unsigned)last);
            if (lane == 0 && m > 0) atomicMax(&s_max, m);
        }
        __syncthreads();
        const int list_end = start + min(s_max, (int)rg.y - start);  // n_iter never exceeds the list
        for (int b1 = list_end; b1 > start; b1 -= B) {
            const int b0 = max(start, b1 - B);
            __syncthreads();
            const int j = b0 + tid;
            if (j < b1) {
                const uint32_t id = ival[j];
                const Rec r = rec[id];
                s0[tid] = make_float4((r.r0.x - ox) + r.r0.z, (r.r0.y - oy) + r.r0.w, r.r1.x, r.r1.y);
                s1[tid] = make_float4(r.r1.z, r.r1.w, r.r2.x, r.r2.y);
                s2[tid] = make_float4(r.r2.z, r.r2.w, r.r3.x, 0.f);
                s_id[tid] = id;
            }
            __syncthreads();
            for (int k = b1 - b0 - 1; k >= 0; --k) {
                const int jj = b0 + k - start;
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
                bool act = jj < last;
                if (act) {
                    const float4 a = s0[k], b = s1[k];
                    const float dx = pxl - a.x, dy = pyl - a.y;
                    const PairEval e = eval_pair(dx, dy, a.z, a.w, b.x, b.y, b.z, o.alpha_max);
                    if (e.alpha < o.alpha_min) {
                        act = false;
                    } else {
                        const float4 c = s2[k];
                        const float om = 1.f - e.alpha;
                        T = T / om;
                        const float w = e.alpha * T;
                        v[6] = w * gC0;
                        v[7] = w * gC1;
                        v[8] = w * gC2;
                        v[9] = w * gD;
                        const float dA = (gC0 * (c.x - B0) + gC1 * (c.y - B1) + gC2 * (c.z - B2) +
                                          gD * (b.w - BD)) * T + gA * T_fin / om;
                        B0 = fmaf(e.alpha, c.x, om * B0);
                        B1 = fmaf(e.alpha, c.y, om * B1);
                        B2 = fmaf(e.alpha, c.z, om * B2);
                        BD = fmaf(e.alpha, b.w, om * BD);
                        if (b.z * e.G <= o.alpha_max) {
                            const float dpow = dA * e.alpha;
                            v[5] = dA * e.G;
                            v[0] = dpow * (a.z * e.t1 + b.x * e.t2);
                            v[1] = dpow * (a.w * e.t1 + b.y * e.t2);
                            v[2] = -0.5f * dpow * dx * dx;
                            v[3] = -dpow * dx * dy;
                            v[4] = -0.5f * dpow * dy * dy;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, act)) warp_reduce_add10(v, g2d + 10 * (int64_t)s_id[k], lane);
            }
        }
        if (!work) return;
        __syncthreads();
    }
}

static size_t comp_smem(int B, bool bwd) { return sizeof(float4) * 3 * B + (bwd ? sizeof(uint32_t) * B : 0); }

static int persistent_grid(const void *kernel, int B, size_t smem, int per_sm, int n_tiles) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, B, smem);
    if (occ <= 0) occ = 1;
    const int g = device_sm_count() * std::min(occ, per_sm);
    return std::min(g, n_tiles);
}

cudaError_t launch_composite_fwd(const RenderWs &ws, const uint32_t *ival, int V,
                                 const CamParams &cam, const OptParams &o, const vpgs_images &out,
                                 int persistent_ctas, cudaStream_t s) {
    const int B = cam.tile_w * cam.tile_h;
    const int n_tiles = V * cam.T;
    const size_t sm = comp_smem(B, false);
    uint32_t *work = nullptr;
    int grid = n_tiles;
    if (persistent_ctas > 0) {
        work = ws.counters + CNT_WORK;
        cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        grid = persistent_grid((const void *)composite_fwd_kernel, B, sm, persistent_ctas, n_tiles);
    }
    if (grid == 0) return cudaSuccess;
    if (sm > 48 * 1024)
        cudaFuncSetAttribute((const void *)composite_fwd_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    VPGS_LAUNCH("composite_fwd", s,
                composite_fwd_kernel<<<grid, B, sm, s>>>(ws.rec, ival, ws.ranges, n_tiles, cam, o, out,
                                                         ws.status, work));
    return cudaGetLastError();
}

cudaError_t launch_composite_bwd(const RenderWs &ws, const uint32_t *ival, int V,
                                 const CamParams &cam, const OptParams &o, const vpgs_images &fwd,
                                 const float *dL_drgb, const float *dL_ddepth,
                                 const float *dL_dalpha, int persistent_ctas, cudaStream_t s) {
    const int B = cam.tile_w * cam.tile_h;
    const int n_tiles = V * cam.T;
    const size_t sm = comp_smem(B, true);
    uint32_t *work = nullptr;
    int grid = n_tiles;
    if (persistent_ctas > 0) {
        work = ws.counters + CNT_WORK;
        cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        grid = persistent_grid((const void *)composite_bwd_kernel, B, sm, persistent_ctas, n_tiles);
    }
    if (grid == 0) return cudaSuccess;
    if (sm > 48 * 1024)
        cudaFuncSetAttribute((const void *)composite_bwd_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    VPGS_LAUNCH("composite_bwd", s,
                composite_bwd_kernel<<<grid, B, sm, s>>>(ws.rec, ival, ws.ranges, n_tiles, cam, o,
                                                         fwd.t_final, fwd.n_iter, dL_drgb, dL_ddepth,
                                                         dL_dalpha, ws.g2d, ws.status, work));
    return cudaGetLastError();
}

}  // namespace vpgs
