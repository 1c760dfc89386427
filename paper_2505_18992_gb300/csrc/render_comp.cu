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

// Each thread owns kPix pixels of its tile column: rows ly and ly + tile_h/kPix.
constexpr int kPix = 2;
constexpr int kMaxThreads = 512;

__global__ void __launch_bounds__(kMaxThreads)
composite_fwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, int n_tiles, CamParams cam, OptParams o,
                     vpgs_images out, const uint32_t *status, uint32_t *work) {
    extern __shared__ float4 smem[];
    const int NT = blockDim.x;
    float4 *s0 = smem, *s1 = smem + NT, *s2 = smem + 2 * NT;
    __shared__ int s_tile;
    if (*status != 0u) return;
    const int tid = threadIdx.x;
    const int half = cam.tile_h / kPix;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f;
    float pyl[kPix];
#pragma unroll
    for (int q = 0; q < kPix; ++q) pyl[q] = (float)(ly + q * half) + 0.5f;
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
        const int px = tc.tx * cam.tile_w + lx;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const uint2 rg = ranges[t];
        const int start = (int)rg.x, end = (int)rg.y;
        float T[kPix], C0[kPix], C1[kPix], C2[kPix], D[kPix];
        int cnt[kPix], last[kPix];
        bool done[kPix];
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            T[q] = 1.f; C0[q] = C1[q] = C2[q] = D[q] = 0.f; cnt[q] = 0; last[q] = 0;
            const int py = tc.ty * cam.tile_h + ly + q * half;
            done[q] = !(px < cam.W && py < cam.H);
        }
        bool all_done = done[0] && done[1];
        for (int b0 = start; b0 < end; b0 += NT) {
            if (__syncthreads_count(all_done) == NT) break;
            const int j = b0 + tid;
            if (j < end) {
                const Rec r = rec[ival[j]];
                s0[tid] = make_float4((r.r0.x - ox) + r.r0.z, (r.r0.y - oy) + r.r0.w, r.r1.x, r.r1.y);
                s1[tid] = make_float4(r.r1.z, r.r1.w, r.r2.x, r.r2.y);
                s2[tid] = make_float4(r.r2.z, r.r2.w, r.r3.x, 0.f);
            }
            __syncthreads();
            if (!all_done) {
                const int nb = min(NT, end - b0);
                for (int k = 0; k < nb; ++k) {
                    const float4 a = s0[k], b = s1[k];
#pragma unroll
                    for (int q = 0; q < kPix; ++q) {
                        if (done[q]) continue;
                        const PairEval e = eval_pair(pxl - a.x, pyl[q] - a.y, a.z, a.w, b.x, b.y, b.z, o.alpha_max);
                        if (e.alpha < o.alpha_min) continue;
                        const float nt = T[q] * (1.f - e.alpha);
                        if (nt < o.t_min) {
                            done[q] = true;
                            continue;
                        }
                        const float w = e.alpha * T[q];
                        const float4 c = s2[k];
                        C0[q] = fmaf(w, c.x, C0[q]);
                        C1[q] = fmaf(w, c.y, C1[q]);
                        C2[q] = fmaf(w, c.z, C2[q]);
                        D[q] = fmaf(w, b.w, D[q]);
                        T[q] = nt;
                        ++cnt[q];
                        last[q] = b0 + k - start + 1;
                    }
                    if (done[0] && done[1]) {
                        all_done = true;
                        break;
                    }
                }
            }
        }
        const int64_t HW = (int64_t)cam.H * cam.W;
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            const int py = tc.ty * cam.tile_h + ly + q * half;
            if (!(px < cam.W && py < cam.H)) continue;
            const int64_t pix = (int64_t)tc.v * HW + (int64_t)py * cam.W + px;
            if (out.rgb) {
                float *rgb = out.rgb + (int64_t)tc.v * 3 * HW + (int64_t)py * cam.W + px;
                rgb[0] = fmaf(T[q], o.bg0, C0[q]);
                rgb[HW] = fmaf(T[q], o.bg1, C1[q]);
                rgb[2 * HW] = fmaf(T[q], o.bg2, C2[q]);
            }
            if (out.depth) out.depth[pix] = D[q];
            if (out.alpha) out.alpha[pix] = 1.f - T[q];
            out.t_final[pix] = T[q];
            if (out.n_contrib) out.n_contrib[pix] = cnt[q];
            out.n_iter[pix] = last[q];
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

// sum v[0..9] over the warp; lanes 0,2,..,18 end up holding the totals of slots 0..9
VPGS_D int warp_reduce10(float (&v)[16], int lane) {
    tr_step<16, 16>(v, lane);
    tr_step<8, 8>(v, lane);
    tr_step<4, 4>(v, lane);
    tr_step<2, 2>(v, lane);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int slot = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    return (lane & 1) ? 16 : slot;
}

constexpr int kPartStride = 11;  // floats per (warp, Gaussian) partial, padded against bank conflicts

__global__ void __launch_bounds__(kMaxThreads)
composite_bwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, int n_tiles, CamParams cam, OptParams o,
                     const float *__restrict__ t_final, const int32_t *__restrict__ n_iter,
                     const float *__restrict__ dL_drgb, const float *__restrict__ dL_ddepth,
                     const float *__restrict__ dL_dalpha, float *__restrict__ g2d,
                     const uint32_t *status, uint32_t *work) {
    extern __shared__ float4 smem[];
    const int NT = blockDim.x;
    const int NW = NT >> 5;
    float4 *s0 = smem, *s1 = smem + NT, *s2 = smem + 2 * NT;
    uint32_t *s_id = reinterpret_cast<uint32_t *>(smem + 3 * NT);
    float *s_part = reinterpret_cast<float *>(s_id + NT);  // [NW][NT][kPartStride]
    __shared__ int s_tile;
    __shared__ int s_max;
    if (*status != 0u) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = cam.tile_h / kPix;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f;
    float pyl[kPix];
#pragma unroll
    for (int q = 0; q < kPix; ++q) pyl[q] = (float)(ly + q * half) + 0.5f;
    float *my_part = s_part + (size_t)warp * NT * kPartStride;
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
        const int px = tc.tx * cam.tile_w + lx;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const uint2 rg = ranges[t];
        const int start = (int)rg.x;
        const int64_t HW = (int64_t)cam.H * cam.W;
        float T[kPix], T_fin[kPix], gC0[kPix], gC1[kPix], gC2[kPix], gD[kPix], gA[kPix];
        float B0[kPix], B1[kPix], B2[kPix], BD[kPix];
        int last[kPix];
        int my_max = 0;
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            T[q] = 1.f; gC0[q] = gC1[q] = gC2[q] = gD[q] = gA[q] = 0.f; last[q] = 0;
            B0[q] = o.bg0; B1[q] = o.bg1; B2[q] = o.bg2; BD[q] = 0.f;
            const int py = tc.ty * cam.tile_h + ly + q * half;
            if (px < cam.W && py < cam.H) {
                const int64_t pix = (int64_t)tc.v * HW + (int64_t)py * cam.W + px;
                T[q] = t_final[pix];
                last[q] = n_iter[pix];
                if (dL_drgb) {
                    const float *gp = dL_drgb + (int64_t)tc.v * 3 * HW + (int64_t)py * cam.W + px;
                    gC0[q] = gp[0]; gC1[q] = gp[HW]; gC2[q] = gp[2 * HW];
                }
                if (dL_ddepth) gD[q] = dL_ddepth[pix];
                if (dL_dalpha) gA[q] = dL_dalpha[pix];
            }
            T_fin[q] = T[q];
            my_max = max(my_max, last[q]);
        }
        // the warp's own list length: warps whose pixels stop early skip the tail
        const int warp_max = (int)__reduce_max_sync(0xffffffffu, (unsigned)my_max);
        if (lane == 0 && warp_max > 0) atomicMax(&s_max, warp_max);
        __syncthreads();
        const int list_end = start + min(s_max, (int)rg.y - start);  // n_iter never exceeds the list
        for (int b1 = list_end; b1 > start; b1 -= NT) {
            const int b0 = max(start, b1 - NT);
            const int nb = b1 - b0;
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
            for (int e = lane; e < nb * kPartStride; e += 32) my_part[e] = 0.f;
            __syncthreads();
            const int k_end = min(nb, warp_max - (b0 - start));  // warp-uniform
            for (int k = k_end - 1; k >= 0; --k) {
                const int jj = b0 + k - start;
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
                bool act_any = false;
                const float4 a = s0[k], b = s1[k];
#pragma unroll
                for (int q = 0; q < kPix; ++q) {
                    if (jj >= last[q]) continue;
                    const float dx = pxl - a.x, dy = pyl[q] - a.y;
                    const PairEval e = eval_pair(dx, dy, a.z, a.w, b.x, b.y, b.z, o.alpha_max);
                    if (e.alpha < o.alpha_min) continue;
                    act_any = true;
                    const float4 c = s2[k];
                    const float om = 1.f - e.alpha;
                    T[q] = T[q] / om;
                    const float w = e.alpha * T[q];
                    v[6] = fmaf(w, gC0[q], v[6]);
                    v[7] = fmaf(w, gC1[q], v[7]);
                    v[8] = fmaf(w, gC2[q], v[8]);
                    v[9] = fmaf(w, gD[q], v[9]);
                    const float dA = (gC0[q] * (c.x - B0[q]) + gC1[q] * (c.y - B1[q]) + gC2[q] * (c.z - B2[q]) +
                                      gD[q] * (b.w - BD[q])) * T[q] + gA[q] * T_fin[q] / om;
                    B0[q] = fmaf(e.alpha, c.x, om * B0[q]);
                    B1[q] = fmaf(e.alpha, c.y, om * B1[q]);
                    B2[q] = fmaf(e.alpha, c.z, om * B2[q]);
                    BD[q] = fmaf(e.alpha, b.w, om * BD[q]);
                    if (b.z * e.G <= o.alpha_max) {
                        const float dpow = dA * e.alpha;
                        v[5] = fmaf(dA, e.G, v[5]);
                        v[0] = fmaf(dpow, a.z * e.t1 + b.x * e.t2, v[0]);
                        v[1] = fmaf(dpow, a.w * e.t1 + b.y * e.t2, v[1]);
                        v[2] = fmaf(-0.5f * dpow, dx * dx, v[2]);
                        v[3] = fmaf(-dpow, dx * dy, v[3]);
                        v[4] = fmaf(-0.5f * dpow, dy * dy, v[4]);
                    }
                }
                if (__any_sync(0xffffffffu, act_any)) {
                    const int slot = warp_reduce10(v, lane);
                    if (slot < 10) my_part[k * kPartStride + slot] = v[0];
                }
            }
            __syncthreads();
            // one thread per Gaussian of the batch: sum the warps, one atomic per value
            for (int k = tid; k < nb; k += NT) {
                float *dst = g2d + 10 * (int64_t)s_id[k];
#pragma unroll
                for (int slot = 0; slot < 10; ++slot) {
                    float acc = 0.f;
                    for (int w = 0; w < NW; ++w) acc += s_part[((size_t)w * NT + k) * kPartStride + slot];
                    if (acc != 0.f) atomicAdd(dst + slot, acc);
                }
            }
        }
        if (!work) return;
        __syncthreads();
    }
}

static size_t comp_smem(int NT, bool bwd) {
    return sizeof(float4) * 3 * NT +
           (bwd ? sizeof(uint32_t) * NT + sizeof(float) * (size_t)(NT / 32) * NT * kPartStride : 0);
}

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
    const int B = cam.tile_w * cam.tile_h / kPix;
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
    const int B = cam.tile_w * cam.tile_h / kPix;
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
