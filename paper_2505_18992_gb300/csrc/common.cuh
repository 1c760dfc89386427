// Internal definitions shared by the CUDA translation units of libvpgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "../../include/vpgs.h"

#define VPGS_HD __host__ __device__ __forceinline__
#define VPGS_D __device__ __forceinline__

// Compositing launch geometry (compile-time tuning knobs):
//   VPGS_PIX    pixels per thread: VPGS_PIX adjacent rows of one column
#ifndef VPGS_PIX
#define VPGS_PIX 2
#endif
//   VPGS_BWD_ACC how the backward combines per-warp sums of a Gaussian's 2D
//                gradient: 0 = one global atomic per warp, 1 = per-warp shared
//                slots summed per batch, 2 = shared-memory atomics per batch,
//                -1 = by the tile's warps (1 from 2 warps per tile up, 0 for a
//                one-warp tile, which has no warps' sums to combine).  0 by
//                default: with batches of 256 records (render_comp.cu,
//                VPGS_BWD_BATCH) the shared slots of 1 and 2 would cost resident
//                blocks
#ifndef VPGS_BWD_ACC
#define VPGS_BWD_ACC 0
#endif
//   VPGS_DEPTH_SORT_GRID, VPGS_OFFSET_SCAN_GRID  blocks per SM of the depth
//                sort's passes and of the instance-offset scan (0: what is
//                resident).  Their item count, the visible pairs, is usually far
//                below the capacity (every pair visible) that the resident grid
//                is sized for, and every block past the last tile still
//                launches, takes a ticket and leaves
#ifndef VPGS_DEPTH_SORT_GRID
#define VPGS_DEPTH_SORT_GRID 2
#endif
#ifndef VPGS_OFFSET_SCAN_GRID
#define VPGS_OFFSET_SCAN_GRID 2
#endif
//   VPGS_BWD_RCP 1: the backward takes one approximate reciprocal of 1 - alpha
//                per blended pair (relative error ~1e-7 per step), 0: IEEE divisions
#ifndef VPGS_BWD_RCP
#define VPGS_BWD_RCP 1
#endif

namespace vpgs {

constexpr int kWarp = 32;

// A launch-geometry value that depends only on the device (an occupancy, a grid
// size): computed by f() once per device ordinal and kept in `cache` (zero-
// initialised, one slot per ordinal); ordinals beyond the cache compute it on
// every call.  Safe to call from several host threads.
constexpr int kDeviceCache = 64;
template <typename F>
int per_device(std::atomic<int> (&cache)[kDeviceCache], F f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    if (dev >= 0 && dev < kDeviceCache) {
        const int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
        const int w = std::max(f(), 1);
        cache[dev].store(w, std::memory_order_relaxed);
        return w;
    }
    return std::max(f(), 1);
}

// ---------------------------------------------------------------------------
// status word: the first error wins (atomicCAS from OK)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// programmatic dependent launch (VPGS_PDL: 0 off, 1 the render kernels are
// launched so that they may be scheduled while their predecessor finishes,
// 2 and they also let their own successor be scheduled at once).  Every such
// kernel starts with grid_dep_enter(), which waits for the predecessor grid to
// complete and its memory to be visible before anything else runs.
// ---------------------------------------------------------------------------
#ifndef VPGS_PDL
#define VPGS_PDL 1
#endif
VPGS_D void grid_dep_enter() {
#if VPGS_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#if VPGS_PDL >= 2
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
#endif
}

// Kernel launch used by the render path: with VPGS_PDL the launch allows
// programmatic stream serialisation (the kernel must begin with
// grid_dep_enter()); errors surface through cudaGetLastError as for <<< >>>.
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
#if VPGS_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
#else
    k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return cudaSuccess;
#endif
}

VPGS_D void set_status(uint32_t *status, uint32_t code) {
    atomicCAS(status, (uint32_t)VPGS_OK, code);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations per Dekker / Knuth (TwoSum), with the product
// error taken by one fused multiply-add.  Used where FP32 rounding of a pixel
// position (~1e-4 px at u ~ 1000) would be visible in alpha.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

VPGS_D df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
VPGS_D df quick_two_sum(float a, float b) {  // requires |a| >= |b|
    float s = a + b;
    return {s, b - (s - a)};
}
VPGS_D df two_prod(float a, float b) {
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}
VPGS_D df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    return quick_two_sum(s.hi, e);
}
VPGS_D df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
VPGS_D df df_div(df a, df b) {
    float q1 = a.hi / b.hi;
    df qb = df_mul_f(b, q1);
    df r = df_add(a, df{-qb.hi, -qb.lo});
    float q2 = r.hi / b.hi;
    return quick_two_sum(q1, q2);
}
VPGS_D df df_from_double(double x) {
    float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// ---------------------------------------------------------------------------
// camera pose in the two precisions the kernels use
// ---------------------------------------------------------------------------
struct PoseDF {
    df R[9];
    df t[3];
};

// T (float64 [4,4]) -> 24 floats: R[9] and t[3] as (hi, lo) pairs.  Done once
// per view and call; FP64 is far too slow on this part to convert per Gaussian.
VPGS_D void pose_to_df(const double *T, float *out) {
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            const df x = df_from_double(T[4 * r + c]);
            out[2 * (3 * r + c)] = x.hi;
            out[2 * (3 * r + c) + 1] = x.lo;
        }
        const df x = df_from_double(T[4 * r + 3]);
        out[18 + 2 * r] = x.hi;
        out[18 + 2 * r + 1] = x.lo;
    }
}

VPGS_D void load_pose(const float *pd, PoseDF &P) {
#pragma unroll
    for (int k = 0; k < 9; ++k) P.R[k] = df{__ldg(pd + 2 * k), __ldg(pd + 2 * k + 1)};
#pragma unroll
    for (int r = 0; r < 3; ++r) P.t[r] = df{__ldg(pd + 18 + 2 * r), __ldg(pd + 19 + 2 * r)};
}

// p_c = R mu + t in double-float, mu exact float32
VPGS_D void transform_df(const PoseDF &P, float mx, float my, float mz, df out[3]) {
    const float m[3] = {mx, my, mz};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        df acc = P.t[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            df p = two_prod(P.R[3 * r + c].hi, m[c]);
            p.lo = fmaf(P.R[3 * r + c].lo, m[c], p.lo);
            acc = df_add(acc, p);
        }
        out[r] = acc;
    }
}

// rotation matrix of q / |q|, q = (w, x, y, z)
VPGS_D void quat_to_rot(float w, float x, float y, float z, float R[9]) {
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// ---------------------------------------------------------------------------
// per-(view, Gaussian) screen-space record: 4 x float4 = 64 bytes
//   r0 = (u_hi, v_hi, u_lo, v_lo)   image mean as a double-float pair
//   r1 = (w1x, w1y, w2x, w2y)       whitening rows times sqrt(log2(e)/2):
//                                   (w1.d)^2 + (w2.d)^2 = log2(e)/2 d^T Sigma'^-1 d
//   r2 = (opacity, z, r, g)
//   r3 = (b, w2x_lo, +-ry, w2y_lo)  ry: conservative pixel half-extent in y (alpha >=
//                                   alpha_min is impossible farther than this from the
//                                   mean), negative for a near-degenerate Gaussian, whose
//                                   second whitening row is the double-float pair
//                                   (w2x + w2x_lo, w2y + w2y_lo) (zero low parts otherwise)
// The whitening rows are the eigenvectors of Sigma' scaled by 1/sqrt(lambda) (and
// by sqrt(log2(e)/2), so that alpha needs a single ex2),
// which evaluates the quadratic form without the cancellation the
// (a dx^2 + 2 b dx dy + c dy^2) form suffers on elongated Gaussians.
// ---------------------------------------------------------------------------
struct __align__(16) Rec {
    float4 r0, r1, r2, r3;
};

// evaluated per pixel/Gaussian pair, bit-identically in forward and backward
struct PairEval {
    float t1, t2, G, alpha;
};

// exp(-q/2) = 2^(-q log2(e)/2): the factor rides in the whitening rows
constexpr float kRowScale = 0.84932180028801907f;     // sqrt(log2(e) / 2)
constexpr float kInvExp2Half = 1.38629436111989061f;  // 2 ln 2

VPGS_D float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha of a near-degenerate record at pixel (px, py): d = (px - ux - rx, py - uy - ry) in
// double-float (ux, uy the staged tile-local mean, (rx, ry) its rounding
// residual) and t2 = w2 . d with w2 = (w2x + w2x_lo, w2y + w2y_lo) as an
// error-free dot product of the high parts plus the low-order terms; t1 stays
// FP32 (its error is not amplified by the condition number).
VPGS_D PairEval eval_pair_fine(float px, float py, float ux, float uy, float rx, float ry, float w1x, float w1y,
                               float w2x, float w2y, float w2x_lo, float w2y_lo, float opac, float alpha_max) {
    df dx = two_sum(px, -ux), dy = two_sum(py, -uy);
    dx.lo -= rx;
    dy.lo -= ry;
    PairEval e;
    e.t1 = fmaf(w1x, dx.hi, w1y * dy.hi);
    const df p1 = two_prod(w2x, dx.hi), p2 = two_prod(w2y, dy.hi);
    const df sh = two_sum(p1.hi, p2.hi);
    float lo = sh.lo + (p1.lo + p2.lo);
    lo = fmaf(w2x, dx.lo, lo);
    lo = fmaf(w2y, dy.lo, lo);
    lo = fmaf(w2x_lo, dx.hi, lo);
    lo = fmaf(w2y_lo, dy.hi, lo);
    e.t2 = sh.hi + lo;
    e.G = ex2_approx(-fmaf(e.t1, e.t1, e.t2 * e.t2));
    e.alpha = fminf(alpha_max, opac * e.G);
    return e;
}

// ---------------------------------------------------------------------------
// Tile cover.  A Gaussian is listed in a tile when its alpha_min ellipse
// d^T Sigma'^-1 d <= kq (kq = 2 ln(o / alpha_min)) meets the rectangle of the
// tile's pixel centres widened by the extent margins (mx, my).  With
// Sigma' = [[A, B], [B, C]] the ellipse at row offset y spans
//   x = beta y -/+ sqrt(g1 - g2 y^2),  beta = B/C, g1 = kq det/C, g2 = det/C^2,
// for |y| <= ry = sqrt(kq C); its leftmost point sits at y = yL = -B sqrt(kq/A)
// and its rightmost at -yL.  x_min(y) is convex and x_max(y) concave, so over a
// band of rows the x extent is reached at yL (resp. -yL) clamped into the band.
// The counting pass (preprocess) stores the spans themselves when the box has
// at most kCoverRows tile rows, else these parameters; the emitting pass then
// walks the rows with the same function in round-to-nearest intrinsics, so
// both see identical spans.
// ---------------------------------------------------------------------------
constexpr int kCoverRows = 8;
struct Cover {
    float4 a;  // ry, my, yL, beta          | packed spans of rows 0-3
    float4 b;  // g1, g2, mx, 0             | packed spans of rows 4-7
};
// packed span of one tile row: first tile column | last << 16 (first > last: empty)
constexpr uint32_t kEmptySpan = 0xffffu;

// What the emitting pass needs of one visible (view, Gaussian), in one 64-byte
// record: a single aligned gather per Gaussian.
struct __align__(16) BinRec {
    float4 uv;     // (u_hi, v_hi, u_lo, v_lo)
    uint2 rect;    // (tx0 | tx1 << 16, ty0 | ty1 << 16): bounding box in tiles
    uint32_t cnt;  // tiles of the cover
    uint32_t pad;
    Cover cv;
};

// Tile columns [x, y] of tile row ty (x > y: none) within [tx_lo, tx_hi].
VPGS_D int2 cover_row(const Cover &cv, float u_hi, float u_lo, float v_hi, float v_lo, int ty, int tx_lo,
                      int tx_hi, int tw_shift, int tile_h, int W, int H) {
    const int y_first = ty * tile_h;
    const int y_last = min(y_first + tile_h, H) - 1;
    float ya = __fsub_rn(__fsub_rn(__fsub_rn((float)y_first + 0.5f, v_hi), v_lo), cv.a.y);
    float yb = __fadd_rn(__fsub_rn(__fsub_rn((float)y_last + 0.5f, v_hi), v_lo), cv.a.y);
    ya = fmaxf(ya, -cv.a.x);
    yb = fminf(yb, cv.a.x);
    if (!(ya <= yb)) return make_int2(1, 0);
    const float yl = fminf(fmaxf(cv.a.z, ya), yb);
    const float yr = fminf(fmaxf(-cv.a.z, ya), yb);
    const float wl = __fsqrt_rn(fmaxf(__fsub_rn(cv.b.x, __fmul_rn(cv.b.y, __fmul_rn(yl, yl))), 0.f));
    const float wr = __fsqrt_rn(fmaxf(__fsub_rn(cv.b.x, __fmul_rn(cv.b.y, __fmul_rn(yr, yr))), 0.f));
    const float xmin = __fsub_rn(__fsub_rn(__fmul_rn(cv.a.w, yl), wl), cv.b.z);
    const float xmax = __fadd_rn(__fadd_rn(__fmul_rn(cv.a.w, yr), wr), cv.b.z);
    const float u0 = __fsub_rn(u_hi, 0.5f);
    const float lx = fmaxf(__fadd_rn(__fadd_rn(u0, xmin), u_lo), -1.f);
    const float hx = fminf(__fadd_rn(__fadd_rn(u0, xmax), u_lo), (float)W);
    const int x0 = max(0, (int)ceilf(lx)), x1 = min(W - 1, (int)floorf(hx));
    if (x0 > x1) return make_int2(1, 0);
    return make_int2(max(x0 >> tw_shift, tx_lo), min(x1 >> tw_shift, tx_hi));
}

// ---------------------------------------------------------------------------
// Workspace of a render call.  All pointers are carved from one caller buffer.
// ---------------------------------------------------------------------------
struct RenderLayout {
    int64_t N;          // Gaussian capacity
    int32_t V;          // views
    int32_t tiles_x, tiles_y, T;  // tiles per view
    int64_t VN;         // V * N
    int64_t M_cap;      // instance capacity
    int32_t tile_bits;  // bits of a global tile id
    // offsets in bytes
    size_t off_status, off_counters, off_rec, off_tcount, off_dkey0,
        off_dval0, off_dkey1, off_dval1, off_ikey0, off_ival0, off_ikey1, off_ival1, off_ranges,
        off_sort_hist, off_sort_look, off_sort_look_t, off_scan_look, off_g2d, off_posedf, off_bin,
        off_vis_idx, off_tile_order, off_tile_work, total;
    int64_t sort_blocks_max, scan_blocks_max;
};

// counters[] slots
enum {
    CNT_VISIBLE = 0,   // number of visible (view, Gaussian) pairs
    CNT_INSTANCES = 1, // number of tile instances
    CNT_TICKET_A = 2,  // decoupled look-back tickets: visibility scan
    CNT_TICKET_O = 3,  // instance-offset scan
    CNT_TICKET_D = 4,  // 4..7: depth sort passes
    CNT_TICKET_T = 8,  // 8..11: tile sort passes
    CNT_WORK = 12,     // persistent-kernel work queue
    CNT_CAND = 13,     // pre-cull survivors of the projection pass
    CNT_N = 16         // all zeroed by the prepare kernel at the start of a call
};

struct RenderWs {
    uint32_t *status;
    uint32_t *counters;
    Rec *rec;
    uint32_t *tcount;
    uint32_t *dkey[2], *dval[2];
    uint32_t *ikey[2], *ival[2];
    uint2 *ranges;
    uint32_t *sort_hist[2];            // depth / tile sort: [passes][256] global digit histograms
    uint32_t *sort_look[2];            // depth / tile sort: [passes][tiles][256] look-back words
    unsigned long long *scan_look[2];  // visibility / offset scan: look-back words
    float *g2d;           // [VN,10] 2D gradient sums: u, v, conic a, b, c (without their
                          // constant factors), opacity, r, g, b, z
    float *posedf;        // [V,24] poses as double-float pairs
    BinRec *bin;          // [VN] binning records of visible Gaussians
    uint32_t *vis_idx;    // [VN] visible (view, Gaussian) indices in index order
    uint32_t *tile_order; // [V*T] global tile ids, most work first (compositing launch order)
    uint32_t *tile_work;  // [V*T] the backward's list steps per tile (the forward's largest n_iter)
};

// radix sort geometry
constexpr int kSortThreads = 256;
#ifndef VPGS_DEPTH_SORT_ITEMS
#define VPGS_DEPTH_SORT_ITEMS 4
#endif
#ifndef VPGS_TILE_SORT_ITEMS
#define VPGS_TILE_SORT_ITEMS 16
#endif
constexpr int kDepthSortItems = VPGS_DEPTH_SORT_ITEMS;  // keys per thread in the depth sort (<= 16)
static_assert(kDepthSortItems <= 16, "the depth sort's look-back space must cover the 16-key form");
constexpr int kTileSortItems = VPGS_TILE_SORT_ITEMS;    // keys per thread in the tile-id sort
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxSortPasses = 8;

// compositing launch order: 1 = tiles with the most instances first (a
// bucketed counting sort after the tile ranges), 0 = tile-id order
#ifndef VPGS_TILE_ORDER
#define VPGS_TILE_ORDER 1
#endif
// backward launch order: 1 = by the steps each tile's backward walks (the
// largest n_iter of its pixels, from the forward), 0 = by instance count
#ifndef VPGS_BWD_ORDER_NITER
#define VPGS_BWD_ORDER_NITER 1
#endif

// scan geometry
constexpr int kScanThreads = 256;
#ifndef VPGS_SCAN_ITEMS
#define VPGS_SCAN_ITEMS 4
#endif
constexpr int kScanItems = VPGS_SCAN_ITEMS;  // items per thread of a scan tile
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kScanItemsWide = 8;  // the same for scans of many millions of items
static_assert(kScanItemsWide >= kScanItems, "look-back space is sized for the narrower tiles");

// bounded spin for decoupled look-back: the predecessor always holds an
// earlier ticket and is therefore resident, so this bound is never reached in
// a healthy run; reaching it records VPGS_ERR_TIMEOUT and the kernel goes on.
constexpr int kSpinLimit = 1 << 22;

}  // namespace vpgs
