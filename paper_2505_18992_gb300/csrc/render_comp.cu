// Front-to-back alpha compositing per tile, and its backward pass.
//
// One CTA renders one tile (tile_w x tile_h threads, one pixel each), or, in
// persistent mode, a fixed number of CTAs per SM pull tiles from a work queue.
// The tile's depth-ordered Gaussian list is staged through shared memory in
// batches of one record per thread; each pixel walks the batch in order:
//   alpha = min(alpha_max, o 2^-((w1.d)^2 + (w2.d)^2)), d = pixel - mean, with
//           the whitening rows w scaled by sqrt(log2(e)/2) when the record is made
//   skip alpha < alpha_min; stop before T (1 - alpha) < t_min
// Each warp first compacts the staged batch into its own list of the Gaussians
// whose widened y extent reaches one of the warp's pixel rows (at the others
// alpha < alpha_min at every pixel of the warp), then walks only that list.
//   C += alpha T c, D += alpha T z, T *= 1 - alpha
// Means are made tile-local when staged ((u_hi - x0) + u_lo), so d keeps
// ~1e-7 px accuracy anywhere in the image.
//
// The backward pass walks the same list from the back, recovering T_i as
// T_{i+1} / (1 - alpha_i), and keeps the colour/depth "behind" each Gaussian,
//   B <- alpha c + (1 - alpha) B   (B starts at the background),
// giving dC/dalpha_i = T_i (c_i - B_i), dA/dalpha_i = T_final / (1 - alpha_i).
// Only g . B enters dL/dalpha (g the pixel's upstream gradient), so each pixel
// carries that scalar instead of B.
// Per-Gaussian 2D gradient sums of a warp (in the Gaussian's whitened frame
// t = W d: sum dpow t1, sum dpow t2, sum dpow t1^2, sum dpow t1 t2, sum dpow
// t2^2; then opacity, rgb, z) are summed by a transpose reduction (12 shuffles
// for 10 values) and added with one atomic per value per warp.
// Near-degenerate records (negative y half extent) take the double-float pair
// evaluation (eval_pair_fine): one warp-uniform branch per list entry.
#include <type_traits>

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

// Each thread owns kPix pixels of its tile column: rows kPix*ly .. kPix*ly + kPix - 1.
constexpr int kPix = VPGS_PIX;
#ifndef VPGS_BWD_DIRECT
#define VPGS_BWD_DIRECT 2
#endif
constexpr int kDirect = VPGS_BWD_DIRECT;  // at most this many active lanes: per-lane atomics, no reduction
constexpr int kMaxThreads = 512;
#ifndef VPGS_FWD_BATCH
#define VPGS_FWD_BATCH 2  // records each forward thread stages per batch
#endif
constexpr int kFwdBatch = VPGS_FWD_BATCH;
#ifndef VPGS_BWD_BATCH
#define VPGS_BWD_BATCH 2  // records each backward thread stages per batch
#endif
constexpr int kBwdBatch = VPGS_BWD_BATCH;
// list entries whose alphas the forward evaluates before blending them
#ifndef VPGS_FWD_WALK
#define VPGS_FWD_WALK 2
#endif
constexpr int kWalk = VPGS_FWD_WALK;

// Centre and half height of the band of tile-local pixel-centre rows held by
// this thread's warp.
VPGS_D float2 warp_rows(const float (&pyl)[kPix]) {
    float lo = pyl[0], hi = pyl[kPix - 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    return make_float2(0.5f * (lo + hi), 0.5f * (hi - lo));
}

// Whether a staged (plain) Gaussian can reach alpha_min at a pixel centre of
// the tile-local box [x0, x1] x [y0, y1]: the minimum over the box of the
// whitened square distance q = |W d|^2, d = p - mean, against log2(o /
// alpha_min) (alpha = o 2^-q).  The minimum of the convex q lies inside the box
// (then 0) or on an edge, where q is a quadratic in one variable.  The bound
// is widened by 0.1 % + 1e-3 so that every pixel the FP32 per-pixel evaluation
// would blend stays listed.
VPGS_D bool reaches_box(const float4 &a, const float4 &b, float x0, float x1, float y0, float y1,
                        float lg_amin) {
    const float A = fmaf(a.z, a.z, b.x * b.x), B = fmaf(a.z, a.w, b.x * b.y), C = fmaf(a.w, a.w, b.y * b.y);
    if (!(A > 0.f && C > 0.f)) return true;
    const float dx0 = x0 - a.x, dx1 = x1 - a.x, dy0 = y0 - a.y, dy1 = y1 - a.y;
    if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
    auto q = [&](float dx, float dy) { return fmaf(A * dx, dx, fmaf(2.f * B * dx, dy, C * dy * dy)); };
    const float ra = -B / A, rc = -B / C;
    float m = q(fminf(fmaxf(ra * dy0, dx0), dx1), dy0);
    m = fminf(m, q(fminf(fmaxf(ra * dy1, dx0), dx1), dy1));
    m = fminf(m, q(dx0, fminf(fmaxf(rc * dx0, dy0), dy1)));
    m = fminf(m, q(dx1, fminf(fmaxf(rc * dx1, dy0), dy1)));
    const float level = __log2f(b.z) - lg_amin;
    return !(m > fmaf(1e-3f, fabsf(level), level) + 1e-3f);
}

// Compacts the batch positions [0, n) whose Gaussian reaches the warp's pixel
// rows into list, in ascending order; returns how many (warp-uniform).  A
// Gaussian is listed when its widened y extent reaches the rows and, with
// kExact and a plain record, its alpha_min ellipse also meets the rows' pixel
// centres within the tile's columns [0.5, xmax].  All 32 lanes take part.
// `fine` tells (warp-uniform) whether a listed record is near-degenerate.
// Both forms list every Gaussian that blends into a pixel of the rows, so the
// forward (y extent alone: the exact test costs it more than it saves) and the
// backward (exact) may differ in what they skip but not in what they blend.
template <bool kExact>
VPGS_D int warp_list(const float4 *s0, const float4 *s1, int n, float2 band, uint16_t *list, int lane,
                     bool &fine, float xmax, float lg_amin) {
    const uint32_t below = (1u << lane) - 1u;
    int cnt = 0;
    bool any = false;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int k = c0 + lane;
        bool touch = false, f = false;
        if (k < n) {
            const float4 a = s0[k], b = s1[k];
            const float ry = b.w;
            touch = fabsf(a.y - band.x) <= fabsf(ry) + band.y;
            f = touch && ry < 0.f;
            if (kExact && touch && !f) touch = reaches_box(a, b, 0.5f, xmax, band.x - band.y, band.x + band.y, lg_amin);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, touch);
        any |= __any_sync(0xffffffffu, f);
        if (touch) list[cnt + __popc(m & below)] = (uint16_t)k;
        cnt += __popc(m);
    }
    __syncwarp();
    fine = any;
    return cnt;
}

// record -> shared staging: s0 = (u, v) tile-local, w1; s1 = w2, opacity, widened
// y half extent (negative: near-degenerate); s2 = colour, camera z.  The
// forward also stages fine_extra of a near-degenerate record (s3); the
// backward, whose shared memory sets its occupancy, reads it from the record.
// what a near-degenerate record adds to its staged a = (ux, uy, ...): the
// rounding residual of the tile-local mean ((u_hi - ox) + u_lo = ux + residual,
// the subtraction split exactly) and the low parts of w2
VPGS_D float4 fine_extra(const Rec &r, float ox, float oy, float ux, float uy) {
    const df ex = two_sum(r.r0.x, -ox), ey = two_sum(r.r0.y, -oy);
    return make_float4(((ex.hi - ux) + r.r0.z) + ex.lo, ((ey.hi - uy) + r.r0.w) + ey.lo, r.r3.y, r.r3.w);
}

VPGS_D void stage(const Rec &r, float ox, float oy, float4 &a, float4 &b, float4 &c) {
    a = make_float4((r.r0.x - ox) + r.r0.z, (r.r0.y - oy) + r.r0.w, r.r1.x, r.r1.y);
    b = make_float4(r.r1.z, r.r1.w, r.r2.x, r.r3.z);
    c = make_float4(r.r2.z, r.r2.w, r.r3.x, r.r2.y);
}

// alpha of the thread's pixel q (tile-local (px, py)) for the staged Gaussian
// (a, b[, f]).  A thread's pixels are kPix consecutive rows of one column, so in
// the plain form the whitened coordinates of row q are those of its first row
// (t1_0, t2_0) plus q times the rows' y coefficients (w1y, w2y); the
// near-degenerate form evaluates each row in double-float.
template <bool kFine>
VPGS_D PairEval eval_staged(int q, float t1_0, float t2_0, float px, float py, const float4 &a, const float4 &b,
                            const float4 &f, float alpha_max) {
    if constexpr (kFine) {
        return eval_pair_fine(px, py, a.x, a.y, f.x, f.y, a.z, a.w, b.x, b.y, f.z, f.w, b.z, alpha_max);
    } else {
        PairEval e;
        e.t1 = fmaf((float)q, a.w, t1_0);
        e.t2 = fmaf((float)q, b.y, t2_0);
        e.G = ex2_approx(-fmaf(e.t1, e.t1, e.t2 * e.t2));
        e.alpha = fminf(alpha_max, b.z * e.G);
        return e;
    }
}

// whitened coordinates of the first of the thread's rows (plain form)
VPGS_D float2 first_row(float px, float py0, const float4 &a, const float4 &b) {
    const float dx = px - a.x, dy = py0 - a.y;
    return make_float2(fmaf(a.z, dx, a.w * dy), fmaf(b.x, dx, b.y * dy));
}

// register cap of the forward (0: only the 512-thread launch bound)
#ifndef VPGS_FWD_MAXREG
#define VPGS_FWD_MAXREG 0
#endif
#if VPGS_FWD_MAXREG > 0
#define VPGS_FWD_BOUNDS __maxnreg__(VPGS_FWD_MAXREG)
#else
#define VPGS_FWD_BOUNDS __launch_bounds__(kMaxThreads)
#endif

__global__ void VPGS_FWD_BOUNDS
composite_fwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, int n_tiles,
                     CamParams cam, OptParams o,
                     vpgs_images out, const uint32_t *status, uint32_t *work) {
    grid_dep_enter();
    extern __shared__ float4 smem[];
    const int NT = blockDim.x * kFwdBatch;  // records per batch
    float4 *s0 = smem, *s1 = smem + NT, *s2 = smem + 2 * NT, *s3 = smem + 3 * NT;
    uint16_t *s_wl = reinterpret_cast<uint16_t *>(smem + 4 * NT);  // [NW][NT] per-warp lists
    __shared__ int s_tile;
    if (*status != 0u) return;
    const int tid = threadIdx.x, lane = tid & 31;
    uint16_t *wl = s_wl + (size_t)(tid >> 5) * NT;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f;
    float pyl[kPix];
#pragma unroll
    for (int q = 0; q < kPix; ++q) pyl[q] = (float)(kPix * ly + q) + 0.5f;
    const float2 band = warp_rows(pyl);
    const float lg_amin = __log2f(o.alpha_min);
    int t = blockIdx.x;
    for (;;) {
        if (work) {
            if (tid == 0) s_tile = (int)atomicAdd(work, 1u);
            __syncthreads();
            t = s_tile;
            __syncthreads();
        }
        if (t >= n_tiles) return;
        const int tile = order ? (int)order[t] : t;  // launch order -> global tile id
        const TileCoord tc = tile_coord(tile, cam);
        const int px = tc.tx * cam.tile_w + lx;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const float xmax = fminf((float)cam.tile_w, (float)cam.W - ox) - 0.5f;  // last pixel centre column
        const uint2 rg = ranges[tile];
        const int start = (int)rg.x, end = (int)rg.y;
        float T[kPix], C0[kPix], C1[kPix], C2[kPix], D[kPix];
        int cnt[kPix], last[kPix];
        bool done[kPix];
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            T[q] = 1.f; C0[q] = C1[q] = C2[q] = D[q] = 0.f; cnt[q] = 0; last[q] = 0;
            const int py = tc.ty * cam.tile_h + kPix * ly + q;
            done[q] = !(px < cam.W && py < cam.H);
        }
        bool all_done = true;
#pragma unroll
        for (int q = 0; q < kPix; ++q) all_done = all_done && done[q];
        for (int b0 = start; b0 < end; b0 += NT) {
            if (__syncthreads_count(all_done) == (int)blockDim.x) break;
#pragma unroll 1
            for (int u = 0; u < kFwdBatch; ++u) {
                const int k = tid + u * (int)blockDim.x;
                const int j = b0 + k;
                if (j < end) {
                    const Rec r = rec[ival[j]];
                    stage(r, ox, oy, s0[k], s1[k], s2[k]);
                    if (r.r3.z < 0.f) s3[k] = fine_extra(r, ox, oy, s0[k].x, s0[k].y);
                }
            }
            __syncthreads();
            bool any_fine;
            const int nl = warp_list<false>(s0, s1, min(NT, end - b0), band, wl, lane, any_fine, xmax, lg_amin);
            // one blend step of this thread's pixels against list entry k
            auto blend = [&](int k, const float4 &a, const float4 &b, auto fine) -> bool {
                    constexpr bool kFine = decltype(fine)::value;
                    float4 f;
                    if constexpr (kFine) f = s3[k];
                    const float2 t0 = kFine ? make_float2(0.f, 0.f) : first_row(pxl, pyl[0], a, b);
                    bool fin = true;
#pragma unroll
                    for (int q = 0; q < kPix; ++q) {
                        if (!done[q]) {
                            const PairEval e = eval_staged<kFine>(q, t0.x, t0.y, pxl, pyl[q], a, b, f, o.alpha_max);
                            if (e.alpha >= o.alpha_min) {
                                const float nt = T[q] * (1.f - e.alpha);
                                if (nt < o.t_min) {
                                    done[q] = true;
                                } else {
                                    const float w = e.alpha * T[q];
                                    const float4 col = s2[k];
                                    C0[q] = fmaf(w, col.x, C0[q]);
                                    C1[q] = fmaf(w, col.y, C1[q]);
                                    C2[q] = fmaf(w, col.z, C2[q]);
                                    D[q] = fmaf(w, col.w, D[q]);
                                    T[q] = nt;
                                    ++cnt[q];
                                    last[q] = b0 + k - start + 1;
                                }
                            }
                        }
                        fin = fin && done[q];
                    }
                    return fin;
            };
            // the list walk; a batch with a near-degenerate record takes the walk that
            // chooses the precision form per entry (a warp-uniform branch), the others
            // the plain one, kWalk entries at a time: their alphas (which do not depend
            // on the transmittance) are evaluated before the blends, so the pixels'
            // blend chains overlap with independent work
            auto walk_plain = [&]() {
                for (int i = 0; i < nl; i += kWalk) {
                    float al[kWalk][kPix];
                    int kk[kWalk];
#pragma unroll
                    for (int u = 0; u < kWalk; ++u) kk[u] = wl[min(i + u, nl - 1)];
#pragma unroll
                    for (int u = 0; u < kWalk; ++u) {
                        const float4 a = s0[kk[u]], b = s1[kk[u]];
                        const float2 t0 = first_row(pxl, pyl[0], a, b);
#pragma unroll
                        for (int q = 0; q < kPix; ++q)
                            al[u][q] = eval_staged<false>(q, t0.x, t0.y, pxl, pyl[q], a, b, a, o.alpha_max).alpha;
                    }
                    bool fin = false;
#pragma unroll
                    for (int u = 0; u < kWalk; ++u) {
                        if (fin || i + u >= nl) break;
                        fin = true;
#pragma unroll
                        for (int q = 0; q < kPix; ++q) {
                            if (!done[q] && al[u][q] >= o.alpha_min) {
                                const float nt = T[q] * (1.f - al[u][q]);
                                if (nt < o.t_min) {
                                    done[q] = true;
                                } else {
                                    const float w = al[u][q] * T[q];
                                    const float4 col = s2[kk[u]];
                                    C0[q] = fmaf(w, col.x, C0[q]);
                                    C1[q] = fmaf(w, col.y, C1[q]);
                                    C2[q] = fmaf(w, col.z, C2[q]);
                                    D[q] = fmaf(w, col.w, D[q]);
                                    T[q] = nt;
                                    ++cnt[q];
                                    last[q] = b0 + kk[u] - start + 1;
                                }
                            }
                            fin = fin && done[q];
                        }
                    }
                    if (fin) {
                        all_done = true;
                        break;
                    }
                }
            };
            auto walk = [&](auto maybe_fine) {
                for (int i = 0; i < nl; ++i) {
                    const int k = wl[i];
                    const float4 a = s0[k], b = s1[k];
                    bool fin;
                    if constexpr (decltype(maybe_fine)::value)
                        fin = b.w < 0.f ? blend(k, a, b, std::true_type{}) : blend(k, a, b, std::false_type{});
                    else
                        fin = blend(k, a, b, std::false_type{});
                    if (fin) {
                        all_done = true;
                        break;
                    }
                }
            };
            if (!all_done) {
                if (any_fine) walk(std::true_type{});
                else walk_plain();
            }
        }
        const int64_t HW = (int64_t)cam.H * cam.W;
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            const int py = tc.ty * cam.tile_h + kPix * ly + q;
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

// Transpose reduction of R values over a warp (R = 10: all 2D gradient slots;
// R = 6: the geometric ones).  Each halving step keeps ceil(R/2) live values
// per lane: one half of the lanes keeps the low slots, its partners the high
// slots, and each adds what the partner sent (5+3+2+1 shuffles for R = 10,
// 3+2+1 for R = 6), then the lane groups that hold the same slot are summed.
// Afterwards lane l holds the warp total of slot red_slot<R>(l) in v[0] (or
// nothing, red_slot = -1).
template <int R, int O, int N>
VPGS_D void half_step(float (&v)[N], int lane) {
    constexpr int S = (R + 1) / 2;
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const float lo = v[i];
        const float hi = (i + S < R) ? v[i + S] : 0.f;
        v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, O);
    }
}

template <int R>
VPGS_D int red_slot(int lane) {
    int n = R, off = 0, r = R, bit = 16;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (r <= 1) break;
        const int S = (r + 1) / 2;
        if (lane & bit) {
            off += S;
            n = max(n - S, 0);
        } else {
            n = min(n, S);
        }
        r = S;
        bit >>= 1;
    }
    return (n >= 1 && (lane & (2 * bit - 1)) == 0) ? off : -1;
}

VPGS_D void warp_reduce(float (&a)[10], int lane) {
    half_step<10, 16>(a, lane);
    half_step<5, 8>(a, lane);
    half_step<3, 4>(a, lane);
    half_step<2, 2>(a, lane);
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
}

VPGS_D void warp_reduce(float (&a)[6], int lane) {
    half_step<6, 16>(a, lane);
    half_step<3, 8>(a, lane);
    half_step<2, 4>(a, lane);
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// 2D gradient slot [u, v, a, b, c, o, r, g, b, z] of accumulator q: the
// geometric form (NV = 6) keeps u, v, a, b, c and the depth z in q = 0..5
template <int NV>
VPGS_D int g2d_slot(int q) {
    return (NV == 6 && q == 5) ? 9 : q;
}

// per-pixel backward state
// beta = g . B: the upstream gradient (colour, depth) dotted with the colour /
// depth "behind" the current Gaussian, the only way B enters the gradient
struct PixState {
    float T, gAT, gC0, gC1, gC2, gD, beta;  // gAT = dL/dalpha_pixel * T_final
    int last;
};

// gradient of one pixel-Gaussian pair (Gaussian at list position jj), added to v;
// updates the pixel's transmittance and behind-colour; returns whether it blended.
// NV = 10: every 2D slot; NV = 6: only what the means, covariances and pose need
// (no opacity or colour sums), the form taken when no opacity or colour
// gradient is asked for
template <int NV>
VPGS_D bool pair_grad(PixState &p, int jj, const PairEval &e, const float4 &b, const float4 &c,
                      const OptParams &o, float (&v)[NV]) {
    if (jj >= p.last || e.alpha < o.alpha_min) return false;
    const float om = 1.f - e.alpha;
#if VPGS_BWD_RCP
    const float iom = __fdividef(1.f, om);  // om >= 1 - alpha_max > 0
    p.T *= iom;
    const float gat = p.gAT * iom;  // dA/dalpha_i = T_final / (1 - alpha_i)
#else
    p.T = p.T / om;
    const float gat = p.gAT / om;
#endif
    const float w = e.alpha * p.T;
    if constexpr (NV == 10) {
        v[6] = fmaf(w, p.gC0, v[6]);
        v[7] = fmaf(w, p.gC1, v[7]);
        v[8] = fmaf(w, p.gC2, v[8]);
        v[9] = fmaf(w, p.gD, v[9]);
    } else {
        v[5] = fmaf(w, p.gD, v[5]);
    }
    // dL/dalpha_i = T_i g . (c_i - B_i) + gat; behind this Gaussian
    // B <- B + alpha (c - B), so beta = g . B <- beta + alpha (g . c - beta)
    const float diff = fmaf(p.gC0, c.x, fmaf(p.gC1, c.y, fmaf(p.gC2, c.z, p.gD * c.w))) - p.beta;
    const float dA = fmaf(diff, p.T, gat);
    p.beta = fmaf(e.alpha, diff, p.beta);
    if (b.z * e.G <= o.alpha_max) {
        // slots 0-4 hold sums in the Gaussian's whitened frame t = W d, turned into
        // gradients once per Gaussian by the preprocess backward: sum dpow t1 and
        // sum dpow t2 for the mean (through the whitening rows and 2 ln 2), and
        // sum dpow t t^T (t1^2, t1 t2, t2^2) for the covariance (dL/dSigma' =
        // 2 ln^2 2 W^T S W).  t is O(1) where alpha matters, so these sums keep
        // their precision however elongated the Gaussian is.
        const float dpow = dA * e.alpha;
        if constexpr (NV == 10) v[5] = fmaf(dA, e.G, v[5]);
        const float pt1 = dpow * e.t1, pt2 = dpow * e.t2;
        v[0] += pt1;
        v[1] += pt2;
        v[2] = fmaf(pt1, e.t1, v[2]);
        v[3] = fmaf(pt1, e.t2, v[3]);
        v[4] = fmaf(pt2, e.t2, v[4]);
    }
    return true;
}

constexpr int kPartStride = 11;  // floats per (warp, Gaussian) partial, padded against bank conflicts

// register cap of the backward (0: only the 512-thread launch bound).  72
// registers keep 7 blocks of 4 warps (28 warps) resident per SM: registers are
// granted in units of 8 per thread, so 73-80 would leave room for 6 blocks.
// The backward needs no spill under this cap.
#ifndef VPGS_BWD_MAXREG
#define VPGS_BWD_MAXREG 72
#endif
#if VPGS_BWD_MAXREG > 0
#define VPGS_BWD_BOUNDS __maxnreg__(VPGS_BWD_MAXREG)
#else
#define VPGS_BWD_BOUNDS __launch_bounds__(kMaxThreads)
#endif

// ACC: how the warps' sums of a Gaussian are combined (VPGS_BWD_ACC): 0 = one
// global atomic per (warp, Gaussian, slot); 1 = each warp stores its sums in its
// own shared slots and one thread per Gaussian adds the warps' slots into one
// global atomic per batch; 2 = shared-memory atomics per batch
template <int NV, int ACC>
__global__ void VPGS_BWD_BOUNDS
composite_bwd_kernel(const Rec *__restrict__ rec, const uint32_t *__restrict__ ival,
                     const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, int n_tiles,
                     CamParams cam, OptParams o,
                     const float *__restrict__ t_final, const int32_t *__restrict__ n_iter,
                     const float *__restrict__ dL_drgb, const float *__restrict__ dL_ddepth,
                     const float *__restrict__ dL_dalpha, float *__restrict__ g2d,
                     const uint32_t *status, uint32_t *work) {
    grid_dep_enter();
    extern __shared__ float4 smem[];
    const int NT = blockDim.x * kBwdBatch;  // records per batch
    const int NW = blockDim.x >> 5;
    float4 *s0 = smem, *s1 = smem + NT, *s2 = smem + 2 * NT;
    uint32_t *s_id = reinterpret_cast<uint32_t *>(smem + 3 * NT);
    uint16_t *s_wl = reinterpret_cast<uint16_t *>(s_id + NT);             // [NW][NT] per-warp lists
    float *s_part = reinterpret_cast<float *>(s_wl + (size_t)NW * NT);  // [NW][NT][kPartStride]
    __shared__ int s_tile;
    __shared__ int s_max;
    if (*status != 0u) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = tid % cam.tile_w, ly = tid / cam.tile_w;
    const float pxl = (float)lx + 0.5f;
    float pyl[kPix];
#pragma unroll
    for (int q = 0; q < kPix; ++q) pyl[q] = (float)(kPix * ly + q) + 0.5f;
    const float2 band = warp_rows(pyl);
    const float lg_amin = __log2f(o.alpha_min);
    uint16_t *wl = s_wl + (size_t)warp * NT;
    float *my_part = s_part + (size_t)warp * NT * kPartStride;
    const int rs = red_slot<NV>(lane);
    const int slot = rs >= 0 ? g2d_slot<NV>(rs) : -1;
    // hands one warp total (this lane's slot) of Gaussian k to the combination scheme
    auto put = [&](int k, float val) {
        if (ACC == 0) {
            if (val != 0.f) atomicAdd(g2d + 10 * (int64_t)s_id[k] + slot, val);
        } else if (ACC == 1) {
            my_part[k * kPartStride + slot] = val;
        } else {
            if (val != 0.f) atomicAdd(s_part + k * kPartStride + slot, val);
        }
    };
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
        const int tile = order ? (int)order[t] : t;  // launch order -> global tile id
        const TileCoord tc = tile_coord(tile, cam);
        const int px = tc.tx * cam.tile_w + lx;
        const float ox = (float)(tc.tx * cam.tile_w), oy = (float)(tc.ty * cam.tile_h);
        const float xmax = fminf((float)cam.tile_w, (float)cam.W - ox) - 0.5f;  // last pixel centre column
        const uint2 rg = ranges[tile];
        const int start = (int)rg.x;
        const int64_t HW = (int64_t)cam.H * cam.W;
        PixState ps[kPix];
        int my_max = 0;
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
            PixState &p = ps[q];
            p.T = 1.f; p.gC0 = p.gC1 = p.gC2 = p.gD = 0.f; p.last = 0;
            float gA = 0.f;
            const int py = tc.ty * cam.tile_h + kPix * ly + q;
            if (px < cam.W && py < cam.H) {
                const int64_t pix = (int64_t)tc.v * HW + (int64_t)py * cam.W + px;
                p.T = t_final[pix];
                p.last = n_iter[pix];
                if (dL_drgb) {
                    const float *gp = dL_drgb + (int64_t)tc.v * 3 * HW + (int64_t)py * cam.W + px;
                    p.gC0 = gp[0]; p.gC1 = gp[HW]; p.gC2 = gp[2 * HW];
                }
                if (dL_ddepth) p.gD = dL_ddepth[pix];
                if (dL_dalpha) gA = dL_dalpha[pix];
            }
            p.gAT = gA * p.T;  // p.T holds T_final here
            p.beta = fmaf(p.gC0, o.bg0, fmaf(p.gC1, o.bg1, p.gC2 * o.bg2));  // B starts at the background
            my_max = max(my_max, p.last);
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
#pragma unroll 1
            for (int u = 0; u < kBwdBatch; ++u) {
                const int k = tid + u * (int)blockDim.x;
                if (b0 + k < b1) {
                    const uint32_t id = ival[b0 + k];
                    stage(rec[id], ox, oy, s0[k], s1[k], s2[k]);
                    s_id[k] = id;
                }
            }
            if (ACC == 1)
                for (int e = lane; e < nb * kPartStride; e += 32) my_part[e] = 0.f;
            if (ACC == 2)
                for (int e = tid; e < nb * kPartStride; e += (int)blockDim.x) s_part[e] = 0.f;
            __syncthreads();
            const int k_end = min(nb, warp_max - (b0 - start));  // warp-uniform
            bool any_fine;
            const int nl = warp_list<true>(s0, s1, k_end, band, wl, lane, any_fine, xmax, lg_amin);
            // back to front; a batch with a near-degenerate record takes the walk that
            // chooses the precision form per entry (a warp-uniform branch), the others
            // the plain one
            auto walk = [&](auto maybe_fine) {
            for (int i = nl - 1; i >= 0; --i) {
                const int kk = wl[i];
                const float4 a = s0[kk], b = s1[kk], c = s2[kk];
                float v[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) v[q] = 0.f;
                const int jj = b0 + kk - start;
                // this thread's pixels against the Gaussian
                auto grads = [&](auto fine) -> bool {
                    constexpr bool kFine = decltype(fine)::value;
                    float4 f;
                    if constexpr (kFine) f = fine_extra(rec[s_id[kk]], ox, oy, a.x, a.y);
                    const float2 t0 = kFine ? make_float2(0.f, 0.f) : first_row(pxl, pyl[0], a, b);
                    bool any = false;
#pragma unroll
                    for (int q = 0; q < kPix; ++q) {
                        const PairEval e = eval_staged<kFine>(q, t0.x, t0.y, pxl, pyl[q], a, b, f, o.alpha_max);
                        any |= pair_grad(ps[q], jj, e, b, c, o, v);
                    }
                    return any;
                };
                bool act;
                if constexpr (decltype(maybe_fine)::value)
                    act = b.w < 0.f ? grads(std::true_type{}) : grads(std::false_type{});
                else
                    act = grads(std::false_type{});
                const uint32_t am = __ballot_sync(0xffffffffu, act);
                if (ACC == 0 && am != 0u && __popc(am) <= kDirect) {
                    // few active lanes: their own atomics beat a reduction
                    if (act) {
                        float *dst = g2d + 10 * (int64_t)s_id[kk];
#pragma unroll
                        for (int q = 0; q < NV; ++q)
                            if (v[q] != 0.f) atomicAdd(dst + g2d_slot<NV>(q), v[q]);
                    }
                } else if (am != 0u) {
                    warp_reduce(v, lane);
                    if (slot >= 0) put(kk, v[0]);
                }
            }
            };
            if (any_fine) walk(std::true_type{});
            else walk(std::false_type{});
            if (ACC != 0) {
                __syncthreads();
                // one thread per Gaussian of the batch: one global atomic per value
                for (int k = tid; k < nb; k += (int)blockDim.x) {
                    float *dst = g2d + 10 * (int64_t)s_id[k];
#pragma unroll
                    for (int sl = 0; sl < 10; ++sl) {
                        float acc = 0.f;
                        if (ACC == 1) {
                            for (int w = 0; w < NW; ++w) acc += s_part[((size_t)w * NT + k) * kPartStride + sl];
                        } else {
                            acc = s_part[k * kPartStride + sl];
                        }
                        if (acc != 0.f) atomicAdd(dst + sl, acc);
                    }
                }
            }
        }
        if (!work) return;
        __syncthreads();
    }
}

// dynamic shared memory of a compositing block of `threads` threads staging
// `records` per batch: forward s0-s3 and the warps' lists; backward s0-s2, the
// ids, the lists and the per-Gaussian partial sums of the combination scheme
static size_t comp_smem(int threads, int records, bool bwd, int acc = 0) {
    const size_t warps = (size_t)threads / 32;
    const size_t parts = acc == 1 ? warps * records * kPartStride : (acc == 2 ? (size_t)records * kPartStride : 0);
    const size_t lists = sizeof(uint16_t) * warps * records;
    return sizeof(float4) * (bwd ? 3 : 4) * records + lists +
           (bwd ? sizeof(uint32_t) * records + sizeof(float) * parts : 0);
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
    const size_t sm = comp_smem(B, B * kFwdBatch, false);
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
                launch_k(composite_fwd_kernel, grid, B, sm, s, ws.rec, ival, ws.ranges,
                         VPGS_TILE_ORDER ? (const uint32_t *)ws.tile_order : nullptr, n_tiles, cam, o, out,
                         ws.status, work));
    return cudaGetLastError();
}

template <int NV, int ACC>
static cudaError_t composite_bwd_as(const RenderWs &ws, const uint32_t *ival, int V, const CamParams &cam,
                                    const OptParams &o, const vpgs_images &fwd, const float *dL_drgb,
                                    const float *dL_ddepth, const float *dL_dalpha, int persistent_ctas,
                                    cudaStream_t s) {
    const int B = cam.tile_w * cam.tile_h / kPix;
    const int n_tiles = V * cam.T;
    const size_t sm = comp_smem(B, B * kBwdBatch, true, ACC);
    const void *kern = (const void *)composite_bwd_kernel<NV, ACC>;
    uint32_t *work = nullptr;
    int grid = n_tiles;
    if (persistent_ctas > 0) {
        work = ws.counters + CNT_WORK;
        cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        grid = persistent_grid(kern, B, sm, persistent_ctas, n_tiles);
    }
    if (grid == 0) return cudaSuccess;
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    VPGS_LAUNCH("composite_bwd", s,
                launch_k(composite_bwd_kernel<NV, ACC>, grid, B, sm, s, ws.rec, ival, ws.ranges,
                         VPGS_TILE_ORDER ? (const uint32_t *)ws.tile_order : nullptr, n_tiles, cam, o,
                         fwd.t_final, fwd.n_iter, dL_drgb, dL_ddepth, dL_dalpha, ws.g2d, ws.status, work));
    return cudaGetLastError();
}

template <int NV>
static cudaError_t composite_bwd_nv(int acc, const RenderWs &ws, const uint32_t *ival, int V,
                                    const CamParams &cam, const OptParams &o, const vpgs_images &fwd,
                                    const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                                    int persistent_ctas, cudaStream_t s) {
    switch (acc) {
    case 1: return composite_bwd_as<NV, 1>(ws, ival, V, cam, o, fwd, dL_drgb, dL_ddepth, dL_dalpha, persistent_ctas, s);
    case 2: return composite_bwd_as<NV, 2>(ws, ival, V, cam, o, fwd, dL_drgb, dL_ddepth, dL_dalpha, persistent_ctas, s);
    default: return composite_bwd_as<NV, 0>(ws, ival, V, cam, o, fwd, dL_drgb, dL_ddepth, dL_dalpha, persistent_ctas, s);
    }
}

cudaError_t launch_composite_bwd(const RenderWs &ws, const uint32_t *ival, int V,
                                 const CamParams &cam, const OptParams &o, const vpgs_images &fwd,
                                 const float *dL_drgb, const float *dL_ddepth,
                                 const float *dL_dalpha, bool geometric_only, int persistent_ctas,
                                 cudaStream_t s) {
    // per-warp shared slots pay off as soon as a tile has warps' sums to combine
    const int warps = cam.tile_w * cam.tile_h / kPix / 32;
    const int acc = VPGS_BWD_ACC >= 0 ? VPGS_BWD_ACC : (warps >= 2 ? 1 : 0);
    return geometric_only
               ? composite_bwd_nv<6>(acc, ws, ival, V, cam, o, fwd, dL_drgb, dL_ddepth, dL_dalpha, persistent_ctas, s)
               : composite_bwd_nv<10>(acc, ws, ival, V, cam, o, fwd, dL_drgb, dL_ddepth, dL_dalpha, persistent_ctas, s);
}

}  // namespace vpgs
