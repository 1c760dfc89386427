// C ABI entry points of the rasterizer: argument checks, workspace layout and
// the launch sequence.  Decoder entry points live in decode.cu.
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.h"
#include "prims.cuh"

using namespace vpgs;

namespace {

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

inline int bits_for(int64_t max_value) {
    int b = 0;
    while (b < 63 && (int64_t(1) << b) <= max_value) ++b;
    return b < 1 ? 1 : b;
}

bool valid_opts(const vpgs_render_opts *o) {
    if (!o) return false;
    // a warp covers whole rows of a tile: tile_w divides 32
    if (o->tile_w != 4 && o->tile_w != 8 && o->tile_w != 16 && o->tile_w != 32) return false;
    if (o->tile_h < 2 || o->tile_h > 64) return false;
    // at most 512 pixels per tile; VPGS_PIX adjacent rows per compositing thread, whole warps
    const int B = o->tile_w * o->tile_h;
    if (o->tile_h % 2 != 0 || B % 64 != 0 || B > 512 || o->tile_h % VPGS_PIX != 0) return false;
    if (!(o->alpha_min > 0.f && o->alpha_min < 1.f)) return false;
    if (!(o->alpha_max > o->alpha_min && o->alpha_max < 1.f)) return false;
    if (!(o->t_min > 0.f && o->t_min < 1.f)) return false;
    if (!(o->dilation >= 0.f) || !(o->near_z >= 0.f)) return false;
    if (o->persistent_ctas < 0 || o->persistent_ctas > 32) return false;
    if ((o->flags & ~VPGS_RENDER_REUSE_BINNING) != 0) return false;
    if (o->spin_limit < 0) return false;
    return true;
}

bool make_layout(int64_t N, int V, const vpgs_camera *cam, const vpgs_render_opts *o, int64_t M_cap,
                 RenderLayout &L) {
    if (N < 0 || V <= 0 || V > 4096 || !cam || !valid_opts(o) || M_cap < 0) return false;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 || cam->height > 65535) return false;
    memset(&L, 0, sizeof(L));
    L.N = N;
    L.V = V;
    L.tiles_x = (cam->width + o->tile_w - 1) / o->tile_w;
    L.tiles_y = (cam->height + o->tile_h - 1) / o->tile_h;
    L.T = L.tiles_x * L.tiles_y;
    L.VN = (int64_t)V * N;
    if (L.VN >= (int64_t(1) << 31)) return false;
    if ((int64_t)V * L.T >= (int64_t(1) << 31)) return false;
    if (M_cap >= (int64_t(1) << 30)) return false;
    L.M_cap = M_cap < 1 ? 1 : M_cap;
    L.tile_bits = bits_for((int64_t)V * L.T - 1);
    SortPass ps[kMaxSortPasses];
    const int np_tile = plan_passes(0, L.tile_bits, ps);
    const int64_t VN1 = L.VN < 1 ? 1 : L.VN;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = align_up(off + bytes);
        return o2;
    };
    L.off_status = take(4);
    L.off_counters = take(4 * CNT_N);
    L.off_rec = take(sizeof(Rec) * VN1);
    L.off_tcount = take(4 * VN1);
    L.off_dkey0 = take(4 * VN1);
    L.off_dval0 = take(4 * VN1);
    L.off_dkey1 = take(4 * VN1);
    L.off_dval1 = take(4 * VN1);
    L.off_ikey0 = take(4 * L.M_cap);
    L.off_ival0 = take(4 * L.M_cap);
    L.off_ikey1 = take(4 * L.M_cap);
    L.off_ival1 = take(4 * L.M_cap);
    L.off_ranges = take(sizeof(uint2) * (size_t)V * L.T);
    L.off_sort_hist = take(2 * 4 * kRadix * 4);
    const int64_t look_a = 4 * sort_blocks(VN1, kDepthSortItems);
    const int64_t look_b = (int64_t)std::max(np_tile, 1) * sort_blocks(L.M_cap, kTileSortItems);
    L.sort_blocks_max = look_a > look_b ? look_a : look_b;
    L.off_sort_look = take(4 * kRadix * (size_t)look_a);
    L.off_sort_look_t = take(4 * kRadix * (size_t)look_b);
    // scans: visibility and offsets over V*N items
    L.scan_blocks_max = scan_blocks(VN1);
    L.off_scan_look = take(2 * 8 * (size_t)L.scan_blocks_max);
    L.off_g2d = take(4 * 10 * (size_t)VN1);
    L.off_posedf = take(4 * 24 * (size_t)V);
    L.off_bin = take(sizeof(BinRec) * (size_t)VN1);
    L.off_vis_idx = take(4 * (size_t)VN1);
    L.off_tile_order = take(4 * (size_t)V * L.T);
    L.off_tile_work = take(4 * (size_t)V * L.T);
    L.total = off;
    return true;
}

RenderWs carve(void *base, const RenderLayout &L) {
    char *b = static_cast<char *>(base);
    RenderWs w;
    w.status = reinterpret_cast<uint32_t *>(b + L.off_status);
    w.counters = reinterpret_cast<uint32_t *>(b + L.off_counters);
    w.rec = reinterpret_cast<Rec *>(b + L.off_rec);
    w.tcount = reinterpret_cast<uint32_t *>(b + L.off_tcount);
    w.dkey[0] = reinterpret_cast<uint32_t *>(b + L.off_dkey0);
    w.dval[0] = reinterpret_cast<uint32_t *>(b + L.off_dval0);
    w.dkey[1] = reinterpret_cast<uint32_t *>(b + L.off_dkey1);
    w.dval[1] = reinterpret_cast<uint32_t *>(b + L.off_dval1);
    w.ikey[0] = reinterpret_cast<uint32_t *>(b + L.off_ikey0);
    w.ival[0] = reinterpret_cast<uint32_t *>(b + L.off_ival0);
    w.ikey[1] = reinterpret_cast<uint32_t *>(b + L.off_ikey1);
    w.ival[1] = reinterpret_cast<uint32_t *>(b + L.off_ival1);
    w.ranges = reinterpret_cast<uint2 *>(b + L.off_ranges);
    w.sort_hist[0] = reinterpret_cast<uint32_t *>(b + L.off_sort_hist);
    w.sort_hist[1] = w.sort_hist[0] + 4 * kRadix;
    w.sort_look[0] = reinterpret_cast<uint32_t *>(b + L.off_sort_look);
    w.sort_look[1] = reinterpret_cast<uint32_t *>(b + L.off_sort_look_t);
    w.scan_look[0] = reinterpret_cast<unsigned long long *>(b + L.off_scan_look);
    w.scan_look[1] = w.scan_look[0] + L.scan_blocks_max;
    w.g2d = reinterpret_cast<float *>(b + L.off_g2d);
    w.posedf = reinterpret_cast<float *>(b + L.off_posedf);
    w.bin = reinterpret_cast<BinRec *>(b + L.off_bin);
    w.vis_idx = reinterpret_cast<uint32_t *>(b + L.off_vis_idx);
    w.tile_order = reinterpret_cast<uint32_t *>(b + L.off_tile_order);
    w.tile_work = reinterpret_cast<uint32_t *>(b + L.off_tile_work);
    return w;
}

// Largest instance capacity whose layout fits in ws_bytes (-1 if none).
int64_t capacity_for(size_t ws_bytes, int64_t N, int V, const vpgs_camera *cam,
                     const vpgs_render_opts *o) {
    RenderLayout L;
    if (!make_layout(N, V, cam, o, 1, L) || L.total > ws_bytes) return -1;
    int64_t lo = 1, hi = (int64_t(1) << 30) - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (make_layout(N, V, cam, o, mid, L) && L.total <= ws_bytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool valid_gaussians(const vpgs_gaussians *g) {
    if (!g || g->n < 0) return false;
    if (g->n == 0) return true;
    if (!g->means || !g->scales || !g->quats || !g->opacities || !g->colors) return false;
    return aligned16(g->quats);
}

struct Setup {
    RenderLayout L;
    RenderWs ws;
    CamParams cam;
    OptParams o;
    GaussIn g;
};

vpgs_status setup(void *ws, size_t ws_bytes, const vpgs_gaussians *g, const vpgs_camera *cam,
                  const double *T_cw, int32_t V, const vpgs_render_opts *opts, Setup &S) {
    if (!ws || !valid_gaussians(g) || !cam || !T_cw || V <= 0 || !valid_opts(opts))
        return VPGS_ERR_INVALID_ARG;
    if (!aligned16(ws)) return VPGS_ERR_INVALID_ARG;
    const int64_t cap = capacity_for(ws_bytes, g->n, V, cam, opts);
    if (cap < 1 || !make_layout(g->n, V, cam, opts, cap, S.L)) return VPGS_ERR_INVALID_ARG;
    S.ws = carve(ws, S.L);
    S.cam = CamParams{cam->width, cam->height, cam->fx, cam->fy, cam->cx, cam->cy,
                      opts->tile_w, opts->tile_h, S.L.tiles_x, S.L.tiles_y, S.L.T,
                      __builtin_ctz((unsigned)opts->tile_w)};
    S.o = OptParams{opts->alpha_min, opts->alpha_max, opts->t_min, opts->dilation, opts->near_z,
                    opts->bg[0], opts->bg[1], opts->bg[2], opts->spin_limit > 0 ? opts->spin_limit : kSpinLimit};
    S.g = GaussIn{g->means, g->scales, g->quats, g->opacities, g->colors, g->n, g->n_dev};
    return VPGS_OK;
}

vpgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA; }

// Arguments of the last call that left a complete projection + tile lists in a
// workspace.  A backward with VPGS_RENDER_REUSE_BINNING reuses them only when
// its own arguments match.
struct BinTag {
    const void *ws;
    size_t ws_bytes;
    vpgs_gaussians g;
    vpgs_camera cam;
    const double *T_cw;
    int32_t V;
    vpgs_render_opts o;  // flags and persistent_ctas cleared
};

std::mutex g_tag_mu;
std::vector<BinTag> g_tags;
constexpr size_t kMaxTags = 256;

BinTag make_tag(const void *ws, size_t ws_bytes, const vpgs_gaussians *g, const vpgs_camera *cam,
                const double *T_cw, int32_t V, const vpgs_render_opts *o) {
    BinTag t;
    memset(&t, 0, sizeof(t));
    t.ws = ws;
    t.ws_bytes = ws_bytes;
    t.g = *g;
    t.cam = *cam;
    t.T_cw = T_cw;
    t.V = V;
    t.o = *o;
    t.o.flags = 0;
    t.o.persistent_ctas = 0;
    return t;
}

bool same_tag(const BinTag &a, const BinTag &b) {
    const bool g = a.g.means == b.g.means && a.g.scales == b.g.scales && a.g.quats == b.g.quats &&
                   a.g.opacities == b.g.opacities && a.g.colors == b.g.colors && a.g.n == b.g.n &&
                   a.g.n_dev == b.g.n_dev;
    const bool c = a.cam.width == b.cam.width && a.cam.height == b.cam.height && a.cam.fx == b.cam.fx &&
                   a.cam.fy == b.cam.fy && a.cam.cx == b.cam.cx && a.cam.cy == b.cam.cy;
    const bool o = a.o.tile_w == b.o.tile_w && a.o.tile_h == b.o.tile_h && a.o.alpha_min == b.o.alpha_min &&
                   a.o.alpha_max == b.o.alpha_max && a.o.t_min == b.o.t_min &&
                   a.o.dilation == b.o.dilation && a.o.near_z == b.o.near_z && a.o.bg[0] == b.o.bg[0] &&
                   a.o.bg[1] == b.o.bg[1] && a.o.bg[2] == b.o.bg[2];
    return a.ws == b.ws && a.ws_bytes == b.ws_bytes && g && c && o && a.T_cw == b.T_cw && a.V == b.V;
}

void tag_set(const BinTag &t) {
    std::lock_guard<std::mutex> lk(g_tag_mu);
    for (auto &x : g_tags)
        if (x.ws == t.ws) {
            x = t;
            return;
        }
    if (g_tags.size() >= kMaxTags) g_tags.erase(g_tags.begin());
    g_tags.push_back(t);
}

void tag_clear(const void *ws) {
    std::lock_guard<std::mutex> lk(g_tag_mu);
    for (size_t i = 0; i < g_tags.size(); ++i)
        if (g_tags[i].ws == ws) {
            g_tags.erase(g_tags.begin() + (long)i);
            return;
        }
}

bool tag_matches(const BinTag &t) {
    std::lock_guard<std::mutex> lk(g_tag_mu);
    for (const auto &x : g_tags)
        if (x.ws == t.ws) return same_tag(x, t);
    return false;
}

}  // namespace

extern "C" {

void vpgs_render_opts_default(vpgs_render_opts *o) {
    if (!o) return;
    o->tile_w = 16;  // 16x16 tiles: measured fastest fwd+bwd on GB300 with the tiles
    o->tile_h = 16;  // launched heaviest first (the image does not depend on the tile shape)
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_min = 1e-4f;
    o->dilation = 0.3f;
    o->near_z = 0.2f;
    o->bg[0] = o->bg[1] = o->bg[2] = 0.f;
    o->persistent_ctas = 0;
    o->flags = 0;
    o->spin_limit = 0;
}

size_t vpgs_render_workspace_bytes(int64_t max_gaussians, int32_t n_views, const vpgs_camera *cam,
                                   const vpgs_render_opts *opts, int64_t max_instances) {
    RenderLayout L;
    if (!make_layout(max_gaussians, n_views, cam, opts, max_instances, L)) return 0;
    return L.total;
}

vpgs_status vpgs_render_fwd(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                            const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                            const vpgs_render_opts *opts, const vpgs_images *out, vpgs_stream stream) {
    if (!out || !out->t_final || !out->n_iter) return VPGS_ERR_INVALID_ARG;
    Setup S;
    vpgs_status st = setup(ws, ws_bytes, g, cam, T_cw, n_views, opts, S);
    if (st != VPGS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    tag_clear(ws);
    // the 2D gradient slots of visible Gaussians start at zero for a backward that reuses this call
    cudaError_t e = launch_preprocess_fwd(S.g, T_cw, n_views, S.cam, S.o, S.ws, S.L, true, s);
    int buf = 0;
    if (e == cudaSuccess) e = build_tile_lists(S.g, n_views, S.cam, S.o, S.ws, S.L, &buf, s);
    if (e == cudaSuccess)
        e = launch_composite_fwd(S.ws, S.ws.ival[buf], n_views, S.cam, S.o, *out, opts->persistent_ctas, s);
    if (e == cudaSuccess) tag_set(make_tag(ws, ws_bytes, g, cam, T_cw, n_views, opts));
    return cuda_status(e);
}

vpgs_status vpgs_render_bwd(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                            const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                            const vpgs_render_opts *opts, const vpgs_images *fwd,
                            const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                            const vpgs_gaussian_buffers *grads, double *dL_dpose,
                            vpgs_stream stream) {
    if (!fwd || !fwd->t_final || !fwd->n_iter) return VPGS_ERR_INVALID_ARG;
    if (grads && grads->quats && !aligned16(grads->quats)) return VPGS_ERR_INVALID_ARG;
    Setup S;
    vpgs_status st = setup(ws, ws_bytes, g, cam, T_cw, n_views, opts, S);
    if (st != VPGS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    GaussGrad gg{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (grads) gg = GaussGrad{grads->means, grads->scales, grads->quats, grads->opacities, grads->colors};
    if (!grads && !dL_dpose) return VPGS_OK;  // nothing to compute
    const BinTag tag = make_tag(ws, ws_bytes, g, cam, T_cw, n_views, opts);
    int buf = 0;
    cudaError_t e;
    if ((opts->flags & VPGS_RENDER_REUSE_BINNING) && tag_matches(tag)) {
        // the forward's projection and lists stand; its status word is kept, so an
        // error it recorded stops this pass too
        e = cudaSuccess;
        buf = tile_list_buffer(S.L);
    } else {
        // recompute projection, binning and per-tile sort
        e = launch_preprocess_fwd(S.g, T_cw, n_views, S.cam, S.o, S.ws, S.L, true, s);
        if (e == cudaSuccess)
            e = build_tile_lists(S.g, n_views, S.cam, S.o, S.ws, S.L, &buf, s,
                                 !(VPGS_TILE_ORDER && VPGS_BWD_ORDER_NITER));
        if (e == cudaSuccess) tag_set(tag);
        else tag_clear(ws);
    }
    // the backward walks each tile's list only as far as its pixels' n_iter: launch
    // the tiles with the most steps first
    if (e == cudaSuccess && VPGS_TILE_ORDER && VPGS_BWD_ORDER_NITER)
        e = order_tiles_by_steps(S.ws, fwd->n_iter, n_views, S.cam, s);
    // no opacity or colour gradient asked for (pose tracking): the compositing
    // backward sums only the slots the means, covariances, depths and pose need
    const bool geometric_only = !gg.opac && !gg.colors;
    if (e == cudaSuccess)
        e = launch_composite_bwd(S.ws, S.ws.ival[buf], n_views, S.cam, S.o, *fwd, dL_drgb, dL_ddepth,
                                 dL_dalpha, geometric_only, opts->persistent_ctas, s);
    if (e == cudaSuccess && (grads || dL_dpose))
        e = launch_preprocess_bwd(S.g, T_cw, n_views, S.cam, S.o, S.ws, gg, dL_dpose, s);
    return cuda_status(e);
}

vpgs_status vpgs_render_project(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                                const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                                const vpgs_render_opts *opts, int32_t *tile_count,
                                int32_t *tile_rect, float *mean2d, float *depth, float *conic,
                                vpgs_stream stream) {
    Setup S;
    vpgs_status st = setup(ws, ws_bytes, g, cam, T_cw, n_views, opts, S);
    if (st != VPGS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    tag_clear(ws);
    cudaError_t e = launch_preprocess_fwd(S.g, T_cw, n_views, S.cam, S.o, S.ws, S.L, false, s);
    if (e == cudaSuccess)
        e = launch_export_projection(S.ws, S.L.VN, tile_count, tile_rect, mean2d, depth, conic, s);
    return cuda_status(e);
}

vpgs_status vpgs_workspace_status(const void *ws, vpgs_render_stats *stats, vpgs_stream stream) {
    if (!ws || !stats) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t host[64 / 4 + CNT_N];
    RenderLayout L;
    // status and counters sit at fixed offsets (0 and 256) in every layout
    (void)L;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VPGS_ERR_CUDA;
    if (cudaMemcpy(host, ws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return VPGS_ERR_CUDA;
    if (cudaMemcpy(host + 1, static_cast<const char *>(ws) + 256, 4 * CNT_N, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return VPGS_ERR_CUDA;
    stats->status = (int32_t)host[0];
    stats->n_visible = host[1 + CNT_VISIBLE];
    stats->n_instances = host[1 + CNT_INSTANCES];
    return VPGS_OK;
}

vpgs_status vpgs_workspace_status_copy(const void *ws, int32_t *dst, vpgs_stream stream) {
    if (!ws || !dst) return VPGS_ERR_INVALID_ARG;
    // the status word sits at offset 0 of every render layout
    return cudaMemcpyAsync(dst, ws, sizeof(int32_t), cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? VPGS_OK
               : VPGS_ERR_CUDA;
}

vpgs_status vpgs_pose_step(double *T_cw, double *dL_dpose, double *adam_state, int32_t n_views,
                           const double lr[2], vpgs_stream stream) {
    if (!T_cw || !dL_dpose || n_views <= 0 || !lr) return VPGS_ERR_INVALID_ARG;
    return cuda_status(launch_pose_step(T_cw, dL_dpose, adam_state, n_views, lr[0], lr[1],
                                        reinterpret_cast<cudaStream_t>(stream)));
}

const char *vpgs_status_string(vpgs_status s) {
    switch (s) {
        case VPGS_OK: return "ok";
        case VPGS_ERR_INVALID_ARG: return "invalid argument";
        case VPGS_ERR_CAPACITY: return "tile-instance capacity exceeded";
        case VPGS_ERR_NONFINITE: return "non-finite input";
        case VPGS_ERR_TIMEOUT: return "bounded device wait ran out";
        case VPGS_ERR_CUDA: return "CUDA error";
        case VPGS_ERR_UNSUPPORTED: return "unsupported";
        case VPGS_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

const char *vpgs_version(void) { return "0.1.0"; }

}  // extern "C"
