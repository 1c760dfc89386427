// Submap expansion and anchor maintenance (Sec. III-A, "Voxel-Based Submap
// Expansion and Activation").
//
// Statistics.  Per training step, every decoded neural Gaussian i of anchor
// a = src_index[i] / k adds |dL/dmu_i| and 1 to the anchor's gradient sum and
// count when it was rendered (visible), and its opacity to the anchor's
// opacity sum; the first Gaussian of each anchor's run adds one visit.  FP32
// atomics (the sums' order is not fixed).
//
// Update.  Pruning keeps an anchor unless it was visited and its opacity per
// visit is below tau_o (an order-keeping compaction by scan).  Growth takes
// the decoded Gaussians of anchors whose average gradient exceeds tau_g,
// looks their voxels (edge v_g) up in a voxel hash of the existing anchors,
// keeps the free ones once each (first decoded Gaussian wins: hash insert +
// atomicMin, then a compaction by scan) and writes the voxel centres.
//
// Spawning.  One scan compacts the pixels whose alpha is below tau_alpha or
// whose rendered depth departs from the input depth (input depth > 0); M of
// them, evenly spaced in raster order, are back-projected in FP64 through the
// pixel centre and rounded to float32; their voxels are kept once each (first
// sample wins) and only when no Gaussian mean of the map lies within rho of
// the voxel centre (one warp per voxel over the 27 voxels around it); a last
// scan writes the centres in sample order.
//
// All decisions are taken in float32 with correctly rounded operations (the
// back-projection in FP64 with a fixed order), so they are reproducible off
// the GPU.
#include <cmath>
#include <cstddef>

#include "internal.h"
#include "prims.cuh"
#include "profiler.h"
#include "voxhash.cuh"

namespace vpgs {
namespace {

constexpr int kAThreads = 256;

int agrid(int64_t n) {
    const int64_t g = std::min<int64_t>((n + kAThreads - 1) / kAThreads, (int64_t)device_sm_count() * 8);
    return (int)std::max<int64_t>(g, 1);
}

// ---------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------
struct StatsLayout {
    size_t off_g, off_o, off_cnt, off_vis, off_status, total;
};

inline StatsLayout stats_layout(int64_t A) {
    const size_t a4 = align_up(4 * (size_t)A, 16);
    StatsLayout L;
    L.off_g = 0;
    L.off_o = a4;
    L.off_cnt = 2 * a4;
    L.off_vis = 3 * a4;
    L.off_status = 4 * a4;
    L.total = 4 * a4 + 16;
    return L;
}

struct StatsView {
    float *g_sum, *o_sum;
    uint32_t *g_cnt, *visits, *status;
};

StatsView stats_view(void *stats, int64_t A) {
    const StatsLayout L = stats_layout(A);
    char *b = static_cast<char *>(stats);
    return StatsView{reinterpret_cast<float *>(b + L.off_g), reinterpret_cast<float *>(b + L.off_o),
                     reinterpret_cast<uint32_t *>(b + L.off_cnt), reinterpret_cast<uint32_t *>(b + L.off_vis),
                     reinterpret_cast<uint32_t *>(b + L.off_status)};
}

VPGS_D int64_t clamp_count(int64_t n_cap, const int32_t *n_dev) {
    return n_dev ? max((int64_t)0, min(n_cap, (int64_t)*n_dev)) : n_cap;
}

__global__ void __launch_bounds__(kAThreads)
stats_accumulate_kernel(StatsView sv, int64_t A, int k, const int32_t *__restrict__ src, const int32_t *n_dev,
                        int64_t n_cap, const float *__restrict__ grad, const float *__restrict__ opac,
                        const int32_t *__restrict__ visible) {
    grid_dep_enter();
    const int64_t n = clamp_count(n_cap, n_dev);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t si = src[i];
        const int64_t a = si / k;
        if (si < 0 || a >= A) {
            set_status(sv.status, VPGS_ERR_INVALID_ARG);
            continue;
        }
        atomicAdd(&sv.o_sum[a], opac[i]);
        if (!visible || visible[i] != 0) {
            const float gx = grad[3 * i], gy = grad[3 * i + 1], gz = grad[3 * i + 2];
            atomicAdd(&sv.g_sum[a], sqrtf(gx * gx + gy * gy + gz * gz));
            atomicAdd(&sv.g_cnt[a], 1u);
        }
        if (i == 0 || src[i - 1] / k != a) atomicAdd(&sv.visits[a], 1u);
    }
}

// ---------------------------------------------------------------------------
// update: pruning and growth
// ---------------------------------------------------------------------------
struct UpdState {
    uint32_t ticket[2], status, pad;
};

struct UpdLayout {
    uint32_t cap;
    size_t off_state, off_tab, off_slot, off_look, n_look_a, n_look_n, total;
};

inline UpdLayout upd_layout(int64_t A, int64_t N) {
    UpdLayout L;
    L.cap = table_cap(N);
    size_t o = 0;
    L.off_state = o;
    o += 64;
    L.off_tab = o;
    o += sizeof(VoxEntry) * (size_t)L.cap;
    L.off_slot = o;
    o += align_up(4 * (size_t)N, 16);
    L.off_look = o;
    L.n_look_a = (size_t)std::max<int64_t>(scan_blocks(A), 1);
    L.n_look_n = (size_t)std::max<int64_t>(scan_blocks(N), 1);
    o += 8 * (L.n_look_a + L.n_look_n);
    L.total = o;
    return L;
}

// Clears a first-point table (key empty, lowest index = none), look-back
// words and a small state block.
__global__ void __launch_bounds__(kAThreads)
first_table_clear_kernel(VoxEntry *tab, uint32_t cap, unsigned long long *look, int64_t n_look, uint32_t *state,
                         int n_state) {
    grid_dep_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < cap; i += stride) tab[i] = VoxEntry{kEmptyKey, kNoSlot, 0u};
    for (int64_t i = t0; i < n_look; i += stride) look[i] = 0ull;
    if (t0 < n_state) state[t0] = 0u;
}

struct PruneLoad {
    StatsView sv;
    float tau_o;
    VPGS_D uint32_t operator()(int64_t a) const {
        const uint32_t v = sv.visits[a];
        return (v > 0 && sv.o_sum[a] < __fmul_rn(tau_o, (float)v)) ? 0u : 1u;
    }
};
struct IndexStore {
    int32_t *out;
    VPGS_D void operator()(int64_t i, uint32_t excl, uint32_t v) const {
        if (v) out[excl] = (int32_t)i;
    }
};

// Growth candidates: decoded Gaussians of hot anchors whose voxel holds no
// anchor; the first of each voxel (lowest i) wins the table slot.
__global__ void __launch_bounds__(kAThreads)
grow_insert_kernel(StatsView sv, int k, const int32_t *__restrict__ src, const int32_t *n_dev, int64_t n_cap,
                   const float *__restrict__ means, MapView anchors, float tau_g, VoxEntry *tab, uint32_t mask,
                   uint32_t *__restrict__ slot, uint32_t *status) {
    grid_dep_enter();
    const int64_t n = clamp_count(n_cap, n_dev);
    const bool map_ok = map_header_ok(anchors);
    if (!map_ok && blockIdx.x == 0 && threadIdx.x == 0) set_status(status, VPGS_ERR_INVALID_ARG);
    const float v = anchors.voxel;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t s = kNoSlot;
        const int32_t si = src[i];
        const int64_t a = si / k;
        if (map_ok && si >= 0 && a < anchors.n) {
            const uint32_t c = sv.g_cnt[a];
            if (c > 0 && sv.g_sum[a] > __fmul_rn(tau_g, (float)c)) {
                const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
                int ix, iy, iz;
                if (voxel_index(x, v, ix) && voxel_index(y, v, iy) && voxel_index(z, v, iz)) {
                    const unsigned long long key = pack_voxel(ix, iy, iz);
                    if (find_entry(anchors.tab, anchors.mask, key).b == 0) {
                        bool fresh;
                        s = insert_voxel(tab, mask, key, fresh);
                        if (s == kNoSlot)
                            set_status(status, VPGS_ERR_INTERNAL);
                        else
                            atomicMin(&tab[s].a, (uint32_t)i);
                    }
                } else {
                    set_status(status, isfinite(x) && isfinite(y) && isfinite(z) ? VPGS_ERR_INVALID_ARG
                                                                                   : VPGS_ERR_NONFINITE);
                }
            }
        }
        slot[i] = s;
    }
}

struct FirstLoad {
    const VoxEntry *tab;
    const uint32_t *slot;
    VPGS_D uint32_t operator()(int64_t i) const {
        const uint32_t s = slot[i];
        return (s != kNoSlot && tab[s].a == (uint32_t)i) ? 1u : 0u;
    }
};

// writes the centre of the voxel of point i (stride 3 or 4 floats)
struct CentreStore {
    const float *pts;
    int pstride;
    float v;
    float *out;
    VPGS_D void operator()(int64_t i, uint32_t excl, uint32_t flag) const {
        if (!flag) return;
        int ix = 0, iy = 0, iz = 0;
        voxel_index(pts[pstride * i], v, ix);
        voxel_index(pts[pstride * i + 1], v, iy);
        voxel_index(pts[pstride * i + 2], v, iz);
        out[3 * (int64_t)excl] = voxel_centre(ix, v);
        out[3 * (int64_t)excl + 1] = voxel_centre(iy, v);
        out[3 * (int64_t)excl + 2] = voxel_centre(iz, v);
    }
};

// ---------------------------------------------------------------------------
// spawning
// ---------------------------------------------------------------------------
struct SpawnState {
    uint32_t ticket[2], count, samples, status, pad[3];
};

struct SpawnLayout {
    uint32_t cap;
    size_t off_state, off_list, off_samples, off_slot, off_flag, off_tab, off_look, n_look_p, n_look_m, total;
};

inline SpawnLayout spawn_layout(int64_t P, int64_t M) {
    SpawnLayout L;
    L.cap = table_cap(M);
    size_t o = 0;
    L.off_state = o;
    o += 64;
    L.off_list = o;
    o += align_up(4 * (size_t)P, 16);
    L.off_samples = o;
    o += 16 * (size_t)M;
    L.off_slot = o;
    o += align_up(4 * (size_t)M, 16);
    L.off_flag = o;
    o += align_up(4 * (size_t)M, 16);
    L.off_tab = o;
    o += sizeof(VoxEntry) * (size_t)L.cap;
    L.off_look = o;
    L.n_look_p = (size_t)std::max<int64_t>(scan_blocks(P), 1);
    L.n_look_m = (size_t)std::max<int64_t>(scan_blocks(M), 1);
    o += 8 * (L.n_look_p + L.n_look_m);
    L.total = o;
    return L;
}

struct MaskLoad {
    const float *alpha, *depth, *depth_in;
    float tau_alpha, delta_d;
    VPGS_D uint32_t operator()(int64_t p) const {
        const float di = depth_in[p];
        return (di > 0.f && (alpha[p] < tau_alpha || fabsf(__fsub_rn(depth[p], di)) > delta_d)) ? 1u : 0u;
    }
};
struct ListStore {
    uint32_t *list;
    VPGS_D void operator()(int64_t p, uint32_t excl, uint32_t v) const {
        if (v) list[excl] = (uint32_t)p;
    }
};

struct SpawnCam {
    int W;
    float fx, fy, cx, cy;
};

__global__ void __launch_bounds__(kAThreads)
spawn_sample_kernel(const uint32_t *__restrict__ list, SpawnState *st, int64_t M, SpawnCam cam,
                    const float *__restrict__ depth_in, const double *__restrict__ T, float v,
                    float4 *__restrict__ samples, VoxEntry *tab, uint32_t mask, uint32_t *__restrict__ slot,
                    float *samples_out, int32_t *n_samples) {
    grid_dep_enter();
    const uint64_t C = st->count;
    const uint64_t S = C < (uint64_t)M ? C : (uint64_t)M;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->samples = (uint32_t)S;
        if (n_samples) *n_samples = (int32_t)S;
    }
    double t[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) t[q] = T[q];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < (int64_t)C; r += stride) {
        uint64_t j;
        if (C <= (uint64_t)M) {
            j = (uint64_t)r;
        } else {
            const uint64_t hi = ((uint64_t)r + 1) * (uint64_t)M / C, lo = (uint64_t)r * (uint64_t)M / C;
            if (hi == lo) continue;
            j = hi - 1;
        }
        const uint32_t p = list[r];
        const uint32_t row = p / (uint32_t)cam.W, col = p % (uint32_t)cam.W;
        const double d = depth_in[p];
        // x_c through the pixel centre, then p = R^T (x_c - t), fixed order
        const double xc = __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)col, 0.5), (double)cam.cx), (double)cam.fx), d);
        const double yc = __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)row, 0.5), (double)cam.cy), (double)cam.fy), d);
        const double e0 = __dsub_rn(xc, t[3]), e1 = __dsub_rn(yc, t[7]), e2 = __dsub_rn(d, t[11]);
        float w[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            w[q] = __double2float_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(t[q], e0), __dmul_rn(t[4 + q], e1)), __dmul_rn(t[8 + q], e2)));
        samples[j] = make_float4(w[0], w[1], w[2], 0.f);
        if (samples_out) {
            samples_out[3 * j] = w[0];
            samples_out[3 * j + 1] = w[1];
            samples_out[3 * j + 2] = w[2];
        }
        uint32_t s = kNoSlot;
        int ix, iy, iz;
        if (voxel_index(w[0], v, ix) && voxel_index(w[1], v, iy) && voxel_index(w[2], v, iz)) {
            bool fresh;
            s = insert_voxel(tab, mask, pack_voxel(ix, iy, iz), fresh);
            if (s == kNoSlot)
                set_status(&st->status, VPGS_ERR_INTERNAL);
            else
                atomicMin(&tab[s].a, (uint32_t)j);
        } else {
            set_status(&st->status, isfinite(w[0]) && isfinite(w[1]) && isfinite(w[2]) ? VPGS_ERR_INVALID_ARG
                                                                                       : VPGS_ERR_NONFINITE);
        }
        slot[j] = s;
    }
}

// one warp per sample: flag = first sample of its voxel and no Gaussian mean
// within rho of the voxel centre
__global__ void __launch_bounds__(kAThreads)
spawn_flag_kernel(SpawnState *st, const float4 *__restrict__ samples, const uint32_t *__restrict__ slot,
                  const VoxEntry *tab, MapView gmap, float v, float rho, uint32_t *__restrict__ flag) {
    grid_dep_enter();
    const int lane = threadIdx.x & 31;
    const int64_t S = st->samples;
    const bool map_ok = map_header_ok(gmap);
    if (!map_ok && blockIdx.x == 0 && threadIdx.x == 0) set_status(&st->status, VPGS_ERR_INVALID_ARG);
    const int64_t nw = (int64_t)gridDim.x * (kAThreads / 32);
    for (int64_t j = (int64_t)blockIdx.x * (kAThreads / 32) + (threadIdx.x >> 5); j < S; j += nw) {
        const uint32_t s = slot[j];
        uint32_t f = 0u;
        if (map_ok && s != kNoSlot && tab[s].a == (uint32_t)j) {
            const float4 p = samples[j];
            int ix = 0, iy = 0, iz = 0;
            voxel_index(p.x, v, ix);
            voxel_index(p.y, v, iy);
            voxel_index(p.z, v, iz);
            f = warp_map_any_within(gmap, voxel_centre(ix, v), voxel_centre(iy, v), voxel_centre(iz, v), rho) ? 0u
                                                                                                                : 1u;
        }
        if (lane == 0) flag[j] = f;
    }
}

struct FlagLoad {
    const uint32_t *flag;
    VPGS_D uint32_t operator()(int64_t j) const { return flag[j]; }
};

int warp_grid(int64_t n_warps) {
    const int64_t per = kAThreads / 32;
    const int64_t g = std::min<int64_t>((n_warps + per - 1) / per, (int64_t)device_sm_count() * 8);
    return (int)std::max<int64_t>(g, 1);
}

}  // namespace
}  // namespace vpgs

using namespace vpgs;

extern "C" {

size_t vpgs_anchor_stats_bytes(int64_t n_anchors) {
    if (n_anchors < 0 || n_anchors > (int64_t(1) << 30)) return 0;
    return stats_layout(n_anchors).total;
}

vpgs_status vpgs_anchor_stats_reset(void *stats, size_t stats_bytes, int64_t n_anchors, vpgs_stream stream) {
    const size_t need = vpgs_anchor_stats_bytes(n_anchors);
    if (!stats || !aligned16(stats) || need == 0 || stats_bytes < need) return VPGS_ERR_INVALID_ARG;
    return cudaMemsetAsync(stats, 0, need, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? VPGS_OK
                                                                                                   : VPGS_ERR_CUDA;
}

vpgs_status vpgs_anchor_stats_accumulate(void *stats, size_t stats_bytes, int64_t n_anchors, int32_t k,
                                         const int32_t *src_index, const int32_t *n_dev, int64_t n_cap,
                                         const float *grad_means, const float *opacities, const int32_t *visible,
                                         vpgs_stream stream) {
    const size_t need = vpgs_anchor_stats_bytes(n_anchors);
    if (!stats || !aligned16(stats) || need == 0 || stats_bytes < need || k < 1 || n_cap < 0) return VPGS_ERR_INVALID_ARG;
    if (n_cap > 0 && (!src_index || !grad_means || !opacities)) return VPGS_ERR_INVALID_ARG;
    if (n_cap == 0) return VPGS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VPGS_LAUNCH("anchor_stats", s,
                launch_k(stats_accumulate_kernel, agrid(n_cap), kAThreads, 0, s, stats_view(stats, n_anchors), n_anchors, k,
                                                                           src_index, n_dev, n_cap, grad_means,
                                                                           opacities, visible));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

size_t vpgs_anchor_update_workspace_bytes(int64_t n_anchors, int64_t n_gaussians) {
    if (n_anchors < 0 || n_gaussians < 0 || n_anchors > (int64_t(1) << 30) || n_gaussians > (int64_t(1) << 30))
        return 0;
    return upd_layout(n_anchors, n_gaussians).total;
}

vpgs_status vpgs_anchor_update(void *ws, size_t ws_bytes, const void *stats, size_t stats_bytes, int64_t n_anchors,
                               int32_t k, const int32_t *src_index, const int32_t *n_dev, int64_t n_cap,
                               const float *means, const void *anchor_map, size_t anchor_map_bytes,
                               const vpgs_anchor_update_opts *opts, int32_t *keep_index, int32_t *n_keep,
                               float *grown, int32_t *n_grown, vpgs_stream stream) {
    if (!ws || !aligned16(ws) || !stats || !aligned16(stats) || !opts || !keep_index || !n_keep || !grown ||
        !n_grown || k < 1 || n_cap < 0 || (n_cap > 0 && (!src_index || !means)))
        return VPGS_ERR_INVALID_ARG;
    const vpgs_anchor_update_opts o = *opts;
    if (!std::isfinite(o.tau_g) || !std::isfinite(o.tau_o) || !pos_finite(o.grow_voxel)) return VPGS_ERR_INVALID_ARG;
    const size_t need_s = vpgs_anchor_stats_bytes(n_anchors), need = vpgs_anchor_update_workspace_bytes(n_anchors, n_cap);
    if (need_s == 0 || stats_bytes < need_s || need == 0 || ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    if (!map_args_ok(anchor_map, anchor_map_bytes, n_anchors, o.grow_voxel)) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const UpdLayout L = upd_layout(n_anchors, n_cap);
    char *b = static_cast<char *>(ws);
    UpdState *st = reinterpret_cast<UpdState *>(b + L.off_state);
    VoxEntry *tab = reinterpret_cast<VoxEntry *>(b + L.off_tab);
    uint32_t *slot = reinterpret_cast<uint32_t *>(b + L.off_slot);
    unsigned long long *look = reinterpret_cast<unsigned long long *>(b + L.off_look);
    const StatsView sv = stats_view(const_cast<void *>(stats), n_anchors);
    const int64_t nc = std::max<int64_t>(L.cap, (int64_t)(L.n_look_a + L.n_look_n));
    VPGS_LAUNCH("anchor_update_clear", s,
                launch_k(first_table_clear_kernel, agrid(nc), kAThreads, 0, s, tab, L.cap, look,
                                                                         (int64_t)(L.n_look_a + L.n_look_n),
                                                                         reinterpret_cast<uint32_t *>(st), 16));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (launch_scan("anchor_prune", PruneLoad{sv, o.tau_o}, IndexStore{keep_index}, n_anchors, nullptr, &st->ticket[0],
                    look, reinterpret_cast<uint32_t *>(n_keep), &st->status, s) != cudaSuccess)
        return VPGS_ERR_CUDA;
    if (n_cap == 0) return cudaMemsetAsync(n_grown, 0, 4, s) == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
    const MapView am = map_view(anchor_map, n_anchors, o.grow_voxel);
    VPGS_LAUNCH("anchor_grow_insert", s,
                launch_k(grow_insert_kernel, agrid(n_cap), kAThreads, 0, s, sv, k, src_index, n_dev, n_cap, means, am, o.tau_g,
                                                                      tab, L.cap - 1, slot, &st->status));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (launch_scan("anchor_grow_compact", FirstLoad{tab, slot}, CentreStore{means, 3, o.grow_voxel, grown}, n_cap,
                    reinterpret_cast<const uint32_t *>(n_dev), &st->ticket[1], look + L.n_look_a,
                    reinterpret_cast<uint32_t *>(n_grown), &st->status, s) != cudaSuccess)
        return VPGS_ERR_CUDA;
    return VPGS_OK;
}

size_t vpgs_spawn_workspace_bytes(int32_t width, int32_t height, int32_t max_samples) {
    if (width <= 0 || height <= 0 || width > 65535 || height > 65535 || max_samples < 1 || max_samples > (1 << 26))
        return 0;
    return spawn_layout((int64_t)width * height, max_samples).total;
}

vpgs_status vpgs_spawn_anchors(void *ws, size_t ws_bytes, const float *alpha, const float *depth,
                               const float *depth_in, const vpgs_camera *cam, const double *T_cw,
                               const void *gauss_map, size_t map_bytes, int64_t n_map, float map_voxel,
                               const vpgs_spawn_opts *opts, float *anchors_out, int32_t *n_out, float *samples_out,
                               int32_t *n_samples, vpgs_stream stream) {
    if (!ws || !aligned16(ws) || !alpha || !depth || !depth_in || !cam || !T_cw || !opts || !anchors_out || !n_out)
        return VPGS_ERR_INVALID_ARG;
    const vpgs_spawn_opts o = *opts;
    const size_t need = vpgs_spawn_workspace_bytes(cam->width, cam->height, o.max_samples);
    if (need == 0 || ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    if (!pos_finite(cam->fx) || !pos_finite(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return VPGS_ERR_INVALID_ARG;
    if (!std::isfinite(o.tau_alpha) || !(std::isfinite(o.delta_depth) && o.delta_depth >= 0.f) ||
        !pos_finite(o.voxel) || !pos_finite(o.rho) || o.rho > map_voxel)
        return VPGS_ERR_INVALID_ARG;
    if (!map_args_ok(gauss_map, map_bytes, n_map, map_voxel)) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t P = (int64_t)cam->width * cam->height, M = o.max_samples;
    const SpawnLayout L = spawn_layout(P, M);
    char *b = static_cast<char *>(ws);
    SpawnState *st = reinterpret_cast<SpawnState *>(b + L.off_state);
    uint32_t *list = reinterpret_cast<uint32_t *>(b + L.off_list);
    float4 *samples = reinterpret_cast<float4 *>(b + L.off_samples);
    uint32_t *slot = reinterpret_cast<uint32_t *>(b + L.off_slot);
    uint32_t *flag = reinterpret_cast<uint32_t *>(b + L.off_flag);
    VoxEntry *tab = reinterpret_cast<VoxEntry *>(b + L.off_tab);
    unsigned long long *look = reinterpret_cast<unsigned long long *>(b + L.off_look);
    const int64_t nl = (int64_t)(L.n_look_p + L.n_look_m);
    VPGS_LAUNCH("spawn_clear", s,
                launch_k(first_table_clear_kernel, agrid(std::max<int64_t>(L.cap, nl)), kAThreads, 0, s, 
                    tab, L.cap, look, nl, reinterpret_cast<uint32_t *>(st), 16));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (launch_scan("spawn_mask", MaskLoad{alpha, depth, depth_in, o.tau_alpha, o.delta_depth}, ListStore{list}, P,
                    nullptr, &st->ticket[0], look, &st->count, &st->status, s) != cudaSuccess)
        return VPGS_ERR_CUDA;
    const SpawnCam sc{cam->width, cam->fx, cam->fy, cam->cx, cam->cy};
    VPGS_LAUNCH("spawn_sample", s,
                launch_k(spawn_sample_kernel, agrid(P), kAThreads, 0, s, list, st, M, sc, depth_in, T_cw, o.voxel, samples,
                                                                   tab, L.cap - 1, slot, samples_out, n_samples));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    const MapView gm = map_view(gauss_map, n_map, map_voxel);
    VPGS_LAUNCH("spawn_flag", s,
                launch_k(spawn_flag_kernel, warp_grid(M), kAThreads, 0, s, st, samples, slot, tab, gm, o.voxel, o.rho, flag));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (launch_scan("spawn_compact", FlagLoad{flag},
                    CentreStore{reinterpret_cast<const float *>(samples), 4, o.voxel, anchors_out}, M, &st->samples,
                    &st->ticket[1], look + L.n_look_p, reinterpret_cast<uint32_t *>(n_out), &st->status, s) !=
        cudaSuccess)
        return VPGS_ERR_CUDA;
    return VPGS_OK;
}

vpgs_status vpgs_anchor_status(const void *ws_or_stats, int32_t kind, int64_t n_anchors, int32_t *status_out,
                               vpgs_stream stream) {
    if (!ws_or_stats || !status_out) return VPGS_ERR_INVALID_ARG;
    size_t off;
    if (kind == 0)
        off = stats_layout(n_anchors).off_status;
    else if (kind == 1)
        off = offsetof(UpdState, status);
    else if (kind == 2)
        off = offsetof(SpawnState, status);
    else
        return VPGS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return VPGS_ERR_CUDA;
    uint32_t v = 0;
    if (cudaMemcpy(&v, static_cast<const char *>(ws_or_stats) + off, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return VPGS_ERR_CUDA;
    *status_out = (int32_t)v;
    return VPGS_OK;
}

}  // extern "C"
