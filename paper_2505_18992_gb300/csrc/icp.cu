// Voxel-hash ICP of fine tracking (Sec. III-B, Eq. 10-12).
//
// Map.  The Gaussian means go into an open-addressing hash of their voxels
// (edge v, linear probing, at most half full).  Each occupied voxel records
// the range of its points, which sit grouped by voxel as float4
// (x, y, z, original index).  Built by insert -> scan of the per-voxel counts
// -> scatter; every point of a voxel is kept.
//
// Registration of one scan (local frame) from an initial pose T (local ->
// world, Eq. 10):
//   1. double downsampling: the lowest-index point of each voxel of edge v1
//      (hash insert + atomicMin, then an order-keeping compaction by scan),
//      then the same at v2 over the survivors;
//   2. a fixed number of Gauss-Newton steps, one launch each.  One warp per
//      source point finds the nearest map point closer than tau among the 27
//      voxels around it: lane k probes neighbour k (voxels whose box lies
//      farther than tau are skipped before probing), the home voxel is
//      scanned first, and every other voxel is skipped once its box lies
//      farther than the warp's best distance so far.  The warp's lanes then
//      accumulate the 29 numbers of the Geman-McClure weighted normal
//      equations (Eq. 11-12), lane l owning number l.  The last block to
//      finish adds the block partials in FP64, solves the 6x6 system by
//      Cholesky and updates T in FP64.  A device flag ends the loop early, so
//      the launch sequence is fixed and the call can be captured into a CUDA
//      graph.
// The linearisation is about the centre c = translation of T on entry:
// J = [I, -[s - c]x], T <- Tr(c) Exp(xi) Tr(-c) T.  That gives the same
// iterates as the left perturbation about the origin (Exp(Ad_X xi) =
// X Exp(xi) X^-1) while keeping the FP32 lever arms |s - c| at scan range
// instead of world range.
//
// Decisions are taken in float32 with correctly rounded operations, so that
// they are reproducible off the GPU: the voxel of a coordinate x is
// floor(x / v); the squared distance is (dx^2 + dy^2) + dz^2 of
// d = m - float32(s), accepted when below tau^2, ties to the lower map index.
#include <cmath>

#include "internal.h"
#include "prims.cuh"
#include "profiler.h"
#include "voxhash.cuh"

namespace vpgs {
namespace {

constexpr int kIcpThreads = 256;
constexpr int kIcpWarps = kIcpThreads / kWarp;
constexpr int kSys = 29;  // H upper triangle (21), b (6), sum rho, count
constexpr int kIcpMaxBlocks = 4096;
constexpr int kMinCorr = 6;
constexpr int kStopEps = 1, kStopFew = 2, kStopIndefinite = 3;

struct IcpState {
    uint32_t ticket[2], n1, n2;
    uint32_t status, done, stop, iter;
    double c[3];
    uint32_t blocks_done, pad;
};
static_assert(sizeof(IcpState) <= 128, "state fits its slot");

struct IcpLayout {
    uint32_t cap;
    size_t off_state, off_partial, off_tab1, off_tab2, off_slot1, off_slot2, off_idx1, off_idx2, off_src4,
        off_look, n_look, total;
};

IcpLayout icp_layout(int64_t n) {
    IcpLayout L;
    L.cap = table_cap(n);
    size_t o = 0;
    L.off_state = o;
    o += 128;
    L.off_partial = o;
    o += sizeof(float) * kWarp * kIcpMaxBlocks;
    L.off_tab1 = o;
    o += sizeof(VoxEntry) * (size_t)L.cap;
    L.off_tab2 = o;
    o += sizeof(VoxEntry) * (size_t)L.cap;
    const size_t idx_bytes = align_up(sizeof(uint32_t) * (size_t)n, 16);
    L.off_slot1 = o;
    o += idx_bytes;
    L.off_slot2 = o;
    o += idx_bytes;
    L.off_idx1 = o;
    o += idx_bytes;
    L.off_idx2 = o;
    o += idx_bytes;
    L.off_src4 = o;
    o += sizeof(float4) * (size_t)n;
    L.off_look = o;
    L.n_look = 2 * (size_t)std::max<int64_t>(scan_blocks(n), 1);
    o += sizeof(unsigned long long) * L.n_look;
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// map build
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
map_clear_kernel(MapHeader *hdr, VoxEntry *tab, uint32_t cap, unsigned long long *look, int64_t n_look, int64_t n,
                 float voxel) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < cap; i += stride) tab[i] = VoxEntry{kEmptyKey, 0u, 0u};
    for (int64_t i = t0; i < n_look; i += stride) look[i] = 0ull;
    if (t0 == 0) {
        MapHeader h = {};
        h.magic = kMapMagic;
        h.cap = cap;
        h.n = n;
        h.voxel = voxel;
        *hdr = h;
    }
}

__global__ void __launch_bounds__(256)
map_insert_kernel(const float *__restrict__ pts, int64_t n, float v, VoxEntry *tab, uint32_t mask,
                  uint32_t *__restrict__ slot, MapHeader *hdr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        uint32_t s = kNoSlot;
        int ix, iy, iz;
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
            set_status(&hdr->status, VPGS_ERR_NONFINITE);
        } else if (!(voxel_index(x, v, ix) && voxel_index(y, v, iy) && voxel_index(z, v, iz))) {
            set_status(&hdr->status, VPGS_ERR_INVALID_ARG);
        } else {
            bool fresh;
            s = insert_voxel(tab, mask, pack_voxel(ix, iy, iz), fresh);
            if (s == kNoSlot) {
                set_status(&hdr->status, VPGS_ERR_INTERNAL);
            } else {
                if (fresh) atomicAdd(&hdr->n_voxels, 1u);
                atomicAdd(&tab[s].b, 1u);
            }
        }
        slot[i] = s;
    }
}

struct MapCountLoad {
    const VoxEntry *tab;
    VPGS_D uint32_t operator()(int64_t i) const { return tab[i].b; }
};
struct MapStartStore {
    VoxEntry *tab;
    VPGS_D void operator()(int64_t i, uint32_t excl, uint32_t) const {
        tab[i].a = excl;
        tab[i].b = 0u;  // recounted by the scatter
    }
};

__global__ void __launch_bounds__(256)
map_scatter_kernel(const float *__restrict__ pts, int64_t n, const uint32_t *__restrict__ slot, VoxEntry *tab,
                   float4 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t s = slot[i];
        if (s == kNoSlot) continue;
        const uint32_t pos = tab[s].a + atomicAdd(&tab[s].b, 1u);
        out[pos] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float((int)i));
    }
}

// ---------------------------------------------------------------------------
// double downsampling
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
icp_prepare_kernel(VoxEntry *tab1, VoxEntry *tab2, uint32_t cap, unsigned long long *look, int64_t n_look,
                   IcpState *st, const double *T, const MapHeader *hdr, vpgs_icp_report *rep) {
    grid_dep_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < cap; i += stride) {
        tab1[i] = VoxEntry{kEmptyKey, kNoSlot, 0u};
        tab2[i] = VoxEntry{kEmptyKey, kNoSlot, 0u};
    }
    for (int64_t i = t0; i < n_look; i += stride) look[i] = 0ull;
    if (t0 == 0) {
        IcpState s = {};
        if (T) {
            s.c[0] = T[3];
            s.c[1] = T[7];
            s.c[2] = T[11];
        }
        if (hdr) s.status = hdr->magic == kMapMagic ? hdr->status : (uint32_t)VPGS_ERR_INVALID_ARG;
        *st = s;
        if (rep) {
            vpgs_icp_report r = {};
            r.status = (int32_t)s.status;
            *rep = r;
        }
    }
}

__global__ void __launch_bounds__(256)
ds_insert_kernel(const float *__restrict__ pts, const uint32_t *__restrict__ idx_in, int64_t n_cap,
                 const uint32_t *n_dev, float v, VoxEntry *tab, uint32_t mask, uint32_t *__restrict__ slot,
                 uint32_t *status) {
    grid_dep_enter();
    int64_t n = n_cap;
    if (n_dev) n = min(n, (int64_t)*n_dev);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const int64_t i = idx_in ? (int64_t)idx_in[j] : j;
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        uint32_t s = kNoSlot;
        int ix, iy, iz;
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
            set_status(status, VPGS_ERR_NONFINITE);
        } else if (!(voxel_index(x, v, ix) && voxel_index(y, v, iy) && voxel_index(z, v, iz))) {
            set_status(status, VPGS_ERR_INVALID_ARG);
        } else {
            bool fresh;
            s = insert_voxel(tab, mask, pack_voxel(ix, iy, iz), fresh);
            if (s == kNoSlot)
                set_status(status, VPGS_ERR_INTERNAL);
            else
                atomicMin(&tab[s].a, (uint32_t)j);
        }
        slot[j] = s;
    }
}

struct DsFlagLoad {
    const VoxEntry *tab;
    const uint32_t *slot;
    VPGS_D uint32_t operator()(int64_t j) const {
        const uint32_t s = slot[j];
        return (s != kNoSlot && tab[s].a == (uint32_t)j) ? 1u : 0u;
    }
};
// keeps index j: its original index goes to out[excl] and, when src4 is
// given, its point to src4[excl]
struct DsKeepStore {
    const uint32_t *idx_in;
    uint32_t *out;
    const float *pts;
    float4 *src4;
    VPGS_D void operator()(int64_t j, uint32_t excl, uint32_t v) const {
        if (!v) return;
        const uint32_t i = idx_in ? idx_in[j] : (uint32_t)j;
        out[excl] = i;
        if (src4) src4[excl] = make_float4(pts[3 * (int64_t)i], pts[3 * (int64_t)i + 1], pts[3 * (int64_t)i + 2], 0.f);
    }
};

// ---------------------------------------------------------------------------
// correspondences + normal equations
// ---------------------------------------------------------------------------
// column a of the 3x6 Jacobian [I, -[q]x] of s' = c + Exp(xi)(s - c) at xi = 0:
// e_a for a < 3, e_(a-3) x q for a >= 3 (selected without branches)
VPGS_D float3 jac_col(int a, float qx, float qy, float qz) {
    const float u0 = a == 0, u1 = a == 1, u2 = a == 2, r0 = a == 3, r1 = a == 4, r2 = a == 5;
    return make_float3(u0 + r1 * qz - r2 * qy, u1 + r2 * qx - r0 * qz, u2 + r0 * qy - r1 * qx);
}

VPGS_D float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// Exp of se(3) for xi = (rho, phi) in FP32, returned as the increment
// dR = R - I = A K + B K^2 and te = V rho, V = I + B K + C K^2, with K = [phi]x,
// A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3.  Below
// th = 0.1 the three come from their Taylor series in th^2 (the first omitted
// terms are under 1e-10 relative).  Keeping R - I rather than R lets the FP64
// pose update T + dR T lose nothing to the rounding of the identity.
VPGS_D void se3_exp_delta(const float xi[6], float dR[3][3], float te[3]) {
    const float wx = xi[3], wy = xi[4], wz = xi[5];
    const float t2 = wx * wx + wy * wy + wz * wz;
    float A, B, Cc;
    if (t2 < 1e-2f) {
        A = fmaf(t2, fmaf(t2, fmaf(t2, -1.f / 5040.f, 1.f / 120.f), -1.f / 6.f), 1.f);
        B = fmaf(t2, fmaf(t2, fmaf(t2, -1.f / 40320.f, 1.f / 720.f), -1.f / 24.f), 0.5f);
        Cc = fmaf(t2, fmaf(t2, fmaf(t2, -1.f / 362880.f, 1.f / 5040.f), -1.f / 120.f), 1.f / 6.f);
    } else {
        const float th = sqrtf(t2);
        float sn, cs;
        sincosf(0.5f * th, &sn, &cs);
        const float inv = 1.f / th;
        A = 2.f * sn * cs * inv;
        B = 2.f * sn * sn * inv * inv;
        Cc = (th - 2.f * sn * cs) * inv * inv * inv;
    }
    const float K[3][3] = {{0.f, -wz, wy}, {wz, 0.f, -wx}, {-wy, wx, 0.f}};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float acc = xi[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float k2 = K[r][0] * K[0][c] + K[r][1] * K[1][c] + K[r][2] * K[2][c];
            dR[r][c] = A * K[r][c] + B * k2;
            acc += (B * K[r][c] + Cc * k2) * xi[c];
        }
        te[r] = acc;
    }
}

// One Gauss-Newton step from the summed system (one thread).  H xi = -b is
// solved in FP32 after Jacobi scaling (H~ = S H S, S = diag(H)^-1/2) by an
// LDL^T factorisation: H is taken as positive definite when every pivot of
// H~ is > 0.  The solve's rounding only perturbs the step, not the fixed point
// b = 0, whose sums come in at double-float precision.  Then
// T <- Tr(c) Exp(xi) Tr(-c) T in FP64, the stop flags and the report.
// T_in, c, iter, n2 and status were loaded into shared memory beforehand.
VPGS_D void solve_step(const double *sys, const double *T_in, const double *c, uint32_t iter, uint32_t n2,
                           uint32_t status, double *T, IcpState *st, float eps, vpgs_icp_report *rep) {
    const uint32_t it = iter + 1;
    st->iter = it;
    const double count = sys[28];
    int stop = 0;
    float n2xi = 0.f;
    if (count < kMinCorr) {
        stop = kStopFew;
    } else {
        float H[6][6], L[6][6], D[6], inv[6], sc[6];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int d = i * 6 - i * (i - 1) / 2;  // index of H[i][i] in the upper triangle
            const float hii = (float)sys[d];
            ok = ok && hii > 0.f;
            sc[i] = rsqrtf(hii);
        }
        int k = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int q = r; q < 6; ++q, ++k) H[r][q] = H[q][r] = (float)sys[k] * sc[r] * sc[q];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float d = H[j][j];
#pragma unroll
            for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q] * D[q];
            ok = ok && d > 0.f;  // also false for NaN
            D[j] = d;
            inv[j] = __frcp_rn(d);
#pragma unroll
            for (int i = j + 1; i < 6; ++i) {
                float s = H[i][j];
#pragma unroll
                for (int q = 0; q < j; ++q) s -= L[i][q] * L[j][q] * D[q];
                L[i][j] = s * inv[j];
            }
        }
        if (!ok) {
            stop = kStopIndefinite;
        } else {
            float y[6], x[6], xi[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float s = -(float)sys[21 + i] * sc[i];
#pragma unroll
                for (int q = 0; q < i; ++q) s -= L[i][q] * y[q];
                y[i] = s;
            }
#pragma unroll
            for (int i = 5; i >= 0; --i) {
                float s = y[i] * inv[i];
#pragma unroll
                for (int q = i + 1; q < 6; ++q) s -= L[q][i] * x[q];
                x[i] = s;
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                xi[i] = x[i] * sc[i];
                n2xi = fmaf(xi[i], xi[i], n2xi);
            }
            float dR[3][3], te[3];
            se3_exp_delta(xi, dR, te);
            // T <- Tr(c) Exp(xi) Tr(-c) T = T + dR (T - c) + te in the rotation
            // and translation parts
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double a = T_in[4 * r + q];
#pragma unroll
                    for (int m = 0; m < 3; ++m) a = fma((double)dR[r][m], T_in[4 * m + q], a);
                    T[4 * r + q] = a;
                }
                double a = T_in[4 * r + 3] + (double)te[r];
#pragma unroll
                for (int m = 0; m < 3; ++m) a = fma((double)dR[r][m], T_in[4 * m + 3] - c[m], a);
                T[4 * r + 3] = a;
            }
            if (n2xi < eps * eps) stop = kStopEps;
        }
    }
    if (stop) {
        st->stop = (uint32_t)stop;
        st->done = 1u;
    }
    vpgs_icp_report r;
    r.status = (int32_t)status;
    r.iterations = (int32_t)it;
    r.n_source = (int32_t)n2;
    r.n_corr = (int32_t)count;
    r.stop = stop;
    r.pad = 0;
    r.cost = sys[27];
    r.xi_norm = (double)sqrtf(n2xi);
    *rep = r;
}

VPGS_D float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Source points of one step: float4 (x, y, z, -) when src4 is given, else
// src [n,3] (optionally through idx).
struct SrcView {
    const float4 *src4;
    const float *src;
    const uint32_t *idx;
};

// One linearisation (and, unless sys_out is given, one step) of Eq. 11.
// Blocks whose warps have no source point return at once; the others write
// a partial sum each, and the last of them to finish adds the partials
// (double-float) and solves.
__global__ void __launch_bounds__(kIcpThreads)
icp_step_kernel(MapView map, SrcView sv, int64_t n_cap, const uint32_t *n_dev, double *T,
                const double *__restrict__ centre, float tau, float sigma, float eps, float *partial,
                int32_t *__restrict__ corr, IcpState *st, vpgs_icp_report *rep, double *sys_out) {
    grid_dep_enter();
    __shared__ float s_acc[kIcpWarps][kWarp];
    __shared__ float2 s_part[kIcpWarps][kWarp];
    __shared__ double s_sys[kWarp], s_T[12], s_c[3];
    __shared__ uint32_t s_meta[3];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every load the prologue needs, issued together
    const uint32_t done = st->done;
    const uint32_t n_seen = n_dev ? *n_dev : 0u;
    const MapHeader *h = map.hdr;
    const uint32_t h_magic = h->magic, h_cap = h->cap, h_voxel = __float_as_uint(h->voxel);
    const int64_t h_n = h->n;
    double t[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) t[k] = T[k];
    const double c0 = centre[0], c1 = centre[1], c2 = centre[2];
    if (done) return;  // uniform over the grid: set by an earlier step
    int64_t n = n_cap;
    if (n_dev) n = min(n, (int64_t)n_seen);
    const int64_t nb_active =
        (int64_t)max(1ll, min((long long)gridDim.x, (long long)((n + kIcpWarps - 1) / kIcpWarps)));
    if ((int64_t)blockIdx.x >= nb_active) return;
    // a map buffer that was not built for this size and voxel is never
    // indexed: its ranges could point anywhere
    if (!(h_magic == kMapMagic && h_n == map.n && h_cap == map.mask + 1 && h_voxel == __float_as_uint(map.voxel))) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(&st->status, VPGS_ERR_INVALID_ARG);
        n = 0;
    }
    const float v = map.voxel;
    const float tau2 = __fmul_rn(tau, tau);
    const float kk = sigma / 3.f;
    // lane k < 27 probes neighbour (k % 3 - 1, k / 3 % 3 - 1, k / 9 - 1);
    // lane 13 is the home voxel
    constexpr int kHome = 13;
    const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
    // lane l < 21 owns H[a][b] (upper triangle, row-major), 21..26 b[l-21]
    int ea = 0, eb = 0;
    if (lane < 21) {
        int rem = lane;
        while (rem >= 6 - ea) {
            rem -= 6 - ea;
            ++ea;
        }
        eb = ea + rem;
    } else if (lane < 27) {
        ea = lane - 21;
    }
    float acc = 0.f;
    const int64_t nw = (int64_t)gridDim.x * kIcpWarps;
    for (int64_t j = (int64_t)blockIdx.x * kIcpWarps + warp; j < n; j += nw) {
        double px, py, pz;
        if (sv.src4) {
            const float4 p = sv.src4[j];
            px = p.x;
            py = p.y;
            pz = p.z;
        } else {
            const int64_t i = sv.idx ? (int64_t)sv.idx[j] : j;
            px = sv.src[3 * i];
            py = sv.src[3 * i + 1];
            pz = sv.src[3 * i + 2];
        }
        // s = T p, each coordinate ((T_r0 x + T_r1 y) + T_r2 z) + T_r3 in FP64
        const double sx = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(t[0], px), __dmul_rn(t[1], py)),
                                              __dmul_rn(t[2], pz)), t[3]);
        const double sy = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(t[4], px), __dmul_rn(t[5], py)),
                                              __dmul_rn(t[6], pz)), t[7]);
        const double sz = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(t[8], px), __dmul_rn(t[9], py)),
                                              __dmul_rn(t[10], pz)), t[11]);
        const float fx = __double2float_rn(sx), fy = __double2float_rn(sy), fz = __double2float_rn(sz);
        int cx = 0, cy = 0, cz = 0;
        const bool in_range = voxel_index(fx, v, cx) && voxel_index(fy, v, cy) && voxel_index(fz, v, cz);
        // the slack covers the rounding of the box bounds (a few ulps of |s|)
        const float slack = 1e-4f + 1e-6f * fmaxf(fmaxf(fabsf(fx), fabsf(fy)), fabsf(fz));
        uint32_t start = 0, cnt = 0;
        float gap = 0.f;
        if (in_range && lane < 27) {
            const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
            if (in_voxel_range(nx) && in_voxel_range(ny) && in_voxel_range(nz)) {
                const float gx = slab_gap(nx, v, fx), gy = slab_gap(ny, v, fy), gz = slab_gap(nz, v, fz);
                gap = sqrtf(gx * gx + gy * gy + gz * gz);
                if (gap <= tau + slack) {  // voxels beyond tau are never probed
                    const VoxEntry e = find_entry(map.tab, map.mask, pack_voxel(nx, ny, nz));
                    start = e.a;
                    cnt = e.b;
                }
            }
        }
        float best = tau2;
        uint32_t bidx = kNoSlot;
        float bx = 0.f, by = 0.f, bz = 0.f;
        // Scans the points of the voxels of the lanes in `set` as one list:
        // lane l takes list entries l, l + 32, ...; the voxel of an entry is
        // found by a binary search over the lanes' inclusive count prefix.
        auto scan_set = [&](uint32_t set) {
            const uint32_t ck = (set >> lane) & 1u ? cnt : 0u;
            uint32_t incl = ck;
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - ck;
            const uint32_t total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
            constexpr int kU = 4;  // list entries per lane in flight
            for (uint32_t q0 = 0; q0 < total; q0 += kU * kWarp) {
                float4 m[kU];
                bool ok[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t q = q0 + u * kWarp + lane;
                    int k = 0;
#pragma unroll
                    for (int b = 16; b > 0; b >>= 1)
                        if (__shfl_sync(0xffffffffu, incl, k + b - 1) <= q) k += b;
                    const uint32_t s0 = __shfl_sync(0xffffffffu, start, k);
                    const uint32_t e0 = __shfl_sync(0xffffffffu, excl, k);
                    ok[u] = q < total;
                    m[u] = ok[u] ? map.pts[s0 + (q - e0)] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const float dx = __fsub_rn(m[u].x, fx), dy = __fsub_rn(m[u].y, fy), dz = __fsub_rn(m[u].z, fz);
                    const float d2 =
                        __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                    const uint32_t mi = (uint32_t)__float_as_int(m[u].w);
                    if (ok[u] && (d2 < best || (d2 == best && best < tau2 && mi < bidx))) {
                        best = d2;
                        bidx = mi;
                        bx = m[u].x;
                        by = m[u].y;
                        bz = m[u].z;
                    }
                }
            }
        };
        // first sweep: the home voxel (every live voxel when it is empty);
        // second sweep: the other live voxels not farther than the best so far.
        // A voxel left out of both lies farther than the final best.
        const uint32_t live = __ballot_sync(0xffffffffu, cnt > 0);
        const uint32_t first = (live >> kHome) & 1u ? (1u << kHome) : live;
        if (first) scan_set(first);
        const float lim = sqrtf(warp_min(best)) + slack;
        const uint32_t second = __ballot_sync(0xffffffffu, cnt > 0 && gap <= lim) & ~first;
        if (second) scan_set(second);
        // warp argmin of (d2, map index): every lane ends with the same winner
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const uint32_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            const float ox2 = __shfl_xor_sync(0xffffffffu, bx, o), oy2 = __shfl_xor_sync(0xffffffffu, by, o),
                        oz2 = __shfl_xor_sync(0xffffffffu, bz, o);
            if (ob < best || (ob == best && oi < bidx)) {
                best = ob;
                bidx = oi;
                bx = ox2;
                by = oy2;
                bz = oz2;
            }
        }
        if (corr && lane == 0) corr[j] = bidx == kNoSlot ? -1 : (int32_t)bidx;
        if (bidx != kNoSlot) {
            const float rx = (float)(sx - (double)bx), ry = (float)(sy - (double)by), rz = (float)(sz - (double)bz);
            const float qx = (float)(sx - c0), qy = (float)(sy - c1), qz = (float)(sz - c2);
            const float e2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            const float den = kk + e2;
            const float w = kk / (den * den);  // rho'(e) / e of Eq. 12
            float val = 0.f;
            if (lane < 21) {
                val = w * dot3(jac_col(ea, qx, qy, qz), jac_col(eb, qx, qy, qz));
            } else if (lane < 27) {
                val = w * dot3(jac_col(ea, qx, qy, qz), make_float3(rx, ry, rz));
            } else if (lane == 27) {
                val = 0.5f * e2 / den;  // rho(e)
            } else if (lane == 28) {
                val = 1.f;
            }
            acc += val;
        }
    }
    s_acc[warp][lane] = acc;
    __syncthreads();
    if (threadIdx.x < kWarp) {
        float tot = 0.f;
#pragma unroll
        for (int w = 0; w < kIcpWarps; ++w) tot += s_acc[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * kWarp + threadIdx.x] = tot;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->blocks_done, 1u) == (uint32_t)(nb_active - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: what the solve reads, fetched while the partials are summed
    if (threadIdx.x >= kWarp && threadIdx.x < kWarp + 12) s_T[threadIdx.x - kWarp] = t[threadIdx.x - kWarp];
    if (threadIdx.x == kWarp + 12) {
        s_c[0] = c0;
        s_c[1] = c1;
        s_c[2] = c2;
        s_meta[0] = st->iter;
        s_meta[1] = st->n2;
        s_meta[2] = st->status;
    }
    {
        // double-float sum of the partials in a fixed order; up to 16 loads
        // per thread are in flight at once
        const int comp = threadIdx.x & 31, chunk = threadIdx.x >> 5;
        df a = {0.f, 0.f};
        for (int64_t b0 = chunk; b0 < nb_active; b0 += 16 * kIcpWarps) {
            float x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int64_t b = b0 + (int64_t)u * kIcpWarps;
                x[u] = b < nb_active ? __ldcg(&partial[b * kWarp + comp]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) a = df_add(a, df{x[u], 0.f});
        }
        s_part[chunk][comp] = make_float2(a.hi, a.lo);
    }
    __syncthreads();
    if (threadIdx.x < kWarp) {
        df a = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < kIcpWarps; ++c) a = df_add(a, df{s_part[c][threadIdx.x].x, s_part[c][threadIdx.x].y});
        s_sys[threadIdx.x] = (double)a.hi + (double)a.lo;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    st->blocks_done = 0u;  // ready for the next step
    if (sys_out) {         // linearisation only
        for (int k = 0; k < kSys; ++k) sys_out[k] = s_sys[k];
        return;
    }
    solve_step(s_sys, s_T, s_c, s_meta[0], s_meta[1], s_meta[2], T, st, eps, rep);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
int fill_grid(int64_t n) {
    const int64_t g = std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8);
    return (int)std::max<int64_t>(g, 1);
}

int corr_grid() {
    static std::atomic<int> cache[kDeviceCache];
    return per_device(cache, [] { return resident_grid((const void *)icp_step_kernel, kIcpThreads, 0, kIcpMaxBlocks); });
}

struct IcpWsView {
    IcpLayout L;
    IcpState *st;
    float *partial;
    VoxEntry *tab1, *tab2;
    uint32_t *slot1, *slot2, *idx1, *idx2;
    float4 *src4;
    unsigned long long *look;
};

IcpWsView carve_icp(void *ws, int64_t n) {
    IcpWsView w;
    w.L = icp_layout(n);
    char *b = static_cast<char *>(ws);
    w.st = reinterpret_cast<IcpState *>(b + w.L.off_state);
    w.partial = reinterpret_cast<float *>(b + w.L.off_partial);
    w.tab1 = reinterpret_cast<VoxEntry *>(b + w.L.off_tab1);
    w.tab2 = reinterpret_cast<VoxEntry *>(b + w.L.off_tab2);
    w.slot1 = reinterpret_cast<uint32_t *>(b + w.L.off_slot1);
    w.slot2 = reinterpret_cast<uint32_t *>(b + w.L.off_slot2);
    w.idx1 = reinterpret_cast<uint32_t *>(b + w.L.off_idx1);
    w.idx2 = reinterpret_cast<uint32_t *>(b + w.L.off_idx2);
    w.src4 = reinterpret_cast<float4 *>(b + w.L.off_src4);
    w.look = reinterpret_cast<unsigned long long *>(b + w.L.off_look);
    return w;
}

cudaError_t launch_prepare(const IcpWsView &w, const double *T, const MapHeader *hdr, vpgs_icp_report *rep,
                           cudaStream_t s) {
    const int64_t n = std::max<int64_t>(w.L.cap, (int64_t)w.L.n_look);
    VPGS_LAUNCH("icp_prepare", s,
                launch_k(icp_prepare_kernel, fill_grid(n), 256, 0, s, w.tab1, w.tab2, w.L.cap, w.look,
                                                                (int64_t)w.L.n_look, w.st, T, hdr, rep));
    return cudaGetLastError();
}

// Two first-point passes; the kept original indices go to out[0 .. *count)
// and, when src4 is given, the kept points to src4[0 .. *count).
cudaError_t launch_downsample(const IcpWsView &w, const float *scan, int64_t n, float v1, float v2, uint32_t *out,
                              float4 *src4, uint32_t *count, cudaStream_t s) {
    const uint32_t mask = w.L.cap - 1;
    const size_t half = w.L.n_look / 2;
    VPGS_LAUNCH("icp_ds_insert", s,
                launch_k(ds_insert_kernel, fill_grid(n), 256, 0, s, scan, nullptr, n, nullptr, v1, w.tab1, mask, w.slot1,
                                                              &w.st->status));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan("icp_ds_compact", DsFlagLoad{w.tab1, w.slot1}, DsKeepStore{nullptr, w.idx1, scan, nullptr}, n, nullptr,
                    &w.st->ticket[0], w.look, &w.st->n1, &w.st->status, s);
    if (e != cudaSuccess) return e;
    VPGS_LAUNCH("icp_ds_insert", s,
                launch_k(ds_insert_kernel, fill_grid(n), 256, 0, s, scan, w.idx1, n, &w.st->n1, v2, w.tab2, mask, w.slot2,
                                                              &w.st->status));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_scan("icp_ds_compact", DsFlagLoad{w.tab2, w.slot2}, DsKeepStore{w.idx1, out, scan, src4}, n, &w.st->n1,
                       &w.st->ticket[1], w.look + half, count, &w.st->status, s);
}

}  // namespace
}  // namespace vpgs

using namespace vpgs;

extern "C" {

size_t vpgs_icp_map_bytes(int64_t n_points) {
    if (n_points < 0 || n_points > (int64_t(1) << 30)) return 0;
    return map_layout(n_points).total;
}

vpgs_status vpgs_icp_build_map(void *map, size_t map_bytes, const float *points, int64_t n_points, float voxel,
                               vpgs_stream stream) {
    if (!map_args_ok(map, map_bytes, n_points, voxel)) return VPGS_ERR_INVALID_ARG;
    if (n_points > 0 && !points) return VPGS_ERR_INVALID_ARG;
    const MapLayout L = map_layout(n_points);
    char *b = static_cast<char *>(map);
    MapHeader *hdr = reinterpret_cast<MapHeader *>(b);
    VoxEntry *tab = reinterpret_cast<VoxEntry *>(b + L.off_tab);
    float4 *pts = reinterpret_cast<float4 *>(b + L.off_pts);
    uint32_t *slot = reinterpret_cast<uint32_t *>(b + L.off_slot);
    unsigned long long *look = reinterpret_cast<unsigned long long *>(b + L.off_look);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nc = std::max<int64_t>(L.cap, (int64_t)L.n_look);
    VPGS_LAUNCH("icp_map_clear", s,
                map_clear_kernel<<<fill_grid(nc), 256, 0, s>>>(hdr, tab, L.cap, look, (int64_t)L.n_look, n_points,
                                                               voxel));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (n_points == 0) return VPGS_OK;
    VPGS_LAUNCH("icp_map_insert", s,
                map_insert_kernel<<<fill_grid(n_points), 256, 0, s>>>(points, n_points, voxel, tab, L.cap - 1, slot,
                                                                      hdr));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    if (launch_scan("icp_map_offsets", MapCountLoad{tab}, MapStartStore{tab}, (int64_t)L.cap, nullptr, &hdr->ticket,
                    look, &hdr->total, &hdr->status, s) != cudaSuccess)
        return VPGS_ERR_CUDA;
    VPGS_LAUNCH("icp_map_scatter", s,
                map_scatter_kernel<<<fill_grid(n_points), 256, 0, s>>>(points, n_points, slot, tab, pts));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

vpgs_status vpgs_icp_map_query(const void *map, vpgs_icp_map_info *info, vpgs_stream stream) {
    if (!map || !info) return VPGS_ERR_INVALID_ARG;
    MapHeader h;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return VPGS_ERR_CUDA;
    if (cudaMemcpy(&h, map, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return VPGS_ERR_CUDA;
    if (h.magic != kMapMagic) return VPGS_ERR_INVALID_ARG;
    info->n_points = h.n;
    info->n_voxels = (int32_t)h.n_voxels;
    info->capacity = (int32_t)h.cap;
    info->status = (int32_t)h.status;
    info->voxel = h.voxel;
    return VPGS_OK;
}

size_t vpgs_icp_workspace_bytes(int64_t n_scan) {
    if (n_scan < 0 || n_scan > (int64_t(1) << 30)) return 0;
    return icp_layout(n_scan).total;
}

vpgs_status vpgs_icp_downsample(void *ws, size_t ws_bytes, const float *scan, int64_t n_scan, float voxel_1,
                                float voxel_2, int32_t *idx_out, int32_t *n_out, vpgs_stream stream) {
    if (!ws || !aligned16(ws) || !idx_out || !n_out || n_scan < 0 || (n_scan > 0 && !scan)) return VPGS_ERR_INVALID_ARG;
    if (!pos_finite(voxel_1) || !pos_finite(voxel_2)) return VPGS_ERR_INVALID_ARG;
    const size_t need = vpgs_icp_workspace_bytes(n_scan);
    if (need == 0 || ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const IcpWsView w = carve_icp(ws, n_scan);
    if (launch_prepare(w, nullptr, nullptr, nullptr, s) != cudaSuccess) return VPGS_ERR_CUDA;
    if (n_scan == 0) return cudaMemsetAsync(n_out, 0, sizeof(int32_t), s) == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
    return launch_downsample(w, scan, n_scan, voxel_1, voxel_2, reinterpret_cast<uint32_t *>(idx_out), nullptr,
                             reinterpret_cast<uint32_t *>(n_out), s) == cudaSuccess
               ? VPGS_OK
               : VPGS_ERR_CUDA;
}

vpgs_status vpgs_icp_linearize(void *ws, size_t ws_bytes, const void *map, size_t map_bytes, int64_t n_map,
                               float map_voxel, const float *src, int64_t n_src, const double *T,
                               const double *centre, float tau, float sigma, double *system, int32_t *corr,
                               vpgs_stream stream) {
    if (!ws || !aligned16(ws) || !T || !centre || !system || n_src < 0 || (n_src > 0 && !src))
        return VPGS_ERR_INVALID_ARG;
    if (!map_args_ok(map, map_bytes, n_map, map_voxel)) return VPGS_ERR_INVALID_ARG;
    if (!pos_finite(tau) || tau > map_voxel || !pos_finite(sigma)) return VPGS_ERR_INVALID_ARG;
    const size_t need = vpgs_icp_workspace_bytes(0);
    if (ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const IcpWsView w = carve_icp(ws, 0);
    const MapView mv = map_view(map, n_map, map_voxel);
    if (launch_prepare(w, nullptr, mv.hdr, nullptr, s) != cudaSuccess) return VPGS_ERR_CUDA;
    VPGS_LAUNCH("icp_step", s,
                launch_k(icp_step_kernel, corr_grid(), kIcpThreads, 0, s, mv, SrcView{nullptr, src, nullptr}, n_src, nullptr,
                                                                    const_cast<double *>(T), centre, tau, sigma, 0.f,
                                                                    w.partial, corr, w.st, nullptr, system));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

vpgs_status vpgs_icp_register(void *ws, size_t ws_bytes, const void *map, size_t map_bytes, int64_t n_map,
                              const float *scan, int64_t n_scan, const vpgs_icp_opts *opts, double *T,
                              vpgs_icp_report *report, vpgs_stream stream) {
    if (!ws || !aligned16(ws) || !opts || !T || !report || n_scan < 0 || (n_scan > 0 && !scan))
        return VPGS_ERR_INVALID_ARG;
    const vpgs_icp_opts o = *opts;
    if (!map_args_ok(map, map_bytes, n_map, o.map_voxel)) return VPGS_ERR_INVALID_ARG;
    if (!pos_finite(o.voxel_1) || !pos_finite(o.voxel_2) || !pos_finite(o.tau) || o.tau > o.map_voxel ||
        !pos_finite(o.sigma) || !(std::isfinite(o.eps) && o.eps >= 0.f) || o.iterations < 1 ||
        o.iterations > 1000)
        return VPGS_ERR_INVALID_ARG;
    const size_t need = vpgs_icp_workspace_bytes(n_scan);
    if (need == 0 || ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const IcpWsView w = carve_icp(ws, n_scan);
    const MapView mv = map_view(map, n_map, o.map_voxel);
    if (launch_prepare(w, T, mv.hdr, report, s) != cudaSuccess) return VPGS_ERR_CUDA;
    if (n_scan > 0 && launch_downsample(w, scan, n_scan, o.voxel_1, o.voxel_2, w.idx2, w.src4, &w.st->n2, s) != cudaSuccess)
        return VPGS_ERR_CUDA;
    const int nb = corr_grid();
    for (int it = 0; it < o.iterations; ++it) {
        VPGS_LAUNCH("icp_step", s,
                    launch_k(icp_step_kernel, nb, kIcpThreads, 0, s, mv, SrcView{w.src4, nullptr, nullptr}, n_scan,
                                                               &w.st->n2, T, w.st->c,
                                                               o.tau, o.sigma, o.eps, w.partial, nullptr, w.st,
                                                               report, nullptr));
        if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    }
    return VPGS_OK;
}

}  // extern "C"
