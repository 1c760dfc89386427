// Per-Gaussian projection (EWA splatting) and its backward pass.
//
// Forward (a pre-cull with one thread per Gaussian over all views, then the
// exact projection with one thread per surviving (view, Gaussian)):
//   p_c = R mu + t (double-float), u = fx x/z + cx, v = fy y/z + cy (double-float)
//   Sigma' = J R Sigma R^T J^T + dilation I = K K^T + dilation I,  K = J R R(q) S
//   det(Sigma') via the Lagrange identity |K0 x K1|^2 + ... (no cancellation)
//   whitening rows from the eigenvectors of Sigma'
//   extent: half widths sqrt(2 ln(o/alpha_min) Sigma'_xx), sqrt(... Sigma'_yy),
//           widened by 1e-5 r + 2e-3 px so the pixel set is a superset of the
//           exact one; the alpha test at each pixel then decides membership
//   tile count: the tiles of that box whose pixel-centre rectangle (widened
//           by the same margins) meets the alpha_min ellipse, row by row
// Backward, one thread per visible (view, Gaussian): chain rule from the 2D
// gradients (u, v, conic, opacity, colour, depth) back to mean, scale,
// quaternion, opacity and colour, plus the per-view pose terms summed in FP64.
#include "internal.h"
#include "prims.cuh"
#include "profiler.h"

namespace vpgs {

struct Proj {
    df pc[3];
    float px, py, pz;          // camera-space point (rounded)
    float xz, yz, iz;          // x/z, y/z, 1/z
    float j00, j02, j11, j12;  // projection Jacobian
    float Wf[9];               // world->camera rotation (float)
    float Rq[9];               // rotation of the quaternion
    float WR[9];               // Wf * Rq
    float K0[3], K1[3];        // J * WR * S rows
    float A, B, C, det;        // Sigma' = [[A,B],[B,C]]
    df u, v;
};

VPGS_D void project(const PoseDF &P, float mx, float my, float mz, float sx, float sy, float sz,
                    float qw, float qx, float qy, float qz, const CamParams &cam, float dil,
                    Proj &p) {
    transform_df(P, mx, my, mz, p.pc);
    p.px = p.pc[0].hi;
    p.py = p.pc[1].hi;
    p.pz = p.pc[2].hi;
    df qxz = df_div(p.pc[0], p.pc[2]);
    df qyz = df_div(p.pc[1], p.pc[2]);
    p.u = df_add(df_mul_f(qxz, cam.fx), df{cam.cx, 0.f});
    p.v = df_add(df_mul_f(qyz, cam.fy), df{cam.cy, 0.f});
    p.xz = qxz.hi;
    p.yz = qyz.hi;
    p.iz = 1.0f / p.pz;
    p.j00 = cam.fx * p.iz;
    p.j02 = -cam.fx * p.xz * p.iz;
    p.j11 = cam.fy * p.iz;
    p.j12 = -cam.fy * p.yz * p.iz;
#pragma unroll
    for (int k = 0; k < 9; ++k) p.Wf[k] = P.R[k].hi;
    quat_to_rot(qw, qx, qy, qz, p.Rq);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            p.WR[3 * r + c] = fmaf(p.Wf[3 * r], p.Rq[c],
                                   fmaf(p.Wf[3 * r + 1], p.Rq[3 + c], p.Wf[3 * r + 2] * p.Rq[6 + c]));
    const float s[3] = {sx, sy, sz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p.K0[c] = (p.j00 * p.WR[c] + p.j02 * p.WR[6 + c]) * s[c];
        p.K1[c] = (p.j11 * p.WR[3 + c] + p.j12 * p.WR[6 + c]) * s[c];
    }
    float n0 = p.K0[0] * p.K0[0] + p.K0[1] * p.K0[1] + p.K0[2] * p.K0[2];
    float n1 = p.K1[0] * p.K1[0] + p.K1[1] * p.K1[1] + p.K1[2] * p.K1[2];
    p.B = p.K0[0] * p.K1[0] + p.K0[1] * p.K1[1] + p.K0[2] * p.K1[2];
    p.A = n0 + dil;
    p.C = n1 + dil;
    float c0 = p.K0[1] * p.K1[2] - p.K0[2] * p.K1[1];
    float c1 = p.K0[2] * p.K1[0] - p.K0[0] * p.K1[2];
    float c2 = p.K0[0] * p.K1[1] - p.K0[1] * p.K1[0];
    p.det = (c0 * c0 + c1 * c1 + c2 * c2) + dil * (n0 + n1) + dil * dil;
}

// Conservative FP32 pre-cull.  False only when the Gaussian certainly lies
// behind the near plane or its whole alpha_min extent certainly misses the
// image: p_c carries a 1e-5 relative error bound (about 40 times the FP32
// rounding of the transform), and the screen half width is bounded through
// Sigma'_xx <= (fx/z)^2 (1 + (x/z)^2) s_max^2 + dilation (and likewise in y),
// plus a pixel of slack.  The exact double-float path decides everything else.
VPGS_D bool maybe_in_view(const PoseDF &P, float mx, float my, float mz, float smax, float kq,
                          const CamParams &cam, const OptParams &o) {
    float pc[3], tol[3];
    const float am = fabsf(mx) + fabsf(my) + fabsf(mz);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        pc[r] = fmaf(P.R[3 * r].hi, mx, fmaf(P.R[3 * r + 1].hi, my, fmaf(P.R[3 * r + 2].hi, mz, P.t[r].hi)));
        tol[r] = 1e-5f * (am + fabsf(P.t[r].hi)) + 1e-6f;
    }
    if (pc[2] + tol[2] <= o.near_z) return false;
    const float zl = pc[2] - tol[2];
    if (!(zl > 1e-3f)) return true;  // too close to z = 0 for a bound: the exact path decides
    // approximate reciprocal and square roots (a few ulp): the 1 px and 1e-4 slack below cover them
    const float iz = __fdividef(1.0f, zl);
    const float kqc = fmaxf(kq, 0.f);
    const float xr = (fabsf(pc[0]) + tol[0]) * iz, yr = (fabsf(pc[1]) + tol[1]) * iz;
    const float qx = kqc * (cam.fx * cam.fx * iz * iz * (1.f + xr * xr) * smax * smax + o.dilation);
    const float qy = kqc * (cam.fy * cam.fy * iz * iz * (1.f + yr * yr) * smax * smax + o.dilation);
    const float rx = qx > 0.f ? qx * rsqrtf(qx) : 0.f, ry = qy > 0.f ? qy * rsqrtf(qy) : 0.f;
    // image mean and its error bound
    const float izc = __fdividef(1.0f, pc[2]);
    const float u = fmaf(cam.fx, pc[0] * izc, cam.cx), v = fmaf(cam.fy, pc[1] * izc, cam.cy);
    const float eu = 2.f * cam.fx * (tol[0] + xr * tol[2]) * iz + 1e-4f * fabsf(u);
    const float ev = 2.f * cam.fy * (tol[1] + yr * tol[2]) * iz + 1e-4f * fabsf(v);
    const float sx = 1.001f * rx + eu + 1.f, sy = 1.001f * ry + ev + 1.f;
    return !(u + sx < 0.f || u - sx > (float)cam.W || v + sy < 0.f || v - sy > (float)cam.H);
}

// First kernel of a render call: zeroes the status word, the counters and the
// scratch the later kernels expect at zero (scan look-back words, both sorts'
// digit histograms and first-pass look-back words, tile ranges), and converts
// the poses to double-float pairs.  One launch instead of a memset per array.
struct PrepZero {
    uint32_t *w32[6];
    int64_t n32[6];
    unsigned long long *w64;
    int64_t n64;
};

__global__ void __launch_bounds__(256)
prepare_kernel(const double *__restrict__ T_cw, int V, float *posedf, PrepZero z) {
    grid_dep_enter();
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll
    for (int a = 0; a < 6; ++a)
        for (int64_t i = t0; i < z.n32[a]; i += stride) z.w32[a][i] = 0u;
    for (int64_t i = t0; i < z.n64; i += stride) z.w64[i] = 0ull;
    for (int64_t v = t0; v < V; v += stride) pose_to_df(T_cw + 16 * v, posedf + 24 * v);
}

// Near-degenerate 2D covariances.  The FP32 whitening rows carry a direction
// error of ~1e-7 rad; along a Gaussian of condition number kappa = l1/l2 that
// moves the second whitened coordinate t2 = w2.d by ~1e-7 sqrt(kappa) at the
// pixels where alpha matters, and alpha by about that much relative.  Above
// kFineKappa the covariance and its inverse square root are therefore taken
// in FP64 from the FP32 inputs, the second row is kept as a double-float pair
// (its low parts in the record), and the compositing kernels evaluate t2 in
// double-float for such records (flagged by a negative y half extent).
constexpr float kFineKappa = 256.f;

struct FineCov {
    float A, B, C, det;       // Sigma' rounded from FP64
    float w1x, w1y;           // first whitening row (times kRowScale)
    df w2x, w2y;              // second whitening row (times kRowScale), double-float
};

VPGS_D double dsum(const df &x) { return (double)x.hi + (double)x.lo; }

// pd: the view's pose as double-float pairs (re-read here, so that the common
// path holds no pose registers across this rare one)
VPGS_D void fine_cov(const float *pd, const df pc[3], float sx, float sy, float sz, float qw, float qx,
                     float qy, float qz, const CamParams &cam, float dil, FineCov &fc) {
    const double x = dsum(pc[0]), y = dsum(pc[1]), z = dsum(pc[2]);
    const double iz = 1.0 / z;
    const double fx = cam.fx, fy = cam.fy;
    const double j00 = fx * iz, j02 = -fx * x * iz * iz, j11 = fy * iz, j12 = -fy * y * iz * iz;
    double w = qw, a = qx, b = qy, c = qz;
    const double inv = 1.0 / sqrt(w * w + a * a + b * b + c * c);
    w *= inv; a *= inv; b *= inv; c *= inv;
    const double Rq[9] = {1.0 - 2.0 * (b * b + c * c), 2.0 * (a * b - w * c), 2.0 * (a * c + w * b),
                          2.0 * (a * b + w * c), 1.0 - 2.0 * (a * a + c * c), 2.0 * (b * c - w * a),
                          2.0 * (a * c - w * b), 2.0 * (b * c + w * a), 1.0 - 2.0 * (a * a + b * b)};
    const double sv[3] = {sx, sy, sz};
    double K0[3], K1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        double wr[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double R0 = (double)pd[2 * (3 * r)] + (double)pd[2 * (3 * r) + 1];
            const double R1 = (double)pd[2 * (3 * r + 1)] + (double)pd[2 * (3 * r + 1) + 1];
            const double R2 = (double)pd[2 * (3 * r + 2)] + (double)pd[2 * (3 * r + 2) + 1];
            wr[r] = R0 * Rq[col] + R1 * Rq[3 + col] + R2 * Rq[6 + col];
        }
        K0[col] = (j00 * wr[0] + j02 * wr[2]) * sv[col];
        K1[col] = (j11 * wr[1] + j12 * wr[2]) * sv[col];
    }
    const double n0 = K0[0] * K0[0] + K0[1] * K0[1] + K0[2] * K0[2];
    const double n1 = K1[0] * K1[0] + K1[1] * K1[1] + K1[2] * K1[2];
    const double B = K0[0] * K1[0] + K0[1] * K1[1] + K0[2] * K1[2];
    const double e = dil, A = n0 + e, C = n1 + e;
    const double c0 = K0[1] * K1[2] - K0[2] * K1[1], c1 = K0[2] * K1[0] - K0[0] * K1[2],
                 c2 = K0[0] * K1[1] - K0[1] * K1[0];
    const double det = (c0 * c0 + c1 * c1 + c2 * c2) + e * (n0 + n1) + e * e;
    const double h = 0.5 * (A - C), r = sqrt(h * h + B * B);
    const double l1 = 0.5 * (A + C) + r, l2 = det / l1;
    double ex, ey;
    if (r == 0.0) {
        ex = 1.0; ey = 0.0;
    } else if (h >= 0.0) {
        ex = h + r; ey = B;
    } else {
        ex = B; ey = r - h;
    }
    const double en = 1.0 / sqrt(ex * ex + ey * ey);
    ex *= en; ey *= en;
    const double s1 = (double)kRowScale / sqrt(l1), s2 = (double)kRowScale / sqrt(l2);
    fc.A = (float)A; fc.B = (float)B; fc.C = (float)C; fc.det = (float)det;
    fc.w1x = (float)(ex * s1);
    fc.w1y = (float)(ey * s1);
    fc.w2x = df_from_double(-ey * s2);
    fc.w2y = df_from_double(ex * s2);
}

// Exact projection, extent and tile cover of one (view, Gaussian) that passed
// the pre-cull.  Returns its tile count (0: culled); the screen record is
// written to *R as soon as it is known (its contents do not matter when the
// count is 0, and writing early keeps it out of registers across the cover),
// B is filled when the count is > 0.
VPGS_D uint32_t project_one(const float *pd, float mx, float my, float mz, float sx, float sy, float sz,
                            float4 q, float op, float cr, float cg, float cb, const CamParams &cam,
                            const OptParams &o, uint32_t *status, Rec *R, BinRec &B, float &depth) {
    Proj p;
    {
        PoseDF P;
        load_pose(pd, P);
        project(P, mx, my, mz, sx, sy, sz, q.x, q.y, q.z, q.w, cam, o.dilation, p);
    }
    const bool in_front = p.pc[2].hi > o.near_z || (p.pc[2].hi == o.near_z && p.pc[2].lo > 0.f);
    if (!in_front) return 0u;
    // eigen-decomposition of Sigma' (2x2 symmetric) for the whitening rows
    const float h = 0.5f * (p.A - p.C);
    const float r = hypotf(h, p.B);
    const float lam1 = 0.5f * (p.A + p.C) + r;
    const float lam2 = p.det / lam1;
    float ex, ey;
    if (r == 0.f) {
        ex = 1.f; ey = 0.f;
    } else if (h >= 0.f) {
        ex = h + r; ey = p.B;
    } else {
        ex = p.B; ey = r - h;
    }
    const float en = 1.0f / sqrtf(ex * ex + ey * ey);
    ex *= en; ey *= en;
    const float s1 = kRowScale / sqrtf(lam1), s2 = kRowScale / sqrtf(lam2);
    float4 w = make_float4(ex * s1, ey * s1, -ey * s2, ex * s2);
    float w2x_lo = 0.f, w2y_lo = 0.f;
    const bool fine = lam1 > kFineKappa * lam2;  // near-degenerate (NaN: the finiteness test below)
    if (fine) {
        FineCov fc;
        fine_cov(pd, p.pc, sx, sy, sz, q.x, q.y, q.z, q.w, cam, o.dilation, fc);
        p.A = fc.A; p.B = fc.B; p.C = fc.C; p.det = fc.det;
        w = make_float4(fc.w1x, fc.w1y, fc.w2x.hi, fc.w2y.hi);
        w2x_lo = fc.w2x.lo;
        w2y_lo = fc.w2y.lo;
    }
    // opacity-aware extent
    const float kq = 2.0f * logf(op / o.alpha_min);
    const float rx = sqrtf(fmaxf(kq, 0.f) * p.A), ry = sqrtf(fmaxf(kq, 0.f) * p.C);
    const float rxe = rx * (1.0f + 1e-5f) + 2e-3f, rye = ry * (1.0f + 1e-5f) + 2e-3f;
    const float uf = p.u.hi, vf = p.v.hi;
    float lx = (uf - 0.5f - rxe) + p.u.lo, hx = (uf - 0.5f + rxe) + p.u.lo;
    float ly = (vf - 0.5f - rye) + p.v.lo, hy = (vf - 0.5f + rye) + p.v.lo;
    if (!isfinite(lx + hx + ly + hy + w.x + w.y + w.z + w.w + w2x_lo + w2y_lo)) {
        set_status(status, VPGS_ERR_NONFINITE);
        return 0u;
    }
    R->r0 = make_float4(p.u.hi, p.v.hi, p.u.lo, p.v.lo);
    R->r1 = w;
    R->r2 = make_float4(op, p.pz, cr, cg);
    R->r3 = make_float4(cb, w2x_lo, fine ? -rye : rye, w2y_lo);
    lx = fmaxf(lx, -1.f); hx = fminf(hx, (float)cam.W);
    ly = fmaxf(ly, -1.f); hy = fminf(hy, (float)cam.H);
    const int x0 = max(0, (int)ceilf(lx)), x1 = min(cam.W - 1, (int)floorf(hx));
    const int y0 = max(0, (int)ceilf(ly)), y1 = min(cam.H - 1, (int)floorf(hy));
    if (!(x0 <= x1 && y0 <= y1)) return 0u;
    const int tx0 = x0 >> cam.tw_shift, tx1 = x1 >> cam.tw_shift;
    const int ty0 = y0 / cam.tile_h, ty1 = y1 / cam.tile_h;
    Cover cv;
    const float kc = fmaxf(kq, 0.f), iC = 1.0f / p.C, dC = p.det * iC;
    cv.a = make_float4(ry, fmaf(ry, 1e-5f, 2e-3f), -p.B * sqrtf(kc / p.A), p.B * iC);
    cv.b = make_float4(kc * dC, dC * iC, fmaf(rx, 1e-5f, 2e-3f), 0.f);
    uint32_t cnt = 0;
    const int rows = ty1 - ty0 + 1;
    if (rows <= kCoverRows) {
        // few rows: keep the spans themselves for the emitting pass
        uint32_t pk[kCoverRows];
#pragma unroll
        for (int k = 0; k < kCoverRows; ++k) {
            pk[k] = kEmptySpan;
            if (k < rows) {
                const int2 sp = cover_row(cv, p.u.hi, p.u.lo, p.v.hi, p.v.lo, ty0 + k, tx0, tx1, cam.tw_shift,
                                          cam.tile_h, cam.W, cam.H);
                if (sp.x <= sp.y) {
                    cnt += (uint32_t)(sp.y - sp.x + 1);
                    pk[k] = (uint32_t)sp.x | ((uint32_t)sp.y << 16);
                }
            }
        }
        cv.a = make_float4(__uint_as_float(pk[0]), __uint_as_float(pk[1]), __uint_as_float(pk[2]),
                           __uint_as_float(pk[3]));
        cv.b = make_float4(__uint_as_float(pk[4]), __uint_as_float(pk[5]), __uint_as_float(pk[6]),
                           __uint_as_float(pk[7]));
    } else {
        for (int ty = ty0; ty <= ty1; ++ty) {
            const int2 sp = cover_row(cv, p.u.hi, p.u.lo, p.v.hi, p.v.lo, ty, tx0, tx1, cam.tw_shift, cam.tile_h,
                                      cam.W, cam.H);
            if (sp.x <= sp.y) cnt += (uint32_t)(sp.y - sp.x + 1);
        }
    }
    if (cnt == 0u) return 0u;
    depth = p.pz;
    B.uv = make_float4(p.u.hi, p.v.hi, p.u.lo, p.v.lo);
    B.rect = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    B.cnt = cnt;
    B.pad = 0u;
    B.cv = cv;
    return cnt;
}

// Pass 1, one thread per Gaussian over all views: finiteness check, opacity test
// and the FP32 pre-cull of each (view, Gaussian) pair.  Survivors are appended
// to a candidate list (block-level compaction, one atomic per block and round
// of 8 views); every other pair gets tile count 0.
constexpr int kPreThreads = 256;

__global__ void __launch_bounds__(kPreThreads)
precull_kernel(GaussIn g, int V, CamParams cam, OptParams o, RenderWs ws, uint32_t *cand,
               uint32_t *n_cand) {
    grid_dep_enter();
    // one thread per Gaussian: its parameters are read once and tested against up
    // to 8 views per round; the block appends all its kept (view, Gaussian) pairs
    // with one scan and one atomic per round
    __shared__ int s_wcnt[kPreThreads / 32];
    __shared__ uint32_t s_base;
    __shared__ float s_pose[8 * 24];  // the round's poses (double-float pairs)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gi = (int64_t)blockIdx.x * kPreThreads + tid;
    int64_t nl = g.N;
    if (g.n_dev) nl = min(nl, (int64_t)*g.n_dev);
    bool ok = false;  // live, finite and opaque enough
    float mx = 0, my = 0, mz = 0, smax = 0, kq = 0;
    if (gi < g.N && gi < nl) {
        mx = g.means[3 * gi]; my = g.means[3 * gi + 1]; mz = g.means[3 * gi + 2];
        const float sx = g.scales[3 * gi], sy = g.scales[3 * gi + 1], sz = g.scales[3 * gi + 2];
        const float4 q = reinterpret_cast<const float4 *>(g.quats)[gi];
        const float op = g.opac[gi];
        const float cr = g.colors[3 * gi], cg = g.colors[3 * gi + 1], cb = g.colors[3 * gi + 2];
        const float chk = mx + my + mz + sx + sy + sz + q.x + q.y + q.z + q.w + op + cr + cg + cb;
        if (!isfinite(chk)) {
            set_status(ws.status, VPGS_ERR_NONFINITE);
        } else if (op >= o.alpha_min) {
            ok = true;
            smax = fmaxf(fabsf(sx), fmaxf(fabsf(sy), fabsf(sz)));
            // fast log, widened by 1e-3 relative for the bound
            kq = 2.002f * __logf(op / o.alpha_min) + 1e-3f;
        }
    }
    for (int v0 = 0; v0 < V; v0 += 8) {  // block-uniform
        const int nv = min(8, V - v0);
        for (int i = tid; i < nv * 24; i += kPreThreads) s_pose[i] = ws.posedf[24 * v0 + i];
        __syncthreads();
        uint32_t keep = 0u;  // bit dv: view v0 + dv kept
        if (gi < g.N) {
            for (int dv = 0; dv < nv; ++dv) {
                bool k = false;
                if (ok) {
                    const float *pd = s_pose + 24 * dv;
                    PoseDF P;
#pragma unroll
                    for (int j = 0; j < 9; ++j) P.R[j] = df{pd[2 * j], pd[2 * j + 1]};
#pragma unroll
                    for (int r = 0; r < 3; ++r) P.t[r] = df{pd[18 + 2 * r], pd[19 + 2 * r]};
                    k = maybe_in_view(P, mx, my, mz, smax, kq, cam, o);
                }
                if (k) keep |= 1u << dv;
                else ws.tcount[(int64_t)(v0 + dv) * g.N + gi] = 0u;
            }
        }
        // block exclusive scan of the kept counts
        const int c = __popc(keep);
        int x = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_wcnt[warp] = x;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) t += s_wcnt[w];
            s_base = t ? atomicAdd(n_cand, (uint32_t)t) : 0u;
        }
        __syncthreads();
        if (keep) {
            int pos = x - c;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) pos += w < warp ? s_wcnt[w] : 0;
            for (int dv = 0; dv < nv; ++dv)
                if (keep & (1u << dv)) cand[s_base + pos++] = (uint32_t)((int64_t)(v0 + dv) * g.N + gi);
        }
        __syncthreads();  // s_wcnt and s_base are reused by the next round
    }
}

// Exact projection of one pre-cull survivor ic = (view, Gaussian) from its
// parameters, and everything the binning needs of it: tile count, screen and
// binning records, the digits of its depth key (block histograms s_h), and
// zeroed 2D-gradient slots when asked.
VPGS_D void project_write(int64_t ic, int v, float mx, float my, float mz, float sx, float sy, float sz, float4 q,
                          float op, float cr, float cg, float cb, const CamParams &cam, const OptParams &o,
                          const RenderWs &ws, bool zero_g2d, uint32_t (*s_h)[kRadix]) {
    const SortPass dps[4] = {{0, 8}, {8, 8}, {16, 8}, {24, 8}};  // the depth sort's passes over 32 bits
    BinRec B;
    float depth = 0.f;
    const uint32_t cnt = project_one(ws.posedf + 24 * v, mx, my, mz, sx, sy, sz, q, op, cr, cg, cb, cam, o,
                                     ws.status, ws.rec + ic, B, depth);
    ws.tcount[ic] = cnt;
    if (cnt) {
        ws.bin[ic] = B;
        add_digits(s_h, dps, 4, __float_as_uint(depth));  // the depth key (camera z > 0)
        if (zero_g2d) {
            float2 *z2 = reinterpret_cast<float2 *>(ws.g2d + 10 * ic);
#pragma unroll
            for (int j = 0; j < 5; ++j) z2[j] = make_float2(0.f, 0.f);
        }
    }
}

// Pre-cull and exact projection in one pass, for calls of several views.  Each
// block walks chunks of kPreThreads consecutive Gaussians, one per thread: it
// reads their parameters once (coalesced) and pre-culls its Gaussian against
// each view of a round of up to 8; one block scan numbers the round's
// survivors (thread order, then view), and they are staged with their
// parameters in shared memory kPreThreads at a time, every thread projecting
// one.  The exact projection thus runs on full warps without gathering the
// survivors' parameters from memory again, with a few barriers per round
// (the projection of a pair depends on nothing but the pair, so its order is
// free).  Measured:
// 8 keyframes x 2M Gaussians 803 us against 172 + 753 us for the two-kernel
// form; one 1200x680 view of 1M Gaussians 53.8 us against 20.8 + 30.3 us,
// where the two kernels' overlap under programmatic dependent launch wins.
// VPGS_CULL_PROJECT: the fewest views a call needs to take this kernel.
#ifndef VPGS_CULL_PROJECT
#define VPGS_CULL_PROJECT 2
#endif

struct QItem {
    float4 a;  // mx, my, mz, sx
    float4 b;  // sy, sz, opacity, r
    float4 q;  // quaternion (w, x, y, z)
    float4 c;  // g, b, (view, Gaussian) index bits, view bits
};

__global__ void __launch_bounds__(kPreThreads, 3)
cull_project_kernel(GaussIn g, int V, CamParams cam, OptParams o, RenderWs ws, bool zero_g2d) {
    grid_dep_enter();
    __shared__ uint32_t s_h[4][kRadix];
    __shared__ QItem s_q[kPreThreads];
    __shared__ float s_pose[8 * 24];  // the round's poses (double-float pairs)
    __shared__ int s_wcnt[kPreThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 4 * kRadix; i += kPreThreads) (&s_h[0][0])[i] = 0u;
    __syncthreads();
    int64_t nl = g.N;
    if (g.n_dev) nl = min(nl, (int64_t)*g.n_dev);
    const int64_t n_chunks = (g.N + kPreThreads - 1) / kPreThreads;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {  // block-uniform
        const int64_t gi = ch * kPreThreads + tid;
        bool ok = false;  // live, finite and opaque enough
        float mx = 0, my = 0, mz = 0, sx = 0, sy = 0, sz = 0, op = 0, cr = 0, cg = 0, cb = 0, smax = 0, kq = 0;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gi < g.N && gi < nl) {
            mx = g.means[3 * gi]; my = g.means[3 * gi + 1]; mz = g.means[3 * gi + 2];
            sx = g.scales[3 * gi]; sy = g.scales[3 * gi + 1]; sz = g.scales[3 * gi + 2];
            q = reinterpret_cast<const float4 *>(g.quats)[gi];
            op = g.opac[gi];
            cr = g.colors[3 * gi]; cg = g.colors[3 * gi + 1]; cb = g.colors[3 * gi + 2];
            const float chk = mx + my + mz + sx + sy + sz + q.x + q.y + q.z + q.w + op + cr + cg + cb;
            if (!isfinite(chk)) {
                set_status(ws.status, VPGS_ERR_NONFINITE);
            } else if (op >= o.alpha_min) {
                ok = true;
                smax = fmaxf(fabsf(sx), fmaxf(fabsf(sy), fabsf(sz)));
                // fast log, widened by 1e-3 relative for the bound
                kq = 2.002f * __logf(op / o.alpha_min) + 1e-3f;
            }
        }
        for (int v0 = 0; v0 < V; v0 += 8) {  // block-uniform
            const int nv = min(8, V - v0);
            for (int i = tid; i < nv * 24; i += kPreThreads) s_pose[i] = ws.posedf[24 * v0 + i];
            __syncthreads();
            // this thread's Gaussian against the round's views
            uint32_t keep = 0u;
            for (int dv = 0; dv < nv; ++dv) {
                bool k = false;
                if (ok) {
                    const float *pd = s_pose + 24 * dv;
                    PoseDF P;
#pragma unroll
                    for (int j = 0; j < 9; ++j) P.R[j] = df{pd[2 * j], pd[2 * j + 1]};
#pragma unroll
                    for (int r = 0; r < 3; ++r) P.t[r] = df{pd[18 + 2 * r], pd[19 + 2 * r]};
                    k = maybe_in_view(P, mx, my, mz, smax, kq, cam, o);
                }
                if (k) keep |= 1u << dv;
                else if (gi < g.N) ws.tcount[(int64_t)(v0 + dv) * g.N + gi] = 0u;
            }
            // the block's survivors numbered by one scan (thread order, then view)
            const int c = __popc(keep);
            int x = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) s_wcnt[warp] = x;
            __syncthreads();
            int first = x - c, total = 0;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) {
                first += w < warp ? s_wcnt[w] : 0;
                total += s_wcnt[w];
            }
            // projected kPreThreads at a time on full warps: each owner stages its
            // survivors that fall in the batch, then thread t projects item t
            for (int b0 = 0; b0 < total; b0 += kPreThreads) {  // block-uniform
                int p = first;
                for (int dv = 0; dv < nv; ++dv) {
                    if (!(keep >> dv & 1u)) continue;
                    if (p >= b0 && p < b0 + kPreThreads) {
                        QItem it;
                        it.a = make_float4(mx, my, mz, sx);
                        it.b = make_float4(sy, sz, op, cr);
                        it.q = q;
                        it.c = make_float4(cg, cb, __uint_as_float((uint32_t)gi), __uint_as_float((uint32_t)(v0 + dv)));
                        s_q[p - b0] = it;
                    }
                    ++p;
                }
                __syncthreads();
                if (tid < min(kPreThreads, total - b0)) {
                    const QItem it = s_q[tid];
                    const uint32_t v = __float_as_uint(it.c.w);
                    const int64_t ic = (int64_t)v * g.N + __float_as_uint(it.c.z);
                    project_write(ic, (int)v, it.a.x, it.a.y, it.a.z, it.a.w, it.b.x, it.b.y, it.q, it.b.z, it.b.w,
                                  it.c.x, it.c.y, cam, o, ws, zero_g2d, s_h);
                }
                __syncthreads();  // the staging slots are rewritten by the next batch
            }
        }
    }
    __syncthreads();
    flush_digits(s_h, 4, ws.sort_hist[0]);
}

// Pass 2, grid-strided over the candidates: the exact projection on full warps.
// It also accumulates the digit histograms of the visible Gaussians' depth keys
// for the depth sort.
__global__ void __launch_bounds__(kPreThreads, 3)
project_kernel(GaussIn g, CamParams cam, OptParams o, RenderWs ws, const uint32_t *__restrict__ cand,
               const uint32_t *n_cand, bool zero_g2d) {
    grid_dep_enter();
    __shared__ uint32_t s_h[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0u;
    __syncthreads();
    const SortPass dps[4] = {{0, 8}, {8, 8}, {16, 8}, {24, 8}};  // the depth sort's passes over 32 bits
    const int64_t nc = *n_cand;
    for (int64_t k = (int64_t)blockIdx.x * kPreThreads + threadIdx.x; k < nc;
         k += (int64_t)gridDim.x * kPreThreads) {
        const int64_t ic = cand[k];
        const int v = (int)(ic / g.N);
        const int64_t gi = ic - (int64_t)v * g.N;
        const float4 q = reinterpret_cast<const float4 *>(g.quats)[gi];
        BinRec B;
        float depth = 0.f;
        const uint32_t cnt = project_one(ws.posedf + 24 * v, g.means[3 * gi], g.means[3 * gi + 1], g.means[3 * gi + 2],
                                         g.scales[3 * gi], g.scales[3 * gi + 1], g.scales[3 * gi + 2], q,
                                         g.opac[gi], g.colors[3 * gi], g.colors[3 * gi + 1], g.colors[3 * gi + 2],
                                         cam, o, ws.status, ws.rec + ic, B, depth);
        ws.tcount[ic] = cnt;
        if (cnt) {
            ws.bin[ic] = B;
            add_digits(s_h, dps, 4, __float_as_uint(depth));  // the depth key (camera z > 0)
            if (zero_g2d) {
                float2 *z2 = reinterpret_cast<float2 *>(ws.g2d + 10 * ic);
#pragma unroll
                for (int j = 0; j < 5; ++j) z2[j] = make_float2(0.f, 0.f);
            }
        }
    }
    __syncthreads();
    flush_digits(s_h, 4, ws.sort_hist[0]);
}

VPGS_D float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// blocks per SM the register budget must allow (3: 24 warps to hide gather latency)
#ifndef VPGS_PRE_BWD_MINB
#define VPGS_PRE_BWD_MINB 3
#endif
__global__ void __launch_bounds__(256, VPGS_PRE_BWD_MINB)
preprocess_bwd_kernel(GaussIn g, const double *__restrict__ T_cw, int V, CamParams cam, OptParams o,
                      RenderWs ws, GaussGrad gg, double *dpose, const uint32_t *__restrict__ vis,
                      const uint32_t *n_vis) {
    grid_dep_enter();
    if (*ws.status != 0u) return;  // the binning failed: vis may hold stale entries
    __shared__ double s_pose[8][6];
    __shared__ int s_views[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one thread per visible (view, Gaussian) pair of the compacted list (ascending
    // pair index, so views come in order and a block spans one or two of them);
    // block-uniform grid-stride loop
    const int64_t nv = min((int64_t)*n_vis, (int64_t)V * g.N);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nv; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kk = base + threadIdx.x;
        const bool live = kk < nv;
        const int64_t i = live ? (int64_t)vis[kk] : 0;
        const int v = (int)(i / g.N);
        const int64_t gi = i - (int64_t)v * g.N;
        float gm[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0.f, gc[3] = {0, 0, 0};
        float pv[6] = {0, 0, 0, 0, 0, 0};
        if (live) {
            const float mx = g.means[3 * gi], my = g.means[3 * gi + 1], mz = g.means[3 * gi + 2];
            const float sx = g.scales[3 * gi], sy = g.scales[3 * gi + 1], sz = g.scales[3 * gi + 2];
            const float4 q = reinterpret_cast<const float4 *>(g.quats)[gi];
            const float *g2 = ws.g2d + 10 * i;  // [u, v, a, b, c, o, r, g, b, z]
            const float2 a01 = reinterpret_cast<const float2 *>(g2)[0];
            const float2 a23 = reinterpret_cast<const float2 *>(g2)[1];
            const float2 a45 = reinterpret_cast<const float2 *>(g2)[2];
            const float2 a67 = reinterpret_cast<const float2 *>(g2)[3];
            const float2 a89 = reinterpret_cast<const float2 *>(g2)[4];
            // consumed: the slots start at zero again for the next backward
            float2 *z2 = reinterpret_cast<float2 *>(ws.g2d + 10 * i);
#pragma unroll
            for (int k = 0; k < 5; ++k) z2[k] = make_float2(0.f, 0.f);
            // the compositing backward leaves out these per-Gaussian factors (see
            // pair_grad): the mean's slots hold sum dpow t1 and sum dpow t2, turned
            // into d/du, d/dv by the whitening rows W of the record the pixels saw,
            // and the covariance's slots S = sum dpow t t^T, whence
            // dL/dSigma' = 2 ln^2 2 W^T S W (FP64 for a near-degenerate record)
            const Rec &rc = ws.rec[i];
            const float4 w = rc.r1;  // (w1x, w1y, w2x, w2y)
            const float gu = (w.x * a01.x + w.z * a01.y) * kInvExp2Half;
            const float gv = (w.y * a01.x + w.w * a01.y) * kInvExp2Half;
            float S00, S01, S11;
            {
                constexpr float kc = 0.5f * kInvExp2Half * kInvExp2Half;  // 2 ln^2 2
                const float s11 = a23.x, s12 = a23.y, s22 = a45.x;
                const float4 r3 = rc.r3;
                if (r3.z < 0.f) {
                    const double w1x = w.x, w1y = w.y, w2x = (double)w.z + r3.y, w2y = (double)w.w + r3.w;
                    const double m00 = s11 * w1x * w1x + 2.0 * s12 * w1x * w2x + s22 * w2x * w2x;
                    const double m01 = s11 * w1x * w1y + s12 * (w1x * w2y + w2x * w1y) + s22 * w2x * w2y;
                    const double m11 = s11 * w1y * w1y + 2.0 * s12 * w1y * w2y + s22 * w2y * w2y;
                    S00 = (float)(kc * m00);
                    S01 = (float)(kc * m01);
                    S11 = (float)(kc * m11);
                } else {
                    S00 = kc * (s11 * w.x * w.x + 2.f * s12 * w.x * w.z + s22 * w.z * w.z);
                    S01 = kc * (s11 * w.x * w.y + s12 * (w.x * w.w + w.z * w.y) + s22 * w.z * w.w);
                    S11 = kc * (s11 * w.y * w.y + 2.f * s12 * w.y * w.w + s22 * w.w * w.w);
                }
            }
            go += a45.y;
            gc[0] += a67.x; gc[1] += a67.y; gc[2] += a89.x;
            const float gz = a89.y;
            PoseDF P;
            load_pose(ws.posedf + 24 * v, P);
            Proj p;
            project(P, mx, my, mz, sx, sy, sz, q.x, q.y, q.z, q.w, cam, o.dilation, p);
            // Sigma' = K K^T + eps I  ->  G_K = 2 G_S K
            float GK0[3], GK1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                GK0[c] = 2.f * (S00 * p.K0[c] + S01 * p.K1[c]);
                GK1[c] = 2.f * (S01 * p.K0[c] + S11 * p.K1[c]);
            }
            // K0 = (j00 WR0 + j02 WR2) o s,  K1 = (j11 WR1 + j12 WR2) o s
            const float sv[3] = {sx, sy, sz};
            float Gj00 = 0, Gj02 = 0, Gj11 = 0, Gj12 = 0;
            float GWR[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float a0 = GK0[c] * sv[c], a1 = GK1[c] * sv[c];
                Gj00 += a0 * p.WR[c];
                Gj02 += a0 * p.WR[6 + c];
                Gj11 += a1 * p.WR[3 + c];
                Gj12 += a1 * p.WR[6 + c];
                GWR[c] = p.j00 * a0;
                GWR[3 + c] = p.j11 * a1;
                GWR[6 + c] = p.j02 * a0 + p.j12 * a1;
                gs[c] += (GK0[c] * (p.j00 * p.WR[c] + p.j02 * p.WR[6 + c]) +
                          GK1[c] * (p.j11 * p.WR[3 + c] + p.j12 * p.WR[6 + c]));
            }
            // camera-space point: projection Jacobian, image mean and depth
            const float iz2 = p.iz * p.iz;
            float gpx = Gj02 * (-cam.fx * iz2) + gu * cam.fx * p.iz;
            float gpy = Gj12 * (-cam.fy * iz2) + gv * cam.fy * p.iz;
            float gpz = Gj00 * (-cam.fx * iz2) + Gj02 * (2.f * cam.fx * p.xz * iz2) +
                        Gj11 * (-cam.fy * iz2) + Gj12 * (2.f * cam.fy * p.yz * iz2) -
                        gu * cam.fx * p.xz * p.iz - gv * cam.fy * p.yz * p.iz + gz;
            // WR = Wf Rq: G_Rq = Wf^T G_WR; pose rotation term A = G_WR WR^T
            float GRq[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    GRq[3 * r + c] = p.Wf[r] * GWR[c] + p.Wf[3 + r] * GWR[3 + c] + p.Wf[6 + r] * GWR[6 + c];
            float A[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    A[3 * r + c] = GWR[3 * r] * p.WR[3 * c] + GWR[3 * r + 1] * p.WR[3 * c + 1] +
                                   GWR[3 * r + 2] * p.WR[3 * c + 2];
            // rotation matrix -> normalised quaternion -> raw quaternion
            {
                const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
                const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
                const float *G = GRq;
                float dw = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
                float dx = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] +
                                  w * G[7] - 2.f * x * G[8]);
                float dy = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] +
                                  z * G[7] - 2.f * y * G[8]);
                float dz = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] +
                                  y * G[5] + x * G[6] + y * G[7]);
                const float dot = w * dw + x * dx + y * dy + z * dz;
                gq[0] += (dw - w * dot) * inv;
                gq[1] += (dx - x * dot) * inv;
                gq[2] += (dy - y * dot) * inv;
                gq[3] += (dz - z * dot) * inv;
            }
            // p_c = Wf mu + t
            gm[0] += p.Wf[0] * gpx + p.Wf[3] * gpy + p.Wf[6] * gpz;
            gm[1] += p.Wf[1] * gpx + p.Wf[4] * gpy + p.Wf[7] * gpz;
            gm[2] += p.Wf[2] * gpx + p.Wf[5] * gpy + p.Wf[8] * gpz;
            // left-perturbation pose terms
            pv[0] = gpx; pv[1] = gpy; pv[2] = gpz;
            pv[3] = p.py * gpz - p.pz * gpy + (A[7] - A[5]);
            pv[4] = p.pz * gpx - p.px * gpz + (A[2] - A[6]);
            pv[5] = p.px * gpy - p.py * gpx + (A[3] - A[1]);
        }
        if (dpose) {
            // FP32 within a warp (32 terms), FP64 across warps and blocks, per view
            if (threadIdx.x == 0) {
                s_views[0] = (int)((int64_t)vis[base] / g.N);
                s_views[1] = (int)((int64_t)vis[min(base + (int64_t)blockDim.x, nv) - 1] / g.N);
            }
            __syncthreads();
            const int v_lo = s_views[0], v_hi = s_views[1];
            for (int vv = v_lo; vv <= v_hi; ++vv) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float sm = warp_sum(live && v == vv ? pv[k] : 0.f);
                    if (lane == 0) s_pose[warp][k] = (double)sm;
                }
                __syncthreads();
                if (threadIdx.x < 6) {
                    double t = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_pose[w][threadIdx.x];
                    if (t != 0.0) atomicAdd(dpose + 6 * vv + threadIdx.x, t);
                }
                __syncthreads();
            }
        }
        if (!live) continue;
        // += as fire-and-forget reductions: no load round trip (a Gaussian seen by
        // several views gets one reduction per view)
        auto add = [](float *p, float x) {
            if (x != 0.f) atomicAdd(p, x);
        };
        if (gg.means) {
            add(gg.means + 3 * gi, gm[0]); add(gg.means + 3 * gi + 1, gm[1]); add(gg.means + 3 * gi + 2, gm[2]);
        }
        if (gg.scales) {
            add(gg.scales + 3 * gi, gs[0]); add(gg.scales + 3 * gi + 1, gs[1]); add(gg.scales + 3 * gi + 2, gs[2]);
        }
        if (gg.quats) {
#pragma unroll
            for (int k = 0; k < 4; ++k) add(gg.quats + 4 * gi + k, gq[k]);
        }
        if (gg.opac) add(gg.opac + gi, go);
        if (gg.colors) {
            add(gg.colors + 3 * gi, gc[0]); add(gg.colors + 3 * gi + 1, gc[1]); add(gg.colors + 3 * gi + 2, gc[2]);
        }
    }
}

__global__ void export_projection_kernel(RenderWs ws, int64_t VN, int32_t *tile_count,
                                         int32_t *tile_rect, float *mean2d, float *depth,
                                         float *conic) {
    grid_dep_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= VN) return;
    const uint32_t cnt = ws.tcount[i];
    if (tile_count) tile_count[i] = (int32_t)cnt;
    if (!cnt) return;
    const uint2 rc = ws.bin[i].rect;
    if (tile_rect) {
        tile_rect[4 * i] = (int32_t)(rc.x & 0xffffu);
        tile_rect[4 * i + 1] = (int32_t)(rc.x >> 16);
        tile_rect[4 * i + 2] = (int32_t)(rc.y & 0xffffu);
        tile_rect[4 * i + 3] = (int32_t)(rc.y >> 16);
    }
    const Rec r = ws.rec[i];
    if (mean2d) {
        mean2d[2 * i] = r.r0.x + r.r0.z;
        mean2d[2 * i + 1] = r.r0.y + r.r0.w;
    }
    if (depth) depth[i] = r.r2.y;
    if (conic) {  // Sigma'^-1 = (w1 w1^T + w2 w2^T) 2 / log2(e)
        conic[3 * i] = (r.r1.x * r.r1.x + r.r1.z * r.r1.z) * kInvExp2Half;
        conic[3 * i + 1] = (r.r1.x * r.r1.y + r.r1.z * r.r1.w) * kInvExp2Half;
        conic[3 * i + 2] = (r.r1.y * r.r1.y + r.r1.w * r.r1.w) * kInvExp2Half;
    }
}

cudaError_t launch_export_projection(const RenderWs &ws, int64_t VN, int32_t *tile_count,
                                     int32_t *tile_rect, float *mean2d, float *depth, float *conic,
                                     cudaStream_t s) {
    if (VN == 0) return cudaSuccess;
    VPGS_LAUNCH("export_projection", s,
                launch_k(export_projection_kernel, (unsigned)((VN + 255) / 256), 256, 0, s,
                    ws, VN, tile_count, tile_rect, mean2d, depth, conic));
    return cudaGetLastError();
}

cudaError_t launch_preprocess_fwd(const GaussIn &g, const double *T_cw, int V, const CamParams &cam,
                                  const OptParams &o, const RenderWs &ws, const RenderLayout &L,
                                  bool zero_g2d, cudaStream_t s) {
    const int64_t VN = (int64_t)V * g.N;
    PrepZero z;
    z.w32[0] = ws.status;                      z.n32[0] = 1;
    z.w32[1] = ws.counters;                    z.n32[1] = CNT_N;
    z.w32[2] = ws.sort_hist[0];                z.n32[2] = 2 * 4 * kRadix;  // both sorts
    z.w32[3] = ws.sort_look[0];                z.n32[3] = sort_blocks(std::max<int64_t>(L.VN, 1), kDepthSortItems) * kRadix;
    z.w32[4] = ws.sort_look[1];                z.n32[4] = 0;  // zeroed by emit, sized by the instance count
    z.w32[5] = reinterpret_cast<uint32_t *>(ws.ranges);  z.n32[5] = 2 * (int64_t)V * cam.T;
    z.w64 = ws.scan_look[0];                   z.n64 = 2 * L.scan_blocks_max;  // both scans
    const int prep_grid = 8 * device_sm_count();
    const int64_t words = std::max<int64_t>(z.n32[3] + z.n32[4] + z.n32[5], z.n64);
    VPGS_LAUNCH("prepare", s,
                launch_k(prepare_kernel, (unsigned)std::max<int64_t>(1, std::min<int64_t>(prep_grid, (words + 255) / 256)),
                                 256, 0, s, T_cw, V, ws.posedf, z));
    if (VN == 0) return cudaGetLastError();
    if (VPGS_CULL_PROJECT > 0 && V >= VPGS_CULL_PROJECT) {
        static std::atomic<int> cp_cache[kDeviceCache];
        const int cp_grid = per_device(cp_cache, [] {
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)cull_project_kernel, kPreThreads, 0);
            return std::max(occ, 1) * device_sm_count();
        });
        VPGS_LAUNCH("cull_project", s,
                    launch_k(cull_project_kernel,
                             (unsigned)std::min<int64_t>(cp_grid, (g.N + kPreThreads - 1) / kPreThreads),
                             kPreThreads, 0, s, g, V, cam, o, ws, zero_g2d));
        return cudaGetLastError();
    }
    // the candidate list borrows the second depth-key buffer (free until the depth sort)
    uint32_t *cand = ws.dkey[1], *n_cand = ws.counters + CNT_CAND;
    VPGS_LAUNCH("preprocess_fwd", s,
                launch_k(precull_kernel, (unsigned)((g.N + kPreThreads - 1) / kPreThreads), kPreThreads, 0, s,
                    g, V, cam, o, ws, cand, n_cand));
    static std::atomic<int> proj_cache[kDeviceCache];
    const int proj_grid = per_device(proj_cache, [] {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)project_kernel, kPreThreads, 0);
        return std::max(occ, 1) * device_sm_count();
    });
    VPGS_LAUNCH("project", s,
                launch_k(project_kernel, (unsigned)std::min<int64_t>(proj_grid, (VN + kPreThreads - 1) / kPreThreads),
                                 kPreThreads, 0, s, g, cam, o, ws, cand, n_cand, zero_g2d));
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const GaussIn &g, const double *T_cw, int V, const CamParams &cam,
                                  const OptParams &o, const RenderWs &ws, const GaussGrad &gg,
                                  double *dpose, cudaStream_t s) {
    if (g.N == 0) return cudaSuccess;
    // enough blocks for the visible pairs of a large frame at full occupancy; the
    // live count is read on the device
    const int bwd_grid = 8 * device_sm_count() * VPGS_PRE_BWD_MINB;
    const int64_t VN = (int64_t)V * g.N;
    VPGS_LAUNCH("preprocess_bwd", s,
                launch_k(preprocess_bwd_kernel, (unsigned)std::min<int64_t>((VN + 255) / 256, bwd_grid), 256, 0, s,
                    g, T_cw, V, cam, o, ws, gg, dpose, (const uint32_t *)ws.vis_idx, ws.counters + CNT_VISIBLE));
    return cudaGetLastError();
}

}  // namespace vpgs
