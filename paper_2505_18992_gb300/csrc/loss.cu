// Mapping loss of the submap optimisation (Sec. III-A, Eq. 7-9) and its
// gradient, for rendered RGB / depth and the Gaussians' scales:
//   L_m    = L_c + L_SSIM + lambda_d L_d + lambda_vol L_vol
//   L_SSIM = (1 - lambda_SSIM) |I^ - I|_1 + lambda_SSIM (1 - SSIM(I^, I))
//   L_vol  = sum_i s_x s_y s_z
// L_c, |.|_1: mean absolute colour difference; L_d: absolute depth difference
// where the target depth is > 0, divided by the pixel count; SSIM: 11x11
// Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2, mean
// over views, channels and pixels.
//
// SSIM at pixel p is S(m1, m2, m3) of the windowed moments of x = I^ (given
// y = I): m1 = w*x, m2 = w*x^2, m3 = w*xy.  Hence
//   d mean(S) / dx(q) = (1/n) [ (w*A)(q) + 2 x(q) (w*B)(q) + y(q) (w*C)(q) ],
//   A = dS/dm1, B = dS/dm2, C = dS/dm3 at each p,
// so the gradient is a second blur, of A, B, C.  Two kernels, one kLT x kLT
// output tile per block and channel (256 threads), separable 11-tap blurs from a shared-memory tile
// with a 5-pixel halo, each thread producing kU neighbouring outputs per pass
// from one (kU + 10)-value window (the blurs are bound by shared-memory loads):
//   1. moments -> S, A, B, C (A, B, C to the workspace), block sums of S and
//      |x - y|; the same blocks also take the depth term and the volume term
//      (grid-strided) and write their gradients;
//   2. blur of A, B, C -> colour gradient; block 0 sums the block partials
//      into the loss terms.
// The coarse-tracking loss (the colour and depth L1 terms per view) is a third,
// single-pass kernel further down.
#include <cmath>

#include "internal.h"
#include "profiler.h"

namespace vpgs {

#ifndef VPGS_SSIM_TILE
#define VPGS_SSIM_TILE 32
#endif
constexpr int kLT = VPGS_SSIM_TILE;  // output tile edge
constexpr int kLThreads = 256;      // threads per block
constexpr int kLR = 5;              // window radius
constexpr int kLH = kLT + 2 * kLR;  // tile edge with halo (26)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
#ifndef VPGS_SSIM_U
#define VPGS_SSIM_U 2
#endif
constexpr int kU = VPGS_SSIM_U;          // neighbouring outputs per thread and blur pass
constexpr int kWin = kU + 10;            // their window

struct LossArgs {
    const float *rgb, *target, *depth, *tdepth, *scales;
    const int32_t *n_dev;
    int64_t N;
    int V, W, H, tiles_x, tiles_y;
    float lambda_ssim, lambda_d, lambda_vol;
    float g[11];                    // normalised 1D Gaussian taps
    float *A, *B, *C;               // [V,3,H,W] SSIM partials
    double *partial;                // [blocks][4]: sum S, sum |x - y|, sum depth term, sum volume
    double *loss;                   // [5]: L_m, L_c, L_SSIM, L_d, L_vol
    float *d_rgb, *d_depth, *d_scales;
};

// Separable 11-tap blurs, register-blocked: each thread produces kU
// neighbouring outputs from one (kU + 10)-value window, so a tap costs one
// shared load per kU outputs instead of one per output.
//   horizontal: s_src[NM][kLH][kLH + 1] -> s_h[NM][kLH][kLT + 1] (42 x 32)
//   vertical:   s_h -> kU vertically adjacent outputs (r0 .. r0 + kU - 1, c)
//               for the kLT * kLT / kU work items, looped over the block's threads
template <int NM>
VPGS_D void hblur(const float (*s_src)[kLH][kLH + 1], float (*s_h)[kLH][kLT + 1], const float *g, int tid) {
    for (int w = tid; w < kLH * (kLT / kU); w += kLThreads) {
        const int r = w / (kLT / kU), c0 = kU * (w % (kLT / kU));
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            float v[kWin];
#pragma unroll
            for (int j = 0; j < kWin; ++j) v[j] = s_src[m][r][c0 + j];
            float o[kU] = {};
#pragma unroll
            for (int k = 0; k < 11; ++k)
#pragma unroll
                for (int u = 0; u < kU; ++u) o[u] = fmaf(g[k], v[k + u], o[u]);
#pragma unroll
            for (int u = 0; u < kU; ++u) s_h[m][r][c0 + u] = o[u];
        }
    }
}

template <int NM>
VPGS_D void vblur(const float (*s_h)[kLH][kLT + 1], const float *g, int r0, int c, float (&o)[kU][NM]) {
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        float v[kWin];
#pragma unroll
        for (int j = 0; j < kWin; ++j) v[j] = s_h[m][r0 + j][c];
        float acc[kU] = {};
#pragma unroll
        for (int k = 0; k < 11; ++k)
#pragma unroll
            for (int u = 0; u < kU; ++u) acc[u] = fmaf(g[k], v[k + u], acc[u]);
#pragma unroll
        for (int u = 0; u < kU; ++u) o[u][m] = acc[u];
    }
}

// Block sum (FP32 within the block: FP64 arithmetic is slow on this part and a
// block adds at most a few thousand terms; the block partials are summed in FP64).
VPGS_D float block_sum(float v, float *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;  // valid in thread 0
}

VPGS_D double block_sum_f64(double v, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kLThreads)
ssim_moments_kernel(LossArgs a) {
    grid_dep_enter();
    __shared__ float s_in[2][kLH][kLH + 1];   // x, y with the halo
    __shared__ float s_h[5][kLH][kLT + 1];    // horizontal blurs of x, y, x^2, y^2, xy
    __shared__ float s_red[8];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;            // view * 3 + channel
    const int x0 = blockIdx.x * kLT - kLR, y0 = blockIdx.y * kLT - kLR;
    const int64_t HW = (int64_t)a.H * a.W;
    const float *X = a.rgb + plane * HW, *Y = a.target + plane * HW;
    for (int i = tid; i < kLH * kLH; i += kLThreads) {
        const int r = i / kLH, c = i % kLH, gy = y0 + r, gx = x0 + c;
        float xv = 0.f, yv = 0.f;
        if (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) {
            xv = X[(int64_t)gy * a.W + gx];
            yv = Y[(int64_t)gy * a.W + gx];
        }
        s_in[0][r][c] = xv;
        s_in[1][r][c] = yv;
    }
    __syncthreads();
    // horizontal: the five moment maps from one window of x and y
    for (int w = tid; w < kLH * (kLT / kU); w += kLThreads) {
        const int r = w / (kLT / kU), c0 = kU * (w % (kLT / kU));
        float xs[kWin], ys[kWin];
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            xs[j] = s_in[0][r][c0 + j];
            ys[j] = s_in[1][r][c0 + j];
        }
        float o[5][kU] = {};
#pragma unroll
        for (int k = 0; k < 11; ++k) {
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const float xv = xs[k + u], yv = ys[k + u], gk = a.g[k];
                o[0][u] = fmaf(gk, xv, o[0][u]);
                o[1][u] = fmaf(gk, yv, o[1][u]);
                o[2][u] = fmaf(gk, xv * xv, o[2][u]);
                o[3][u] = fmaf(gk, yv * yv, o[3][u]);
                o[4][u] = fmaf(gk, xv * yv, o[4][u]);
            }
        }
#pragma unroll
        for (int m = 0; m < 5; ++m)
#pragma unroll
            for (int u = 0; u < kU; ++u) s_h[m][r][c0 + u] = o[m][u];
    }
    __syncthreads();
    float ssum = 0.f, l1 = 0.f;
    for (int it = tid; it < kLT * kLT / kU; it += kLThreads) {
        const int tx = it % kLT, r0 = kU * (it / kLT);
        float mm[kU][5];
        vblur<5>(s_h, a.g, r0, tx, mm);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const float *m = mm[u];
            const int ty = r0 + u, px = blockIdx.x * kLT + tx, py = blockIdx.y * kLT + ty;
            if (px < a.W && py < a.H) {
                const float mx = m[0], my = m[1];
                const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
                const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
                const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
                const float id = 1.f / (d1 * d2);
                const float S = n1 * n2 * id;
                const int64_t o = plane * HW + (int64_t)py * a.W + px;
                a.A[o] = (2.f * my * (n2 - n1) - 2.f * mx * S * (d2 - d1)) * id;
                a.B[o] = -S / d2;
                a.C[o] = 2.f * n1 * id;
                ssum += S;
                l1 += fabsf(s_in[0][ty + kLR][tx + kLR] - s_in[1][ty + kLR][tx + kLR]);
            }
        }
    }
    // depth and volume terms, grid-strided over all blocks of this launch
    const int64_t nblk = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int64_t stride = nblk * kLThreads, t0 = bid * kLThreads + tid;
    float dsum = 0.f, vsum = 0.f;
    if (a.depth) {
        const int64_t P = (int64_t)a.V * HW;
        const float scale = a.lambda_d / (float)P;
        for (int64_t i = t0; i < P; i += stride) {
            const float td = a.tdepth[i], e = a.depth[i] - td;
            const bool valid = td > 0.f;
            if (valid) dsum += fabsf(e);
            if (a.d_depth) a.d_depth[i] = valid ? scale * (float)((e > 0.f) - (e < 0.f)) : 0.f;
        }
    } else if (a.d_depth) {
        for (int64_t i = t0; i < (int64_t)a.V * HW; i += stride) a.d_depth[i] = 0.f;
    }
    if (a.scales) {
        int64_t n = a.N;
        if (a.n_dev) n = min(n, (int64_t)*a.n_dev);
        for (int64_t i = t0; i < n; i += stride) {
            const float sx = a.scales[3 * i], sy = a.scales[3 * i + 1], sz = a.scales[3 * i + 2];
            vsum += sx * sy * sz;
            if (a.d_scales) {
                a.d_scales[3 * i] += a.lambda_vol * sy * sz;
                a.d_scales[3 * i + 1] += a.lambda_vol * sx * sz;
                a.d_scales[3 * i + 2] += a.lambda_vol * sx * sy;
            }
        }
    }
    const float t_s = block_sum(ssum, s_red), t_l = block_sum(l1, s_red);
    const float t_d = block_sum(dsum, s_red), t_v = block_sum(vsum, s_red);
    if (tid == 0) {
        double *pp = a.partial + 4 * bid;
        pp[0] = t_s; pp[1] = t_l; pp[2] = t_d; pp[3] = t_v;
    }
}

__global__ void __launch_bounds__(kLThreads)
ssim_grad_kernel(LossArgs a, int64_t n_partial) {
    grid_dep_enter();
    __shared__ float s_in[3][kLH][kLH + 1];
    __shared__ float s_h[3][kLH][kLT + 1];
    __shared__ double s_red[8];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;
    const int64_t HW = (int64_t)a.H * a.W;
    const double n_col = (double)a.V * 3 * HW;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        // loss terms from the first kernel's block sums
        double s[4] = {0, 0, 0, 0};
        for (int64_t i = tid; i < n_partial; i += kLThreads)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += a.partial[4 * i + k];
        double t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = block_sum_f64(s[k], s_red);
        if (tid == 0) {
            const double L_c = t[1] / n_col, ssim = t[0] / n_col;
            const double L_ssim = (1.0 - a.lambda_ssim) * L_c + a.lambda_ssim * (1.0 - ssim);
            const double L_d = t[2] / ((double)a.V * HW), L_vol = t[3];
            a.loss[0] = L_c + L_ssim + a.lambda_d * L_d + a.lambda_vol * L_vol;
            a.loss[1] = L_c; a.loss[2] = L_ssim; a.loss[3] = L_d; a.loss[4] = L_vol;
        }
    }
    if (!a.d_rgb) return;
    const int x0 = blockIdx.x * kLT - kLR, y0 = blockIdx.y * kLT - kLR;
    for (int i = tid; i < kLH * kLH; i += kLThreads) {
        const int r = i / kLH, c = i % kLH, gy = y0 + r, gx = x0 + c;
        float va = 0.f, vb = 0.f, vc = 0.f;
        if (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) {
            const int64_t o = plane * HW + (int64_t)gy * a.W + gx;
            va = a.A[o]; vb = a.B[o]; vc = a.C[o];
        }
        s_in[0][r][c] = va; s_in[1][r][c] = vb; s_in[2][r][c] = vc;
    }
    __syncthreads();
    hblur<3>(s_in, s_h, a.g, tid);
    __syncthreads();
    const float inv_n = (float)(1.0 / n_col);
    for (int it = tid; it < kLT * kLT / kU; it += kLThreads) {
    const int tx = it % kLT, r0 = kU * (it / kLT);
    float mm[kU][3];
    vblur<3>(s_h, a.g, r0, tx, mm);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const float *m = mm[u];
        const int px = blockIdx.x * kLT + tx, py = blockIdx.y * kLT + r0 + u;
        if (px < a.W && py < a.H) {
            const int64_t o = plane * HW + (int64_t)py * a.W + px;
            const float x = a.rgb[o], y = a.target[o];
            const float dssim = m[0] + 2.f * x * m[1] + y * m[2];
            const float e = x - y;
            // L_c + (1 - lambda) L1 share the sign term; the SSIM term enters as -lambda mean(S)
            a.d_rgb[o] = ((2.f - a.lambda_ssim) * (float)((e > 0.f) - (e < 0.f)) - a.lambda_ssim * dssim) * inv_n;
        }
    }
    }
}

size_t loss_workspace_bytes(int V, int W, int H) {
    const int64_t planes = (int64_t)V * 3;
    const int64_t blocks = planes * ((W + kLT - 1) / kLT) * ((H + kLT - 1) / kLT);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    return up(3 * sizeof(float) * (size_t)planes * W * H) + up(4 * sizeof(double) * (size_t)blocks);
}

cudaError_t launch_mapping_loss(void *ws, const float *rgb, const float *target, const float *depth,
                                const float *tdepth, int V, int W, int H, const float *scales, int64_t N,
                                const int32_t *n_dev, float lambda_ssim, float lambda_d, float lambda_vol,
                                double *loss, float *d_rgb, float *d_depth, float *d_scales, cudaStream_t s) {
    LossArgs a;
    a.rgb = rgb; a.target = target; a.depth = depth; a.tdepth = tdepth; a.scales = scales;
    a.n_dev = n_dev; a.N = N; a.V = V; a.W = W; a.H = H;
    a.tiles_x = (W + kLT - 1) / kLT; a.tiles_y = (H + kLT - 1) / kLT;
    a.lambda_ssim = lambda_ssim; a.lambda_d = lambda_d; a.lambda_vol = lambda_vol;
    double gs[11], tot = 0.0;
    for (int k = 0; k < 11; ++k) {
        const double x = k - 5;
        gs[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        tot += gs[k];
    }
    for (int k = 0; k < 11; ++k) a.g[k] = (float)(gs[k] / tot);
    const int64_t planes = (int64_t)V * 3, HW = (int64_t)W * H;
    char *b = static_cast<char *>(ws);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    a.A = reinterpret_cast<float *>(b);
    a.B = a.A + planes * HW;
    a.C = a.B + planes * HW;
    a.partial = reinterpret_cast<double *>(b + up(3 * sizeof(float) * (size_t)planes * HW));
    a.loss = loss; a.d_rgb = d_rgb; a.d_depth = d_depth; a.d_scales = d_scales;
    const dim3 grid((unsigned)a.tiles_x, (unsigned)a.tiles_y, (unsigned)planes);
    VPGS_LAUNCH("ssim_moments", s, launch_k(ssim_moments_kernel, grid, kLThreads, 0, s, a));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    VPGS_LAUNCH("ssim_grad", s, launch_k(ssim_grad_kernel, grid, kLThreads, 0, s, a, (int64_t)grid.x * grid.y * grid.z));
    return cudaGetLastError();
}

// Coarse-tracking loss of each view (Sec. III-B), the per-view colour and depth
// L1 terms of the mapping loss:
//   L_t(v) = w_c sum_{c,p} |x - y| + w_d sum_{p: D(p) > 0} |D^ - D|,
//   w_c = 1 / 3HW, w_d = lambda_d / HW,
// with its gradient sign(e) w (0 at e = 0, and at pixels without a target
// depth) written for every pixel.  One thread per kTlItems pixels of a view
// (blockIdx.y); block sums in FP32, added across blocks in FP64.
constexpr int kTlThreads = 256, kTlItems = 4;

VPGS_D float sgn(float e) { return (float)((e > 0.f) - (e < 0.f)); }

__global__ void __launch_bounds__(kTlThreads)
tracking_loss_kernel(const float *__restrict__ rgb, const float *__restrict__ target,
                     const float *__restrict__ depth, const float *__restrict__ tdepth, int64_t HW, float w_c,
                     float w_d, float *__restrict__ d_rgb, float *__restrict__ d_depth, double *loss) {
    grid_dep_enter();
    __shared__ float s_red[kTlThreads / 32];
    const int v = blockIdx.y;
    const int64_t p0 = (int64_t)blockIdx.x * kTlThreads * kTlItems + threadIdx.x;
    const int64_t cbase = (int64_t)v * 3 * HW, dbase = (int64_t)v * HW;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kTlItems; ++k) {
        const int64_t p = p0 + (int64_t)k * kTlThreads;
        if (p < HW) {
            float l = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t o = cbase + c * HW + p;
                const float e = rgb[o] - target[o];
                if (d_rgb) d_rgb[o] = w_c * sgn(e);
                l += fabsf(e);
            }
            acc = fmaf(w_c, l, acc);
            if (depth) {
                const float t = tdepth[dbase + p];
                const float e = depth[dbase + p] - t;
                const bool ok = t > 0.f;
                if (d_depth) d_depth[dbase + p] = ok ? w_d * sgn(e) : 0.f;
                if (ok) acc = fmaf(w_d, fabsf(e), acc);
            }
        }
    }
    if (loss) {
        const float t = block_sum(acc, s_red);
        if (threadIdx.x == 0) atomicAdd(loss + v, (double)t);
    }
}

cudaError_t launch_tracking_loss(const float *rgb, const float *target, const float *depth, const float *tdepth,
                                 int V, int W, int H, float lambda_d, double *loss, float *d_rgb,
                                 float *d_depth, cudaStream_t s) {
    const int64_t HW = (int64_t)W * H;
    if (loss) {
        const cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double) * (size_t)V, s);
        if (e != cudaSuccess) return e;
    }
    const float w_c = (float)(1.0 / (3.0 * (double)HW));
    const float w_d = (float)((double)lambda_d / (double)HW);
    const dim3 grid((unsigned)((HW + kTlThreads * kTlItems - 1) / (kTlThreads * kTlItems)), (unsigned)V);
    VPGS_LAUNCH("tracking_loss", s,
                launch_k(tracking_loss_kernel, grid, kTlThreads, 0, s, rgb, target, depth, tdepth, HW, w_c, w_d,
                         d_rgb, d_depth, loss));
    return cudaGetLastError();
}

}  // namespace vpgs

using namespace vpgs;

extern "C" {

void vpgs_loss_weights_default(vpgs_loss_weights *w) {
    if (!w) return;
    w->lambda_ssim = 0.2f;
    w->lambda_d = 1.0f;
    w->lambda_vol = 0.001f;
}

size_t vpgs_mapping_loss_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
    if (n_views <= 0 || width <= 0 || height <= 0 || width > 65535 || height > 65535 || n_views > 4096) return 0;
    return loss_workspace_bytes(n_views, width, height);
}

vpgs_status vpgs_mapping_loss(void *ws, size_t ws_bytes, const float *rgb, const float *target_rgb,
                              const float *depth, const float *target_depth, int32_t n_views, int32_t width,
                              int32_t height, const float *scales, int64_t n_gaussians, const int32_t *n_dev,
                              const vpgs_loss_weights *w, double *loss_out, float *dL_drgb, float *dL_ddepth,
                              float *dL_dscales, vpgs_stream stream) {
    if (!ws || !rgb || !target_rgb || !w || !loss_out) return VPGS_ERR_INVALID_ARG;
    if (vpgs_mapping_loss_workspace_bytes(n_views, width, height) == 0) return VPGS_ERR_INVALID_ARG;
    if (ws_bytes < loss_workspace_bytes(n_views, width, height)) return VPGS_ERR_INVALID_ARG;
    if ((depth == nullptr) != (target_depth == nullptr)) return VPGS_ERR_INVALID_ARG;
    if (n_gaussians < 0 || (n_gaussians > 0 && !scales)) return VPGS_ERR_INVALID_ARG;
    if (!(w->lambda_ssim >= 0.f && w->lambda_ssim <= 1.f) || !(w->lambda_d >= 0.f) || !(w->lambda_vol >= 0.f))
        return VPGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 15u) return VPGS_ERR_INVALID_ARG;
    const cudaError_t e = launch_mapping_loss(ws, rgb, target_rgb, depth, target_depth, n_views, width, height,
                                              n_gaussians > 0 ? scales : nullptr, n_gaussians, n_dev,
                                              w->lambda_ssim, w->lambda_d, w->lambda_vol, loss_out, dL_drgb,
                                              dL_ddepth, dL_dscales, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

vpgs_status vpgs_tracking_loss(const float *rgb, const float *target_rgb, const float *depth,
                               const float *target_depth, int32_t n_views, int32_t width, int32_t height,
                               float lambda_d, double *loss_out, float *dL_drgb, float *dL_ddepth,
                               vpgs_stream stream) {
    if (!rgb || !target_rgb) return VPGS_ERR_INVALID_ARG;
    if (n_views <= 0 || width <= 0 || height <= 0 || width > 65535 || height > 65535 || n_views > 4096)
        return VPGS_ERR_INVALID_ARG;
    if ((depth == nullptr) != (target_depth == nullptr)) return VPGS_ERR_INVALID_ARG;
    if (!(lambda_d >= 0.f) || !std::isfinite(lambda_d)) return VPGS_ERR_INVALID_ARG;
    const cudaError_t e = launch_tracking_loss(rgb, target_rgb, depth, target_depth, n_views, width, height,
                                               lambda_d, loss_out, dL_drgb, dL_ddepth,
                                               reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

}  // extern "C"
