// Submap fusion by distillation (Sec. III-C, Eq. 14) and the Adam step of the
// fusion loop.
//
//   L = 1/m sum_keyframes ( mean_{c,p} (c_a - c_b)^2 + mean_p (d_a - d_b)^2 )
//   dL/dc_a = 2 (c_a - c_b) / (m 3 P) = -dL/dc_b,  dL/dd_a = 2 (d_a - d_b) / (m P)
// (c: colour renders of one keyframe from submaps a and b, d: depth renders,
// P pixels per image, m keyframes).  One grid-strided kernel writes the
// gradients and per-block partial sums (FP32 inside a block), a one-block
// kernel adds the partials in FP64 into the loss.
//
// Adam (Kingma and Ba, bias-corrected): m <- b1 m + (1 - b1) g,
// v <- b2 v + (1 - b2) g^2, p <- p - lr m^ / (sqrt(v^) + eps); the gradient is
// zeroed after use so the next backward can accumulate into it.
#include <cmath>

#include "internal.h"
#include "profiler.h"

namespace vpgs {

constexpr int kFuseThreads = 256;
constexpr int kFuseMaxBlocks = 4096;  // partial sums held in the workspace

__global__ void __launch_bounds__(kFuseThreads)
distill_kernel(const float *__restrict__ ca, const float *__restrict__ cb, const float *__restrict__ da,
               const float *__restrict__ db, int64_t n_col, int64_t n_dep, float gc, float gd, float *gca,
               float *gcb, float *gda, float *gdb, float2 *partial) {
    grid_dep_enter();
    __shared__ float s_red[2][kFuseThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * kFuseThreads;
    float sc = 0.f, sd = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * kFuseThreads + threadIdx.x; i < n_col; i += stride) {
        const float e = ca[i] - cb[i];
        sc = fmaf(e, e, sc);
        if (gca) gca[i] = gc * e;
        if (gcb) gcb[i] = -gc * e;
    }
    if (da)
        for (int64_t i = (int64_t)blockIdx.x * kFuseThreads + threadIdx.x; i < n_dep; i += stride) {
            const float e = da[i] - db[i];
            sd = fmaf(e, e, sd);
            if (gda) gda[i] = gd * e;
            if (gdb) gdb[i] = -gd * e;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][warp] = sc;
        s_red[1][warp] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tc = 0.f, td = 0.f;
        for (int w = 0; w < kFuseThreads / 32; ++w) {
            tc += s_red[0][w];
            td += s_red[1][w];
        }
        partial[blockIdx.x] = make_float2(tc, td);
    }
}

__global__ void __launch_bounds__(kFuseThreads)
distill_finalize_kernel(const float2 *__restrict__ partial, int nb, double inv_c, double inv_d, double *loss) {
    grid_dep_enter();
    __shared__ double s_red[2][kFuseThreads / 32];
    double sc = 0.0, sd = 0.0;
    for (int i = threadIdx.x; i < nb; i += kFuseThreads) {
        sc += partial[i].x;
        sd += partial[i].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][warp] = sc;
        s_red[1][warp] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tc = 0.0, td = 0.0;
        for (int w = 0; w < kFuseThreads / 32; ++w) {
            tc += s_red[0][w];
            td += s_red[1][w];
        }
        loss[1] = tc * inv_c;
        loss[2] = td * inv_d;
        loss[0] = loss[1] + loss[2];
    }
}

__global__ void __launch_bounds__(kFuseThreads)
adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m, float *__restrict__ v, int64_t n,
            float lr, float b1, float b2, float eps, float c1, float c2) {
    grid_dep_enter();
    const int64_t stride = (int64_t)gridDim.x * kFuseThreads;
    for (int64_t i = (int64_t)blockIdx.x * kFuseThreads + threadIdx.x; i < n; i += stride) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        g[i] = 0.f;
    }
}

static int fuse_grid(int64_t n) {
    const int64_t g = std::min<int64_t>((n + kFuseThreads - 1) / kFuseThreads, (int64_t)device_sm_count() * 8);
    return (int)std::max<int64_t>(g, 1);
}

}  // namespace vpgs

using namespace vpgs;

extern "C" {

size_t vpgs_distill_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
    if (n_views <= 0 || width <= 0 || height <= 0 || width > 65535 || height > 65535 || n_views > 4096) return 0;
    return sizeof(float2) * (size_t)kFuseMaxBlocks;
}

vpgs_status vpgs_distill_loss(void *ws, size_t ws_bytes, const float *rgb_a, const float *rgb_b,
                              const float *depth_a, const float *depth_b, int32_t n_views, int32_t width,
                              int32_t height, double *loss_out, float *dL_drgb_a, float *dL_drgb_b,
                              float *dL_ddepth_a, float *dL_ddepth_b, vpgs_stream stream) {
    if (!ws || !rgb_a || !rgb_b || !loss_out) return VPGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 15u) return VPGS_ERR_INVALID_ARG;
    if ((depth_a == nullptr) != (depth_b == nullptr)) return VPGS_ERR_INVALID_ARG;
    const size_t need = vpgs_distill_workspace_bytes(n_views, width, height);
    if (need == 0 || ws_bytes < need) return VPGS_ERR_INVALID_ARG;
    const int64_t P = (int64_t)width * height, n_col = 3 * P * n_views, n_dep = depth_a ? P * n_views : 0;
    const int nb = std::min(fuse_grid(n_col), kFuseMaxBlocks);
    const float gc = (float)(2.0 / (double)n_col), gd = (float)(2.0 / (double)(P * n_views));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float2 *partial = static_cast<float2 *>(ws);
    VPGS_LAUNCH("distill", s,
                launch_k(distill_kernel, nb, kFuseThreads, 0, s, rgb_a, rgb_b, depth_a, depth_b, n_col, n_dep, gc, gd,
                                                           dL_drgb_a, dL_drgb_b, dL_ddepth_a, dL_ddepth_b, partial));
    if (cudaGetLastError() != cudaSuccess) return VPGS_ERR_CUDA;
    VPGS_LAUNCH("distill_finalize", s,
                launch_k(distill_finalize_kernel, 1, kFuseThreads, 0, s, partial, nb, 1.0 / (double)n_col,
                                                                   depth_a ? 1.0 / (double)(P * n_views) : 0.0,
                                                                   loss_out));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

vpgs_status vpgs_adam_step(float *params, float *grads, float *m, float *v, int64_t n, const float hyper[4],
                           int32_t step, vpgs_stream stream) {
    if (n < 0 || !hyper || step < 1) return VPGS_ERR_INVALID_ARG;
    if (n == 0) return VPGS_OK;
    if (!params || !grads || !m || !v) return VPGS_ERR_INVALID_ARG;
    const float lr = hyper[0], b1 = hyper[1], b2 = hyper[2], eps = hyper[3];
    if (!(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return VPGS_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, step)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VPGS_LAUNCH("adam", s, launch_k(adam_kernel, fuse_grid(n), kFuseThreads, 0, s, params, grads, m, v, n, lr, b1, b2,
                                                                           eps, c1, c2));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

}  // extern "C"
