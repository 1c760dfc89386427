// Host-side declarations shared by the translation units of libvpgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "common.cuh"

namespace vpgs {

struct CamParams {
    int W, H;
    float fx, fy, cx, cy;
    int tile_w, tile_h, tiles_x, tiles_y, T;  // T = tiles per view
    int tw_shift;                             // log2(tile_w)
};

struct OptParams {
    float alpha_min, alpha_max, t_min, dilation, near_z;
    float bg0, bg1, bg2;
    int spin_limit;  // polls of a look-back wait before VPGS_ERR_TIMEOUT
};

struct GaussIn {
    const float *means, *scales, *quats, *opac, *colors;
    int64_t N;
    const int32_t *n_dev;
};

struct GaussGrad {
    float *means, *scales, *quats, *opac, *colors;
};

int device_sm_count();



// render_pre.cu
// First launches of a render call: the prepare kernel (zeroes status, counters
// and the scratch later kernels expect at zero; converts the poses), the
// pre-cull and the exact projection.
cudaError_t launch_preprocess_fwd(const GaussIn &g, const double *T_cw, int V, const CamParams &cam,
                                  const OptParams &o, const RenderWs &ws, const RenderLayout &L,
                                  bool zero_g2d, cudaStream_t s);
cudaError_t launch_export_projection(const RenderWs &ws, int64_t VN, int32_t *tile_count,
                                     int32_t *tile_rect, float *mean2d, float *depth, float *conic,
                                     cudaStream_t s);
cudaError_t launch_preprocess_bwd(const GaussIn &g, const double *T_cw, int V, const CamParams &cam,
                                  const OptParams &o, const RenderWs &ws, const GaussGrad &gg,
                                  double *dpose, cudaStream_t s);

// render_bin.cu: visibility compaction, depth sort, instance emission, tile
// sort and tile ranges.  On return ws.ival[*sorted_buf] holds the tile lists.
cudaError_t build_tile_lists(const GaussIn &g, int V, const CamParams &cam, const OptParams &o, const RenderWs &ws,
                             const RenderLayout &L, int *sorted_buf, cudaStream_t s, bool order_by_count = true);
// Compositing launch order from the forward's n_iter: tiles by the backward's
// list steps, most first (ws.tile_work, ws.tile_order).
cudaError_t order_tiles_by_steps(const RenderWs &ws, const int32_t *n_iter, int V, const CamParams &cam,
                                 cudaStream_t s);
// Which ival buffer build_tile_lists leaves the tile lists in (host only, no launch).
int tile_list_buffer(const RenderLayout &L);

// render_comp.cu
cudaError_t launch_composite_fwd(const RenderWs &ws, const uint32_t *ival, int V,
                                 const CamParams &cam, const OptParams &o, const vpgs_images &out,
                                 int persistent_ctas, cudaStream_t s);
cudaError_t launch_composite_bwd(const RenderWs &ws, const uint32_t *ival, int V,
                                 const CamParams &cam, const OptParams &o, const vpgs_images &fwd,
                                 const float *dL_drgb, const float *dL_ddepth,
                                 const float *dL_dalpha, bool geometric_only, int persistent_ctas,
                                 cudaStream_t s);

// pose.cu
cudaError_t launch_pose_step(double *T_cw, double *dpose, double *adam, int V, double lr_rho,
                             double lr_phi, cudaStream_t s);

}  // namespace vpgs
