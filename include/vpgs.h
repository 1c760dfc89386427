/*
 * vpgs.h - C ABI of the GB300 (sm_103a) rasterizer and anchor decoder of
 * VPGS-SLAM (voxel-based progressive Gaussian SLAM).
 *
 * The library renders 3D Gaussians into RGB, depth and accumulated alpha, and
 * differentiates the render with respect to every Gaussian parameter and the
 * 6-DoF camera pose.  The mapping loss (Sec. III-A, Eq. 7) and the coarse
 * tracking stage (Sec. III-B) both use this render.  The library also decodes
 * voxel anchors into neural Gaussians (Sec. III-A, Eq. 1-5) and
 * differentiates that decode.
 *
 * Conventions for every entry point
 *   - Pointers are DEVICE pointers unless a comment says "host".  Arrays are
 *     dense, C-contiguous, little-endian and 16-byte aligned.  The caller
 *     owns them all.
 *   - The library allocates no memory.  Entry points that need scratch space
 *     carve it from a caller-provided device workspace.  Size the workspace
 *     with the matching *_workspace_bytes function.  The workspace must not
 *     be shared by calls that may run concurrently.
 *   - Every call is asynchronous on `stream` (NULL = the legacy default
 *     stream).  No call synchronises with the host, so the calls can be
 *     captured into a CUDA graph.
 *   - Argument errors that the host can see (NULL pointers, negative sizes,
 *     a workspace that is too small, unsupported options) return
 *     VPGS_ERR_INVALID_ARG or VPGS_ERR_UNSUPPORTED and launch nothing.
 *     Conditions found on the device (instance capacity exceeded, a
 *     look-back wait that ran out) set a status word in the workspace.  The
 *     outputs are then undefined.  Read the status with vpgs_workspace_status
 *     after the stream has been synchronised.
 *   - Kernel launch failures return VPGS_ERR_CUDA.
 *
 * Camera model (the paper gives only "known intrinsics K" and poses
 * {R|t}, Sec. III).  T_cw is the world-to-camera rigid transform, stored as
 * row-major double[4][4].  A camera-space point is p = R mu + t; the camera
 * looks down +z, with +x right and +y down.  Pixel (i, j) has its centre at
 * (i + 0.5, j + 0.5).
 */
#ifndef VPGS_H
#define VPGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *vpgs_stream; /* a cudaStream_t */

typedef enum {
    VPGS_OK = 0,
    VPGS_ERR_INVALID_ARG = 1,
    VPGS_ERR_CAPACITY = 2,    /* device: more tile instances than the workspace holds */
    VPGS_ERR_NONFINITE = 3,   /* device: a NaN/Inf input was seen */
    VPGS_ERR_TIMEOUT = 4,     /* device: a bounded look-back wait ran out */
    VPGS_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    VPGS_ERR_UNSUPPORTED = 6,
    VPGS_ERR_INTERNAL = 7     /* device: an internal consistency check failed (a bug) */
} vpgs_status;

/* Pinhole intrinsics and image size, shared by every view of a call (host struct). */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
} vpgs_camera;

/* Rasterizer options (host struct).  vpgs_render_opts_default() fills these defaults:
 *   tile 16x16, alpha_min 1/255, alpha_max 0.99, t_min 1e-4, dilation 0.3 px^2,
 *   near_z 0.2, background black.
 * The paper cites 3D Gaussian Splatting for all of these (Sec. I, Sec. II) and
 * states none of them. */
typedef struct {
    int32_t tile_w, tile_h;   /* tile_w in {4,8,16,32}; tile_h even; tile_w*tile_h a multiple of 64, <= 512 */
    float alpha_min;          /* skip a Gaussian at a pixel when alpha < alpha_min */
    float alpha_max;          /* alpha = min(alpha_max, o exp(-d^T Sigma'^-1 d / 2)) */
    float t_min;              /* stop before the first Gaussian that would take T below t_min */
    float dilation;           /* added to the diagonal of the 2D covariance (px^2) */
    float near_z;             /* Gaussians with camera z <= near_z are dropped */
    float bg[3];              /* C = sum_i alpha_i T_i c_i + T_final bg */
    int32_t persistent_ctas;  /* 0 = one CTA per tile; >0 = that many persistent CTAs per SM */
    int32_t flags;            /* VPGS_RENDER_* bits below; 0 by default */
    int32_t spin_limit;       /* polls a bounded look-back wait of the binning (scans, sorts) makes
                               * before it gives up and records VPGS_ERR_TIMEOUT; 0 = the default,
                               * 2^22, never reached in a healthy run.  A few polls make the timeout
                               * path testable: the render's outputs are then undefined, nothing is
                               * written out of range, and the next call starts clean. */
} vpgs_render_opts;

/* vpgs_render_bwd: take the projection and tile lists from the workspace
 * instead of recomputing them.  Valid when the last render call on this
 * workspace was vpgs_render_fwd with the same inputs (same workspace, arrays,
 * camera, poses and options other than flags and persistent_ctas), with their
 * contents unchanged since; backward calls in between are allowed.  The
 * library records the arguments of each forward call per workspace and
 * recomputes everything when they do not match; it cannot see a change made in
 * place to the contents of the arrays, so the caller must not make one. */
#define VPGS_RENDER_REUSE_BINNING 1

/* Gaussians, structure of arrays, float32 (device).
 *   means [n,3], scales [n,3] (linear, > 0), quats [n,4] (w,x,y,z; normalised
 *   inside), opacities [n] (in (0,1)), colors [n,3] (RGB).
 * n is the capacity.  If n_dev is not NULL, the live count is the device scalar
 * *n_dev (<= n), for example the output count of vpgs_decode_anchors.  Entries
 * at and past *n_dev are ignored. */
typedef struct {
    const float *means, *scales, *quats, *opacities, *colors;
    int64_t n;
    const int32_t *n_dev;
} vpgs_gaussians;

/* Writable per-Gaussian arrays with the same layout as vpgs_gaussians.  Used
 * for gradients (accumulated with +=; a NULL field is not computed) and for
 * decoder outputs (written). */
typedef struct {
    float *means, *scales, *quats, *opacities, *colors;
} vpgs_gaussian_buffers;

/* Render outputs for V views (device, written by vpgs_render_fwd).
 *   rgb [V,3,H,W], depth [V,H,W] (sum alpha_i T_i z_i, not normalised),
 *   alpha [V,H,W] (1 - T_final), t_final [V,H,W],
 *   n_contrib [V,H,W] (Gaussians blended into the pixel), n_iter [V,H,W] (how
 *   many entries of the pixel's tile list the pixel walked; vpgs_render_bwd
 *   reads it).  t_final and n_iter are required; the others may be NULL. */
typedef struct {
    float *rgb, *depth, *alpha, *t_final;
    int32_t *n_contrib, *n_iter;
} vpgs_images;

/* Counters that a render leaves in its workspace (host struct, filled by
 * vpgs_workspace_status). */
typedef struct {
    int32_t status;           /* a vpgs_status value */
    int64_t n_visible;        /* (view, Gaussian) pairs touching at least one tile */
    int64_t n_instances;      /* (view, tile, Gaussian) instances that were sorted */
} vpgs_render_stats;

void vpgs_render_opts_default(vpgs_render_opts *opts);            /* opts: host */

/* Workspace size in bytes for renders of up to max_gaussians Gaussians into
 * n_views views of the given camera, with room for max_instances tile
 * instances.  Returns 0 if the arguments are invalid. */
size_t vpgs_render_workspace_bytes(int64_t max_gaussians, int32_t n_views, const vpgs_camera *cam,
                                   const vpgs_render_opts *opts, int64_t max_instances);

/* Differentiable tile rasterization, forward pass (3D Gaussian Splatting as the
 * paper uses it: Sec. I, Sec. II; RGB and depth renders in Sec. III-B and
 * Eq. 14, accumulated alpha in Sec. III-A "Voxel-Based Submap Expansion").
 *
 * For each view v: project every Gaussian (EWA splatting), bin it into the
 * tiles its alpha >= alpha_min ellipse can reach, sort each tile's list by
 * camera depth (ties by Gaussian index), and blend front to back.
 *   T_cw  [n_views,4,4] float64, device.
 *   ws    workspace of ws_bytes bytes, from vpgs_render_workspace_bytes.
 * Results are independent of the tile shape. */
vpgs_status vpgs_render_fwd(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                            const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                            const vpgs_render_opts *opts, const vpgs_images *out, vpgs_stream stream);

/* Backward pass of vpgs_render_fwd.  It recomputes the projection, binning and
 * per-tile sort from the inputs, or, with VPGS_RENDER_REUSE_BINNING in
 * opts->flags, takes them from the forward call's workspace.  It reads
 * fwd->t_final and fwd->n_iter from the forward call with identical inputs and
 * options, then back-propagates
 *   dL_drgb [V,3,H,W], dL_ddepth [V,H,W], dL_dalpha [V,H,W] (each may be NULL = 0)
 * to the Gaussian parameters (grads: += into each non-NULL field; grads may be
 * NULL) and to the camera poses.
 *   dL_dpose [n_views,6] float64, device, += ; may be NULL.  Each pose gets a
 *   left perturbation T_cw <- Exp(xi) T_cw at xi = 0, with
 *   xi = (rho_x, rho_y, rho_z, phi_x, phi_y, phi_z).  The pose is optimised in
 *   the coarse tracking stage (Sec. III-B).  Per-Gaussian pose terms are summed
 *   in float64.
 * Decisions (skips, clamp, stop) are held fixed, as in the forward pass.
 * When neither grads->opacities nor grads->colors is asked for (grads NULL, or
 * both fields NULL, as in pose tracking), the compositing pass sums only the
 * geometric 2D terms; the requested results are the same. */
vpgs_status vpgs_render_bwd(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                            const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                            const vpgs_render_opts *opts, const vpgs_images *fwd,
                            const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                            const vpgs_gaussian_buffers *grads, double *dL_dpose,
                            vpgs_stream stream);

/* Projection stage of vpgs_render_fwd alone: per (view, Gaussian) EWA
 * projection and tile extent, written out for inspection (device outputs,
 * each may be NULL):
 *   tile_count [V,N] int32 (tiles the Gaussian is binned into; 0 = culled):
 *     the tiles whose pixel-centre rectangle, widened by 1e-5 r + 2e-3 px,
 *     meets the ellipse d^T Sigma'^-1 d <= 2 ln(o / alpha_min),
 *   tile_rect [V,N,4] int32 (tx0, tx1, ty0, ty1, inclusive: the bounding box
 *     of that ellipse, widened the same way, in tiles), mean2d [V,N,2]
 *   float32 (u, v), depth [V,N] float32 (camera z), conic [V,N,3] float32
 *   (a, b, c of Sigma'^-1 = [[a,b],[b,c]]).
 * Entries of culled Gaussians other than tile_count are left unchanged. */
vpgs_status vpgs_render_project(void *ws, size_t ws_bytes, const vpgs_gaussians *g,
                                const vpgs_camera *cam, const double *T_cw, int32_t n_views,
                                const vpgs_render_opts *opts, int32_t *tile_count,
                                int32_t *tile_rect, float *mean2d, float *depth, float *conic,
                                vpgs_stream stream);

/* Size of the scratch array behind vpgs_render_fwd_noalloc: 32 MiB.  Every
 * GPU that loads this library holds it until the process exits. */
#define VPGS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* vpgs_render_fwd for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is an interface for hosts whose device memory is
 * not theirs to allocate.  Examples are a plugin handed only a stream and the
 * tensors it must read and write, and a process whose memory pool reserved the
 * GPU up front and forbids further allocations.
 *
 * Same inputs and outputs as vpgs_render_fwd, without the workspace.  The
 * scratch space is a VPGS_NOALLOC_SCRATCH_BYTES array compiled into the library.
 * This call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *   - Returns VPGS_ERR_UNSUPPORTED, launching nothing, when the render needs
 *     more scratch than that (about 10^5 Gaussians per view at most; the tile
 *     instances take the rest).
 *   - status_out (device int32, may be NULL) receives the device status word
 *     of the render.  VPGS_ERR_CAPACITY there means that the tile instances
 *     did not fit in the array.
 *   - The first call on each device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current, and keeps it for the
 *     later calls on that device.  The address belongs to the device's
 *     primary context (the one the CUDA runtime uses): after cudaDeviceReset,
 *     or with another driver context current on the device, it no longer
 *     names the array, so do not call this entry point in either situation.
 *   - Device ordinals from 64 up return VPGS_ERR_UNSUPPORTED.
 *   - Every call shares the one array, and a call leaves its contents behind.
 *     The render clears what it needs zeroed.  Calls that overlap on the GPU
 *     (other streams, other threads) race on the array, so serialise them. */
vpgs_status vpgs_render_fwd_noalloc(const vpgs_gaussians *g, const vpgs_camera *cam,
                                    const double *T_cw, int32_t n_views,
                                    const vpgs_render_opts *opts, const vpgs_images *out,
                                    int32_t *status_out, vpgs_stream stream);

/* Reads the status word and counters of a render workspace (host `stats`).  It
 * synchronises `stream` first, and is the one call here that blocks. */
vpgs_status vpgs_workspace_status(const void *ws, vpgs_render_stats *stats, vpgs_stream stream);

/* Queues a copy of a render workspace's status word (int32, a vpgs_status
 * value) into `dst` on `stream`, after the work queued before it, and returns
 * without waiting.  `dst` is caller-owned device memory or page-locked host
 * memory (4 bytes); it holds the status once the stream reaches the copy.  The
 * way to check renders without stalling the host: copy, record an event, read
 * `dst` once the event has completed.  No counterpart in the paper (error
 * reporting).  Errors: VPGS_ERR_INVALID_ARG for a NULL pointer, VPGS_ERR_CUDA if
 * the copy cannot be queued. */
vpgs_status vpgs_workspace_status_copy(const void *ws, int32_t *dst, vpgs_stream stream);

/* One step of the camera pose on the device (coarse tracking, Sec. III-B;
 * the step rule is not given in the paper).  For each view v:
 *   xi = -lr * m_hat / (sqrt(v_hat) + 1e-15)  (Adam, beta 0.9/0.999; adam_state
 *        [n_views,13] float64 = m[6], v[6], step; zero it before the first step)
 *   or xi = -lr * g  when adam_state is NULL;
 *   T_cw[v] <- Exp(xi) T_cw[v]  (SE(3) exponential, float64)
 * lr[0] applies to rho and lr[1] to phi (host values).  dL_dpose is read,
 * then zeroed, so repeated steps can be replayed from a CUDA graph. */
vpgs_status vpgs_pose_step(double *T_cw, double *dL_dpose, double *adam_state, int32_t n_views,
                           const double lr[2], vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Anchor decoder (Sec. III-A, Eq. 1-5)                                    */
/* ---------------------------------------------------------------------- */

/* Voxel anchors (device).
 *   anchors [n,3] float32 (voxel centres x^a), scaling [n,3] float32 (l),
 *   offsets [n,k,3] float32 (O), features [n,32] float32, or bfloat16 when
 *   features_bf16 != 0 (f^a). */
typedef struct {
    const float *anchors, *scaling, *offsets;
    const void *features;
    int64_t n;
    int32_t k;
    int32_t features_bf16;
} vpgs_anchors;

/* Decoder MLPs (device), float32, flat.  For each MLP in the order opacity,
 * colour, covariance, the layout is W1 [32,36], b1 [32], W2 [out,32],
 * b2 [out], with out = k, 3k, 7k.  That is 3*(36*32+32) + 11k*32 + 11k
 * floats (7,182 at k = 10).  bf16 != 0 selects the tensor-core decode: the
 * network input, W1, W2 and the hidden activations are rounded to bfloat16,
 * and the sums are accumulated in float32.  The FP32 form is used otherwise. */
typedef struct {
    const float *params;
    int32_t bf16;
} vpgs_mlp;

/* Decoder options (host struct). */
typedef struct {
    float near_z;   /* anchors with camera z <= near_z are culled */
    float guard;    /* keep anchors whose projected centre lies in the image widened by guard*W, guard*H */
} vpgs_decode_opts;

size_t vpgs_decode_workspace_bytes(int64_t n_anchors, int32_t k);

/* Decode the anchors seen by one camera into neural Gaussians.
 *   Cull each anchor by its camera depth and projected centre.
 *   Eq. 3: view distance delta and direction d from the camera centre
 *     -R^T t.
 *   Eq. 2: [f^a, d, delta] goes through three LINEAR-ReLU-LINEAR MLPs.
 *   Heads: tanh opacity (valid iff > 0), sigmoid colour (Eq. 4), normalised
 *     quaternion, sigmoid(F_s) * l scale (Eq. 5).
 *   Eq. 1: mu^m = x^a + O^m * l.
 * The valid Gaussians are compacted in (anchor, m) order into `out`, which
 * has capacity n*k.
 *   T_cw [4,4] float64 device; n_out device int32 scalar (written);
 *   src_index [n*k] int32 device (written; entry i = anchor*k + m of output i). */
vpgs_status vpgs_decode_anchors(void *ws, size_t ws_bytes, const vpgs_anchors *a,
                                const vpgs_mlp *mlp, const vpgs_camera *cam, const double *T_cw,
                                const vpgs_decode_opts *opts, const vpgs_gaussian_buffers *out,
                                int32_t *n_out, int32_t *src_index, vpgs_stream stream);

/* Backward pass of vpgs_decode_anchors.  Inputs and options must be those of
 * the forward call.  dL_dgauss holds the gradients with respect to the decoded
 * Gaussians: n is the capacity and n_dev = n_out.  Outputs are float32 and
 * accumulated (+=):
 *   dL_dfeatures [n,32], dL_doffsets [n,k,3], dL_dscaling [n,3], and
 *   dL_dparams, laid out as vpgs_mlp.params.
 * Any output may be NULL.  The anchor centres and the camera receive no gradient. */
vpgs_status vpgs_decode_anchors_bwd(void *ws, size_t ws_bytes, const vpgs_anchors *a,
                                    const vpgs_mlp *mlp, const vpgs_camera *cam,
                                    const double *T_cw, const vpgs_decode_opts *opts,
                                    const vpgs_gaussians *dL_dgauss, const int32_t *src_index,
                                    float *dL_dfeatures, float *dL_doffsets, float *dL_dscaling,
                                    float *dL_dparams, vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Mapping loss (Sec. III-A, Eq. 7-9)                                      */
/* ---------------------------------------------------------------------- */

/* Loss weights (host struct).  vpgs_loss_weights_default(): lambda_ssim 0.2 and
 * lambda_vol 0.001 (the paper's values, Sec. IV), lambda_d 1 (not stated). */
typedef struct {
    float lambda_ssim;  /* in [0, 1] */
    float lambda_d;     /* >= 0 */
    float lambda_vol;   /* >= 0 */
} vpgs_loss_weights;

void vpgs_loss_weights_default(vpgs_loss_weights *w);                 /* w: host */

/* Workspace bytes of vpgs_mapping_loss for n_views images of width x height
 * (0 if invalid: sizes <= 0 or > 65535, more than 4096 views). */
size_t vpgs_mapping_loss_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/* Mapping loss L_m = L_c + L_SSIM + lambda_d L_d + lambda_vol L_vol (Eq. 7),
 * L_SSIM = (1 - lambda_ssim) |I^ - I|_1 + lambda_ssim (1 - SSIM(I^, I)) (Eq. 8),
 * L_vol = sum_i Prod(s_i) (Eq. 9), and its gradient.  Readings: L_c and |.|_1 are
 * mean absolute colour differences; L_d sums |D^ - D| over pixels with target
 * depth > 0 and divides by the pixel count; SSIM uses an 11x11 Gaussian window
 * (sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2), averaged over views,
 * channels and pixels.
 *   rgb, target_rgb [V,3,H,W] float32 device (required).
 *   depth, target_depth [V,H,W] float32 device, both or neither (L_d = 0).
 *   scales [n_gaussians,3] float32 device; n_dev optional device count
 *     (as in vpgs_gaussians); n_gaussians 0 gives L_vol = 0.
 *   loss_out [5] float64 device, written: L_m, L_c, L_SSIM, L_d, L_vol.
 *   dL_drgb [V,3,H,W], dL_ddepth [V,H,W]: written (may be NULL);
 *   dL_dscales [n,3]: accumulated (+=) (may be NULL).
 * ws: 16-byte aligned, ws_bytes from vpgs_mapping_loss_workspace_bytes.
 * Two kernel launches, no host synchronisation; graph-capturable. */
vpgs_status vpgs_mapping_loss(void *ws, size_t ws_bytes, const float *rgb, const float *target_rgb,
                              const float *depth, const float *target_depth, int32_t n_views,
                              int32_t width, int32_t height, const float *scales, int64_t n_gaussians,
                              const int32_t *n_dev, const vpgs_loss_weights *w, double *loss_out,
                              float *dL_drgb, float *dL_ddepth, float *dL_dscales, vpgs_stream stream);

/* Coarse-tracking loss (Sec. III-B): the photometric and depth L1 errors of
 * the render at the current pose, per view v (the colour and depth terms of
 * the mapping loss, normalised per view):
 *   L_t(v) = (1/3HW) sum_{c,p} |I^ - I| + lambda_d (1/HW) sum_{p: D(p) > 0} |D^ - D|
 * and the gradient of sum_v L_t(v): sign(I^ - I) / 3HW and, where D > 0,
 * lambda_d sign(D^ - D) / HW (sign(0) = 0; 0 where D <= 0).
 *   rgb, target_rgb [V,3,H,W] float32 device (required).
 *   depth, target_depth [V,H,W] float32 device, both or neither (no depth term).
 *   lambda_d >= 0, finite.
 *   loss_out [V] float64 device, overwritten (may be NULL).
 *   dL_drgb [V,3,H,W], dL_ddepth [V,H,W] float32 device: overwritten (each may
 *     be NULL; dL_ddepth is not touched without depths).
 * Sizes: 1..65535 pixels per side, 1..4096 views; else VPGS_ERR_INVALID_ARG.
 * One kernel launch (plus a memset of loss_out); graph-capturable. */
vpgs_status vpgs_tracking_loss(const float *rgb, const float *target_rgb, const float *depth,
                               const float *target_depth, int32_t n_views, int32_t width, int32_t height,
                               float lambda_d, double *loss_out, float *dL_drgb, float *dL_ddepth,
                               vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Submap fusion (Sec. III-C, Eq. 14) and the optimiser step              */
/* ---------------------------------------------------------------------- */

/* Workspace bytes of vpgs_distill_loss (32 KiB; 0 if the sizes are invalid). */
size_t vpgs_distill_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/* Distillation loss between the renders of m = n_views overlapping keyframes
 * from two submaps a and b (Eq. 14):
 *   L = 1/m sum_kf ( mean_{c,p} (c_a - c_b)^2 + mean_p (d_a - d_b)^2 )
 * (reading: squared differences averaged over channels and pixels per image).
 *   rgb_a, rgb_b [m,3,H,W], depth_a, depth_b [m,H,W] (both or neither) float32 device.
 *   loss_out [3] float64 device, written: L, colour term, depth term.
 *   dL_d* : written, each may be NULL.
 * ws: 16-byte aligned.  Two launches, no host synchronisation. */
vpgs_status vpgs_distill_loss(void *ws, size_t ws_bytes, const float *rgb_a, const float *rgb_b,
                              const float *depth_a, const float *depth_b, int32_t n_views, int32_t width,
                              int32_t height, double *loss_out, float *dL_drgb_a, float *dL_drgb_b,
                              float *dL_ddepth_a, float *dL_ddepth_b, vpgs_stream stream);

/* One Adam step (Kingma and Ba, bias-corrected) over n float32 device values:
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 * params <- params - lr m^ / (sqrt(v^) + eps) with m^ = m / (1 - b1^step),
 * v^ = v / (1 - b2^step); grads is zeroed.  hyper (host) = {lr, b1, b2, eps};
 * step >= 1 is the 1-based step number.  The paper optimises the overlapping
 * submaps' parameters with the distillation loss; it names no optimiser. */
vpgs_status vpgs_adam_step(float *params, float *grads, float *m, float *v, int64_t n, const float hyper[4],
                           int32_t step, vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Fine tracking: voxel-hash ICP against the Gaussian means (Sec. III-B,   */
/* Eq. 10-12)                                                              */
/* ---------------------------------------------------------------------- */

/* The voxel of a point for an edge v is floor(x / v) per axis, evaluated in
 * float32 with the correctly rounded division.  Every voxel index must lie in
 * [-2^20, 2^20).  Poses here map the scan's local frame to the world (the
 * inverse of the renderer's T_cw) and are row-major double[4][4]. */

typedef struct {
    float map_voxel;    /* edge of the map's voxels: the `voxel` of vpgs_icp_build_map */
    float voxel_1;      /* first downsampling edge (the paper keeps one original point per voxel) */
    float voxel_2;      /* second downsampling edge, applied to the survivors of the first */
    float tau;          /* correspondence threshold tau_t (m), 0 < tau <= map_voxel */
    float sigma;        /* Geman-McClure scale sigma_t > 0 (Eq. 12); the caller adapts it */
    float eps;          /* stop once a step has |xi| < eps (>= 0) */
    int32_t iterations; /* maximum Gauss-Newton iterations, 1..1000 */
    int32_t pad;
} vpgs_icp_opts;

typedef struct {
    int32_t status;     /* VPGS_OK or the first device-side error (map or scan) */
    int32_t iterations; /* Gauss-Newton iterations run */
    int32_t n_source;   /* scan points kept by the double downsampling */
    int32_t n_corr;     /* correspondences of the last linearisation */
    int32_t stop;       /* 0 iterations ran out, 1 |xi| < eps, 2 fewer than 6
                           correspondences, 3 normal matrix not positive definite
                           (2 and 3 leave that iteration's pose unchanged) */
    int32_t pad;
    double cost;        /* sum of rho(e) over the last linearisation */
    double xi_norm;     /* |xi| of the last applied step */
} vpgs_icp_report;

typedef struct {
    int64_t n_points;
    int32_t n_voxels;   /* occupied voxels */
    int32_t capacity;   /* hash slots */
    int32_t status;     /* VPGS_ERR_NONFINITE / VPGS_ERR_INVALID_ARG: a point was
                           non-finite / outside the voxel range and was left out */
    float voxel;
} vpgs_icp_map_info;

/* Bytes of the map buffer for n_points points (0 if n_points < 0 or > 2^30). */
size_t vpgs_icp_map_bytes(int64_t n_points);

/* Builds the voxel hash map of the Gaussian means (the local map M of Sec.
 * III-B): points [n_points,3] float32 device, world frame; voxel > 0 (m).
 * map: device, 16-byte aligned, at least vpgs_icp_map_bytes(n_points); it holds
 * a header, an open-addressing table of the occupied voxels with the range of
 * their points, and the points grouped by voxel with their original index.
 * Every point of a voxel is kept.  Four launches. */
vpgs_status vpgs_icp_build_map(void *map, size_t map_bytes, const float *points, int64_t n_points, float voxel,
                               vpgs_stream stream);

/* Synchronises `stream` and copies the map header to the host. */
vpgs_status vpgs_icp_map_query(const void *map, vpgs_icp_map_info *info, vpgs_stream stream);

/* Workspace bytes of the ICP calls for scans of up to n_scan points (0 if
 * n_scan < 0 or > 2^30).  vpgs_icp_linearize needs vpgs_icp_workspace_bytes(0). */
size_t vpgs_icp_workspace_bytes(int64_t n_scan);

/* Double downsampling of a scan [n_scan,3] float32 device: the lowest-index
 * point of every voxel of edge voxel_1, then the lowest-index survivor of every
 * voxel of edge voxel_2.  Writes *n_out (device int32) and the kept original
 * indices, ascending, to idx_out[0 .. *n_out) (device, n_scan entries).
 * Non-finite or out-of-range points are dropped and set the workspace status. */
vpgs_status vpgs_icp_downsample(void *ws, size_t ws_bytes, const float *scan, int64_t n_scan, float voxel_1,
                                float voxel_2, int32_t *idx_out, int32_t *n_out, vpgs_stream stream);

/* One linearisation of Eq. 11 at pose T (device double[16]) for n_src source
 * points src [n_src,3] float32 device (no downsampling): for every s = T p the
 * nearest map point m with |s - m| < tau (float32 decision, ties to the lower
 * map index) and, over those pairs, the Geman-McClure weighted Gauss-Newton
 * system about the centre c (device double[3]):
 *   H = sum w J^T J, b = sum w J^T r, r = s - m, J = [I, -[s - c]x],
 *   w = k / (k + e^2)^2, k = sigma / 3, e = |r|.
 * system (device double[29]) = H's upper triangle row by row (21), b (6),
 * sum rho(e), the number of pairs.  corr (device int32[n_src] or NULL) = the
 * map point's original index or -1.  0 < tau <= map_voxel. */
vpgs_status vpgs_icp_linearize(void *ws, size_t ws_bytes, const void *map, size_t map_bytes, int64_t n_map,
                               float map_voxel, const float *src, int64_t n_src, const double *T,
                               const double *centre, float tau, float sigma, double *system, int32_t *corr,
                               vpgs_stream stream);

/* Registers a scan [n_scan,3] float32 device (local frame) against the map
 * (Eq. 10-12): double downsampling, then up to opts->iterations reweighted
 * Gauss-Newton steps T <- Tr(c) Exp(xi) Tr(-c) T (c = the translation of T on
 * entry; the same iterates as the left perturbation Exp(xi) T).  T (device
 * double[16]) holds the initial guess T_{i-1} T_pred on entry and the
 * registered pose on return.  report (device) is rewritten by every
 * iteration.  The launch sequence is fixed (2 + 4 + 2 * iterations kernels;
 * the steps after the stop do no work), so the call can be captured. */
vpgs_status vpgs_icp_register(void *ws, size_t ws_bytes, const void *map, size_t map_bytes, int64_t n_map,
                              const float *scan, int64_t n_scan, const vpgs_icp_opts *opts, double *T,
                              vpgs_icp_report *report, vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Submap expansion and anchor maintenance (Sec. III-A, "Voxel-Based      */
/* Submap Expansion and Activation")                                       */
/* ---------------------------------------------------------------------- */

/* Per-anchor statistics, one caller-owned device buffer of
 * vpgs_anchor_stats_bytes(A) bytes, 16-byte aligned.  With a4 = 4 A rounded
 * up to 16: float g_sum[A] at 0, float o_sum[A] at a4, uint32 g_cnt[A] at
 * 2 a4, uint32 visits[A] at 3 a4, uint32 status at 4 a4.  0 if A < 0 or > 2^30. */
size_t vpgs_anchor_stats_bytes(int64_t n_anchors);

/* Zeroes the statistics (one memset on `stream`). */
vpgs_status vpgs_anchor_stats_reset(void *stats, size_t stats_bytes, int64_t n_anchors, vpgs_stream stream);

/* Adds one training step: for every decoded neural Gaussian i < n (n =
 * min(n_cap, *n_dev), or n_cap when n_dev is NULL) of anchor a =
 * src_index[i] / k (the decoder's src_index, ascending):
 *   o_sum[a] += opacities[i];
 *   when visible[i] != 0 (or visible is NULL): g_sum[a] += |grad_means[i]|
 *     (the gradient of the 3D mean, [n,3]) and g_cnt[a] += 1;
 *   visits[a] += 1 for the first i of each anchor's run.
 * The paper averages the neural Gaussians' gradients per voxel and
 * accumulates their opacities; the gradient of the 3D mean and the
 * visibility (a non-empty tile cover) are readings.  FP32 atomics: the sums'
 * rounding order is not fixed.  An index outside [0, A k) sets the status. */
vpgs_status vpgs_anchor_stats_accumulate(void *stats, size_t stats_bytes, int64_t n_anchors, int32_t k,
                                         const int32_t *src_index, const int32_t *n_dev, int64_t n_cap,
                                         const float *grad_means, const float *opacities, const int32_t *visible,
                                         vpgs_stream stream);

typedef struct {
    float tau_g;      /* grow from anchors whose average gradient g_sum / g_cnt exceeds tau_g */
    float tau_o;      /* prune anchors with visits > 0 and o_sum < tau_o * visits */
    float grow_voxel; /* voxel edge of the grown anchors (> 0) */
    int32_t pad;
} vpgs_anchor_update_opts;

/* Workspace bytes of vpgs_anchor_update (0 if a size is negative or > 2^30). */
size_t vpgs_anchor_update_workspace_bytes(int64_t n_anchors, int64_t n_gaussians);

/* Pruning and growth from the statistics.
 *   keep_index [A] int32 device: the kept anchors, ascending, count in *n_keep
 *   (device int32).  An anchor is dropped when visits > 0 and
 *   o_sum < tau_o * visits (float32).
 *   grown [n_cap,3] float32 device: voxel centres (edge grow_voxel) of the
 *   decoded Gaussian means means[i] ([n_cap,3], the decoder's output) of
 *   anchors with g_cnt > 0 and g_sum > tau_g * g_cnt, whose voxel holds no
 *   anchor; each voxel once, in the order of its first i; count in *n_grown.
 *   anchor_map: vpgs_icp_build_map of the A anchor centres with voxel =
 *   grow_voxel (it answers "does a voxel hold an anchor").
 * Four launches; the status word of the workspace (vpgs_anchor_status kind 1)
 * reports non-finite means or a map that does not match. */
vpgs_status vpgs_anchor_update(void *ws, size_t ws_bytes, const void *stats, size_t stats_bytes, int64_t n_anchors,
                               int32_t k, const int32_t *src_index, const int32_t *n_dev, int64_t n_cap,
                               const float *means, const void *anchor_map, size_t anchor_map_bytes,
                               const vpgs_anchor_update_opts *opts, int32_t *keep_index, int32_t *n_keep,
                               float *grown, int32_t *n_grown, vpgs_stream stream);

typedef struct {
    float tau_alpha;   /* spawn where the rendered alpha is below this ... */
    float delta_depth; /* ... or where |rendered depth - input depth| exceeds this (>= 0) */
    float voxel;       /* voxel edge of the new anchors (> 0) */
    float rho;         /* no new anchor within rho of a Gaussian mean; 0 < rho <= map voxel */
    int32_t max_samples; /* M_k, pixels back-projected per keyframe, 1..2^26 */
    int32_t pad;
} vpgs_spawn_opts;

/* Workspace bytes of vpgs_spawn_anchors (0 if the sizes are invalid). */
size_t vpgs_spawn_workspace_bytes(int32_t width, int32_t height, int32_t max_samples);

/* New anchors of one keyframe (Sec. III-A): the pixels with input depth > 0
 * whose rendered alpha < tau_alpha or |rendered depth - input depth| >
 * delta_depth (float32); of their C (raster order) the rank r is kept iff
 * floor((r+1) M / C) > floor(r M / C) (all when C <= M), as sample
 * floor((r+1) M / C) - 1; each sample is back-projected through the pixel
 * centre with its input depth and the world-to-camera pose T_cw (device
 * double[16]) in FP64, rounded to float32; its voxel (edge voxel) becomes an
 * anchor at the voxel centre if it is the voxel's first sample and no point of
 * gauss_map (vpgs_icp_build_map of the Gaussian means, n_map points, edge
 * map_voxel >= rho) lies closer than rho to that centre.
 *   alpha, depth, depth_in [H,W] float32 device (W, H from cam).
 *   anchors_out [max_samples,3] float32 device: the new anchors in sample order;
 *   *n_out (device int32) their number.  samples_out [max_samples,3] and
 *   *n_samples (device) receive the back-projected samples; either may be NULL.
 * The paper samples M_k points at random; the even spread is a reading.  Five
 * launches; status: vpgs_anchor_status kind 2. */
vpgs_status vpgs_spawn_anchors(void *ws, size_t ws_bytes, const float *alpha, const float *depth,
                               const float *depth_in, const vpgs_camera *cam, const double *T_cw,
                               const void *gauss_map, size_t map_bytes, int64_t n_map, float map_voxel,
                               const vpgs_spawn_opts *opts, float *anchors_out, int32_t *n_out, float *samples_out,
                               int32_t *n_samples, vpgs_stream stream);

/* Synchronises `stream` and reads a device status word: kind 0 = statistics
 * buffer (n_anchors gives its layout), 1 = vpgs_anchor_update workspace,
 * 2 = vpgs_spawn_anchors workspace. */
vpgs_status vpgs_anchor_status(const void *ws_or_stats, int32_t kind, int64_t n_anchors, int32_t *status_out,
                               vpgs_stream stream);

/* ---------------------------------------------------------------------- */
/* Diagnostics (host)                                                      */
/* ---------------------------------------------------------------------- */

/* Number of CUDA kernels this process has launched through the library. */
int64_t vpgs_launch_count(void);

/* Per-kernel timing.  While enabled, every library kernel launch is bracketed
 * by a CUDA event pair recorded on its own stream.  Off by default, because
 * each event costs a few microseconds of host time. */
void vpgs_profile_enable(int32_t on);

/* Synchronises the recorded events, aggregates them per kernel name and clears
 * them.  It writes up to max_entries entries: names as consecutive
 * NUL-terminated strings in the host buffer names[name_bytes], launches[i],
 * and total_ms[i].  Returns the number of entries written. */
int32_t vpgs_profile_collect(char *names, size_t name_bytes, int64_t *launches, double *total_ms,
                             int32_t max_entries);

const char *vpgs_status_string(vpgs_status s);
/* Library version, "major.minor.patch" (host string). */
const char *vpgs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VPGS_H */
