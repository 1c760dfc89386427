// Anchor decoder entry points (filled in below the render path).
#include "internal.h"

extern "C" {

size_t vpgs_decode_workspace_bytes(int64_t n_anchors, int32_t k) {
    (void)n_anchors; (void)k;
    return 0;
}

vpgs_status vpgs_decode_anchors(void *, size_t, const vpgs_anchors *, const vpgs_mlp *,
                                const vpgs_camera *, const double *, const vpgs_decode_opts *,
                                const vpgs_gaussian_buffers *, int32_t *, int32_t *, vpgs_stream) {
    return VPGS_ERR_UNSUPPORTED;
}

vpgs_status vpgs_decode_anchors_bwd(void *, size_t, const vpgs_anchors *, const vpgs_mlp *,
                                    const vpgs_camera *, const double *, const vpgs_decode_opts *,
                                    const vpgs_gaussians *, const int32_t *, float *, float *, float *,
                                    float *, vpgs_stream) {
    return VPGS_ERR_UNSUPPORTED;
}

}  // extern "C"
