"""FP64 CPU oracle for the rasterizer and the anchor decoder.

TEST INFRASTRUCTURE: imported only by the test-suite, the package smoke check
and the benchmark's CPU-baseline and reference arms.  The CUDA product path
never imports, links or runs anything in this package, and this package imports
nothing from the product.
"""
from .raster import (Options, Margins, render, render_scene, project, extent, tile_cover,  # noqa: F401
                     rect_min_quadratic, quat_to_rotmat)
from .decode import decode, decode_scene, bf16_round, n_mlp_params, flatten_mlp, MLP_ORDER  # noqa: F401,E402
from .pose import pose_step, se3_exp  # noqa: F401,E402
from .loss import mapping_loss, tracking_loss, ssim_map, gaussian_window  # noqa: F401,E402
from .fusion import distill_loss, adam_step  # noqa: F401,E402
from .icp import icp as voxel_icp, voxel_downsample  # noqa: F401,E402
from .anchors import spawn as spawn_anchors, accumulate_stats, prune as prune_anchors, grow as grow_anchors  # noqa: F401,E402
