"""ctypes binding of libvpgs (include/vpgs.h): struct mirrors and the C entry points.

Argument marshalling only.  Every computation runs in the CUDA library; if
the library is missing or no GPU is present, calling any entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libvpgs.so")

VPGS_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "tile-instance capacity exceeded",
                3: "non-finite input", 4: "bounded device wait ran out", 5: "CUDA error",
                6: "unsupported", 7: "internal consistency check failed"}


class VpgsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({code})")
        self.code = code


class vpgs_camera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float)]


class vpgs_render_opts(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("alpha_min", c_float),
                ("alpha_max", c_float), ("t_min", c_float), ("dilation", c_float),
                ("near_z", c_float), ("bg", c_float * 3), ("persistent_ctas", c_int32),
                ("flags", c_int32),
        ("spin_limit", c_int32)]


RENDER_REUSE_BINNING = 1


class vpgs_gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p),
                ("opacities", c_void_p), ("colors", c_void_p), ("n", c_int64), ("n_dev", c_void_p)]


class vpgs_gaussian_buffers(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p),
                ("opacities", c_void_p), ("colors", c_void_p)]


class vpgs_images(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("alpha", c_void_p), ("t_final", c_void_p),
                ("n_contrib", c_void_p), ("n_iter", c_void_p)]


class vpgs_render_stats(ctypes.Structure):
    _fields_ = [("status", c_int32), ("n_visible", c_int64), ("n_instances", c_int64)]


class vpgs_anchors(ctypes.Structure):
    _fields_ = [("anchors", c_void_p), ("scaling", c_void_p), ("offsets", c_void_p),
                ("features", c_void_p), ("n", c_int64), ("k", c_int32), ("features_bf16", c_int32)]


class vpgs_mlp(ctypes.Structure):
    _fields_ = [("params", c_void_p), ("bf16", c_int32)]


class vpgs_decode_opts(ctypes.Structure):
    _fields_ = [("near_z", c_float), ("guard", c_float)]


class vpgs_loss_weights(ctypes.Structure):
    _fields_ = [("lambda_ssim", c_float), ("lambda_d", c_float), ("lambda_vol", c_float)]


class vpgs_icp_opts(ctypes.Structure):
    _fields_ = [("map_voxel", c_float), ("voxel_1", c_float), ("voxel_2", c_float), ("tau", c_float),
                ("sigma", c_float), ("eps", c_float), ("iterations", c_int32), ("pad", c_int32)]


class vpgs_icp_report(ctypes.Structure):
    _fields_ = [("status", c_int32), ("iterations", c_int32), ("n_source", c_int32), ("n_corr", c_int32),
                ("stop", c_int32), ("pad", c_int32), ("cost", c_double), ("xi_norm", c_double)]


class vpgs_icp_map_info(ctypes.Structure):
    _fields_ = [("n_points", c_int64), ("n_voxels", c_int32), ("capacity", c_int32), ("status", c_int32),
                ("voxel", c_float)]


class vpgs_anchor_update_opts(ctypes.Structure):
    _fields_ = [("tau_g", c_float), ("tau_o", c_float), ("grow_voxel", c_float), ("pad", c_int32)]


class vpgs_spawn_opts(ctypes.Structure):
    _fields_ = [("tau_alpha", c_float), ("delta_depth", c_float), ("voxel", c_float), ("rho", c_float),
                ("max_samples", c_int32), ("pad", c_int32)]


_SIGS = {
    "vpgs_render_opts_default": (None, [POINTER(vpgs_render_opts)]),
    "vpgs_render_workspace_bytes": (c_size_t, [c_int64, c_int32, POINTER(vpgs_camera),
                                               POINTER(vpgs_render_opts), c_int64]),
    "vpgs_render_fwd": (c_int32, [c_void_p, c_size_t, POINTER(vpgs_gaussians), POINTER(vpgs_camera),
                                  c_void_p, c_int32, POINTER(vpgs_render_opts), POINTER(vpgs_images),
                                  c_void_p]),
    "vpgs_render_bwd": (c_int32, [c_void_p, c_size_t, POINTER(vpgs_gaussians), POINTER(vpgs_camera),
                                  c_void_p, c_int32, POINTER(vpgs_render_opts), POINTER(vpgs_images),
                                  c_void_p, c_void_p, c_void_p, POINTER(vpgs_gaussian_buffers),
                                  c_void_p, c_void_p]),
    "vpgs_render_project": (c_int32, [c_void_p, c_size_t, POINTER(vpgs_gaussians),
                                      POINTER(vpgs_camera), c_void_p, c_int32,
                                      POINTER(vpgs_render_opts), c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p]),
    "vpgs_render_fwd_noalloc": (c_int32, [POINTER(vpgs_gaussians), POINTER(vpgs_camera), c_void_p,
                                          c_int32, POINTER(vpgs_render_opts), POINTER(vpgs_images),
                                          c_void_p, c_void_p]),
    "vpgs_workspace_status": (c_int32, [c_void_p, POINTER(vpgs_render_stats), c_void_p]),
    "vpgs_workspace_status_copy": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "vpgs_pose_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, POINTER(c_double),
                                 c_void_p]),
    "vpgs_decode_workspace_bytes": (c_size_t, [c_int64, c_int32]),
    "vpgs_decode_anchors": (c_int32, [c_void_p, c_size_t, POINTER(vpgs_anchors), POINTER(vpgs_mlp),
                                      POINTER(vpgs_camera), c_void_p, POINTER(vpgs_decode_opts),
                                      POINTER(vpgs_gaussian_buffers), c_void_p, c_void_p, c_void_p]),
    "vpgs_decode_anchors_bwd": (c_int32, [c_void_p, c_size_t, POINTER(vpgs_anchors),
                                          POINTER(vpgs_mlp), POINTER(vpgs_camera), c_void_p,
                                          POINTER(vpgs_decode_opts), POINTER(vpgs_gaussians),
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_loss_weights_default": (None, [POINTER(vpgs_loss_weights)]),
    "vpgs_mapping_loss_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "vpgs_mapping_loss": (c_int32, [c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                    c_int32, c_int32, c_void_p, c_int64, c_void_p, POINTER(vpgs_loss_weights),
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_tracking_loss": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_distill_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "vpgs_distill_loss": (c_int32, [c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                    c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_adam_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_float), c_int32,
                                 c_void_p]),
    "vpgs_icp_map_bytes": (c_size_t, [c_int64]),
    "vpgs_icp_build_map": (c_int32, [c_void_p, c_size_t, c_void_p, c_int64, c_float, c_void_p]),
    "vpgs_icp_map_query": (c_int32, [c_void_p, POINTER(vpgs_icp_map_info), c_void_p]),
    "vpgs_icp_workspace_bytes": (c_size_t, [c_int64]),
    "vpgs_icp_downsample": (c_int32, [c_void_p, c_size_t, c_void_p, c_int64, c_float, c_float, c_void_p, c_void_p,
                                      c_void_p]),
    "vpgs_icp_linearize": (c_int32, [c_void_p, c_size_t, c_void_p, c_size_t, c_int64, c_float, c_void_p, c_int64,
                                     c_void_p, c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "vpgs_icp_register": (c_int32, [c_void_p, c_size_t, c_void_p, c_size_t, c_int64, c_void_p, c_int64,
                                    POINTER(vpgs_icp_opts), c_void_p, c_void_p, c_void_p]),
    "vpgs_anchor_stats_bytes": (c_size_t, [c_int64]),
    "vpgs_anchor_stats_reset": (c_int32, [c_void_p, c_size_t, c_int64, c_void_p]),
    "vpgs_anchor_stats_accumulate": (c_int32, [c_void_p, c_size_t, c_int64, c_int32, c_void_p, c_void_p, c_int64,
                                               c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_anchor_update_workspace_bytes": (c_size_t, [c_int64, c_int64]),
    "vpgs_anchor_update": (c_int32, [c_void_p, c_size_t, c_void_p, c_size_t, c_int64, c_int32, c_void_p, c_void_p,
                                     c_int64, c_void_p, c_void_p, c_size_t, POINTER(vpgs_anchor_update_opts),
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_spawn_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "vpgs_spawn_anchors": (c_int32, [c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, POINTER(vpgs_camera),
                                     c_void_p, c_void_p, c_size_t, c_int64, c_float, POINTER(vpgs_spawn_opts),
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vpgs_anchor_status": (c_int32, [c_void_p, c_int32, c_int64, POINTER(c_int32), c_void_p]),
    "vpgs_launch_count": (c_int64, []),
    "vpgs_profile_enable": (None, [c_int32]),
    "vpgs_profile_collect": (c_int32, [c_char_p, c_size_t, POINTER(c_int64), POINTER(c_double),
                                       c_int32]),
    "vpgs_status_string": (c_char_p, [c_int32]),
    "vpgs_version": (c_char_p, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libvpgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2505_18992_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def exported_names():
    return list(_SIGS)


def check(code: int, what: str):
    if code != VPGS_OK:
        raise VpgsError(code, what)


def ptr(t) -> int | None:
    """Device (or host) address of a tensor, None for None."""
    return None if t is None else t.data_ptr()


def _entry(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    return call


# same names as the C entry points
vpgs_render_opts_default = _entry("vpgs_render_opts_default")
vpgs_render_workspace_bytes = _entry("vpgs_render_workspace_bytes")
vpgs_render_fwd = _entry("vpgs_render_fwd")
vpgs_render_bwd = _entry("vpgs_render_bwd")
vpgs_render_project = _entry("vpgs_render_project")
vpgs_render_fwd_noalloc = _entry("vpgs_render_fwd_noalloc")
vpgs_workspace_status = _entry("vpgs_workspace_status")
vpgs_workspace_status_copy = _entry("vpgs_workspace_status_copy")
vpgs_pose_step = _entry("vpgs_pose_step")
vpgs_decode_workspace_bytes = _entry("vpgs_decode_workspace_bytes")
vpgs_decode_anchors = _entry("vpgs_decode_anchors")
vpgs_decode_anchors_bwd = _entry("vpgs_decode_anchors_bwd")
vpgs_loss_weights_default = _entry("vpgs_loss_weights_default")
vpgs_mapping_loss_workspace_bytes = _entry("vpgs_mapping_loss_workspace_bytes")
vpgs_mapping_loss = _entry("vpgs_mapping_loss")
vpgs_tracking_loss = _entry("vpgs_tracking_loss")
vpgs_distill_workspace_bytes = _entry("vpgs_distill_workspace_bytes")
vpgs_distill_loss = _entry("vpgs_distill_loss")
vpgs_adam_step = _entry("vpgs_adam_step")
vpgs_icp_map_bytes = _entry("vpgs_icp_map_bytes")
vpgs_icp_build_map = _entry("vpgs_icp_build_map")
vpgs_icp_map_query = _entry("vpgs_icp_map_query")
vpgs_icp_workspace_bytes = _entry("vpgs_icp_workspace_bytes")
vpgs_icp_downsample = _entry("vpgs_icp_downsample")
vpgs_icp_linearize = _entry("vpgs_icp_linearize")
vpgs_icp_register = _entry("vpgs_icp_register")
vpgs_anchor_stats_bytes = _entry("vpgs_anchor_stats_bytes")
vpgs_anchor_stats_reset = _entry("vpgs_anchor_stats_reset")
vpgs_anchor_stats_accumulate = _entry("vpgs_anchor_stats_accumulate")
vpgs_anchor_update_workspace_bytes = _entry("vpgs_anchor_update_workspace_bytes")
vpgs_anchor_update = _entry("vpgs_anchor_update")
vpgs_spawn_workspace_bytes = _entry("vpgs_spawn_workspace_bytes")
vpgs_spawn_anchors = _entry("vpgs_spawn_anchors")
vpgs_anchor_status = _entry("vpgs_anchor_status")
vpgs_launch_count = _entry("vpgs_launch_count")
vpgs_profile_enable = _entry("vpgs_profile_enable")
vpgs_profile_collect = _entry("vpgs_profile_collect")
vpgs_status_string = _entry("vpgs_status_string")
vpgs_version = _entry("vpgs_version")


def default_opts(**kw) -> vpgs_render_opts:
    o = vpgs_render_opts()
    vpgs_render_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "bg":
            o.bg = (c_float * 3)(*v)
        else:
            setattr(o, k, v)
    return o


def profile_collect(max_entries: int = 64):
    """{kernel name: (launches, total ms)} of the events recorded while profiling was on."""
    names = ctypes.create_string_buffer(64 * max_entries)
    launches = (c_int64 * max_entries)()
    total = (c_double * max_entries)()
    n = vpgs_profile_collect(names, len(names), launches, total, max_entries)
    raw = names.raw.split(b"\0")
    return {raw[i].decode(): (int(launches[i]), float(total[i])) for i in range(n)}
