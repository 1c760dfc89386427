"""Autotuner for the render launch shape.

Picks, for one workload on one GPU, the tile shape (tile_w x tile_h), the
persistent CTAs per SM (0 = one CTA per tile) and how many views go into one
render call, by timing fwd+bwd steps with CUDA events.  The image does not
depend on any of these (the tile cover is a superset of every contributing
pixel), so the choice is about time only -- and each candidate is checked
before it may win: on the tuning frame its contributor counts must equal the
default shape's bit for bit and its images (colour, depth, alpha, final
transmittance) must lie within 1e-5 of them; its list positions (n_iter) must
equal those of the same tile shape rendered one call, one CTA per tile.
Candidates that fail are rejected with the reason.  Results are cached in a
JSON file keyed by the GPU name and the workload's shape.
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import asdict, dataclass

TILE_WIDTHS = (4, 8, 16, 32)
DEFAULT_TILES = ((8, 16), (16, 16), (16, 8), (8, 8), (8, 32), (32, 8))
DEFAULT_PERSISTENT = (0, 4)


@dataclass(frozen=True)
class LaunchShape:
    tile_w: int
    tile_h: int
    persistent_ctas: int = 0
    views_per_call: int = 1


def valid_tile(tile_w: int, tile_h: int, pix_per_thread: int = 1) -> bool:
    """The library's tile rules: tile_w in {4,8,16,32}; tile_h even, at most 64;
    tile_w*tile_h a multiple of 64 and at most 512 threads per tile."""
    b = tile_w * tile_h
    return (tile_w in TILE_WIDTHS and 2 <= tile_h <= 64 and tile_h % 2 == 0 and b % 64 == 0
            and b // pix_per_thread <= 512 and tile_h % pix_per_thread == 0)


def candidates(n_views: int = 1, tiles=DEFAULT_TILES, persistent=DEFAULT_PERSISTENT, views_per_call=None):
    """Every valid LaunchShape of the given choices; views per call must divide n_views."""
    vpc = views_per_call or sorted({v for v in (n_views, n_views // 2, 1) if v >= 1 and n_views % v == 0},
                                   reverse=True)
    out = []
    for tw, th in tiles:
        if not valid_tile(tw, th):
            continue
        for p in persistent:
            for v in vpc:
                if v >= 1 and n_views % v == 0:
                    out.append(LaunchShape(tw, th, int(p), int(v)))
    return out


def workload_key(n_gaussians: int, width: int, height: int, n_views: int) -> str:
    """Cache key of a workload: Gaussian count to 2 significant digits, image size, views."""
    n = int(n_gaussians)
    if n >= 100:
        e = len(str(n)) - 2
        n = round(n / 10 ** e) * 10 ** e
    return f"n{n}_{width}x{height}_v{n_views}"


DEFAULT_SHAPE = LaunchShape(16, 16, 0, 0)  # views_per_call 0: all views in one call
IMAGE_TOL = 1e-5


def compare_outputs(cand: dict, ref: dict, ref_same_tile: dict | None = None, tol: float = IMAGE_TOL):
    """None when the candidate's render matches the reference, else the reason.

    cand/ref: dicts of numpy arrays rgb, depth, alpha, t_final, n_contrib (and
    n_iter).  n_contrib must be identical; the images within tol; n_iter is
    compared (identical) only with ref_same_tile, a render with the same tile
    shape, since list positions depend on the tiles."""
    import numpy as np
    if not np.array_equal(cand["n_contrib"], ref["n_contrib"]):
        return f"n_contrib differs at {int((cand['n_contrib'] != ref['n_contrib']).sum())} pixels"
    for k in ("rgb", "depth", "alpha", "t_final"):
        err = float(np.abs(np.asarray(cand[k], np.float64) - np.asarray(ref[k], np.float64)).max())
        if not err <= tol:
            return f"{k} differs by {err:.3g}"
    if ref_same_tile is not None and not np.array_equal(cand["n_iter"], ref_same_tile["n_iter"]):
        return "n_iter differs from the same tile shape's render"
    return None


def pick(timings: dict) -> LaunchShape:
    """The fastest shape; ties go to the first in candidate order."""
    if not timings:
        raise ValueError("no timings")
    best = min(timings.items(), key=lambda kv: kv[1])
    return best[0]


class Cache:
    """JSON cache: {gpu name: {workload key: {"shape": {...}, "ms": t}}}."""

    def __init__(self, path: str | None):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, gpu: str, key: str):
        e = self.data.get(gpu, {}).get(key)
        return (LaunchShape(**e["shape"]), e["ms"]) if e else None

    def put(self, gpu: str, key: str, shape: LaunchShape, ms: float):
        self.data.setdefault(gpu, {})[key] = {"shape": asdict(shape), "ms": float(ms)}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def time_shape(shape: LaunchShape, gaussians, T_cw, intr, g_rgb, steps: int = 5, warmup: int = 2) -> float:
    """Median ms of one fwd+bwd over all views of T_cw with the given launch shape."""
    import torch

    from .render import Renderer

    V = T_cw.shape[0]
    calls = V // shape.views_per_call
    r = Renderer(intr, n_views=shape.views_per_call, tile_w=shape.tile_w, tile_h=shape.tile_h,
                 persistent_ctas=shape.persistent_ctas)
    Ts = [T_cw[c * shape.views_per_call:(c + 1) * shape.views_per_call].contiguous() for c in range(calls)]
    gs = [g_rgb[c * shape.views_per_call:(c + 1) * shape.views_per_call].contiguous() for c in range(calls)]
    outs = [r.forward(*gaussians, Tc, check=True) for Tc in Ts]  # sizes the instance capacity
    grads = {k: torch.zeros_like(t) for k, t in zip(("means", "scales", "quats", "opacities", "colors"), gaussians)}
    dpose = torch.zeros((shape.views_per_call, 6), dtype=torch.float64, device=T_cw.device)

    def step():
        for Tc, o, gc in zip(Ts, outs, gs):
            r.forward(*gaussians, Tc, out=o, check=False)
            r.backward(*gaussians, Tc, o, gc, None, None, grads=grads, dpose=dpose)

    for _ in range(warmup):
        step()
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    st = r.stats()
    if st.status != 0:
        raise RuntimeError(f"render status {st.status} for {shape}")
    return statistics.median(times)


def render_shape(shape: LaunchShape, gaussians, T_cw, intr) -> dict:
    """Forward render of every view of T_cw with the given launch shape (numpy outputs)."""
    import numpy as np
    import torch

    from .render import Renderer

    V = int(T_cw.shape[0])
    vpc = shape.views_per_call or V
    r = Renderer(intr, n_views=vpc, tile_w=shape.tile_w, tile_h=shape.tile_h,
                 persistent_ctas=shape.persistent_ctas)
    parts = [r.forward(*gaussians, T_cw[c:c + vpc].contiguous(), check=True) for c in range(0, V, vpc)]
    torch.cuda.synchronize()
    return {k: np.concatenate([p[k].cpu().numpy() for p in parts], 0) for k in parts[0]}


def validate(shapes, gaussians, T_cw, intr) -> dict:
    """{shape: None (valid) or the reason it was rejected} on the tuning frame."""
    ref = render_shape(DEFAULT_SHAPE, gaussians, T_cw, intr)
    same_tile = {}
    out = {}
    for s in shapes:
        tile = (s.tile_w, s.tile_h)
        if tile not in same_tile:
            same_tile[tile] = render_shape(LaunchShape(s.tile_w, s.tile_h, 0, 0), gaussians, T_cw, intr)
        out[s] = compare_outputs(render_shape(s, gaussians, T_cw, intr), ref, same_tile[tile])
    return out


def tune(gaussians, T_cw, intr, g_rgb, shapes=None, steps: int = 5, cache_path: str | None = None,
         key: str | None = None, return_rejected: bool = False):
    """Times every candidate shape that renders the tuning frame as the default
    shape does (or returns the cached winner); returns (best LaunchShape,
    {shape: ms}) and, with return_rejected, also {shape: reason} of the
    candidates left out."""
    import torch

    V = int(T_cw.shape[0])
    gpu = torch.cuda.get_device_name(T_cw.device)
    key = key or workload_key(gaussians[0].shape[0], intr.width, intr.height, V)
    cache = Cache(cache_path)
    hit = cache.get(gpu, key)
    if hit is not None and shapes is None:
        return (hit[0], {hit[0]: hit[1]}, {}) if return_rejected else (hit[0], {hit[0]: hit[1]})
    shapes = shapes or candidates(V)
    checks = validate(shapes, gaussians, T_cw, intr)
    rejected = {s: why for s, why in checks.items() if why is not None}
    timings = {s: time_shape(s, gaussians, T_cw, intr, g_rgb, steps=steps) for s in shapes if s not in rejected}
    best = pick(timings)
    cache.put(gpu, key, best, timings[best])
    return (best, timings, rejected) if return_rejected else (best, timings)
