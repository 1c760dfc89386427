#!/usr/bin/env python3
"""Forward+backward RGB-D throughput of the Gaussian rasterizer on one GB300.

Workload: the 1M-Gaussian room (6 walls of a 6x5x3 m room plus 20 boxes) seen
by a 1200x680 camera (fx = fy = 600).  The room stands in for the paper's
Replica/ScanNet rooms, whose data is not available.  One step is
vpgs_render_fwd followed by vpgs_render_bwd: gradients to every Gaussian
parameter and to the 6-DoF pose, with the tile lists recomputed in the
backward.  The upstream gradient is a fixed seeded L1-type pattern
(+-1/(3P) colour, +-1/P depth).  Inputs (56 MB) are smaller than L2, so a
256 MiB buffer is written between timed steps to flush L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun, each rank renders its own copy of the workload (independent
replicas, weak scaling).  There is no data-path collective; a barrier and a
max-reduction of the timings are the only cross-rank steps.
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd RGB-D Mpix/s at 1M Gaussians 1200×680; % HBM roofline; vs plain form"
UNIT = "Mpix/s"
WORKLOAD = "indoor room: 1,000,000 Gaussians, 1200x680 RGB-D-alpha, fwd+bwd (all Gaussian params + 6-DoF pose)"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--cpu-rows", type=int, default=8, help="image rows in the CPU oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip tracking/e2e/profile passes")
    p.add_argument("--no-rows", action="store_true", help="keep the kernel profile, skip the other rows")
    p.add_argument("--row", choices=("tracking", "decode", "batched_keyframes", "fusion", "mapping", "icp",
                                     "anchors"),
                   help="run only this secondary row and print it (a profiling entry point, not a bench line)")
    p.add_argument("--persistent", type=int, default=0, help="persistent CTAs per SM (0 = per tile)")
    p.add_argument("--tile", default="16x16", help="tile shape WxH")
    p.add_argument("--scale", type=float, default=1.0,
                   help="shrink the workload for profiling: N x scale^2 Gaussians, image x scale")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (one MAX all-reduce; identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------

def oracle_sample(scene, n_rows: int):
    """Times the FP64 oracle fwd+bwd on n_rows evenly spaced rows of the frame."""
    import torch

    import oracle
    from paper_2505_18992_gb300 import scenes
    H, W = scene.camera.height, scene.camera.width
    rows = [int(r) for r in np.linspace(0, H - 1, n_rows)]
    g = scenes.upstream_grads(11, 1, H, W)
    t0 = time.perf_counter()
    oracle.render_scene(scene, rows=rows, grads=g)
    dt = time.perf_counter() - t0
    px = n_rows * W
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{n_rows} image rows x {W} px of the same 1M-Gaussian frame (projection of all "
                      f"1M Gaussians + per-pixel compositing and backward), {dt:.2f} s"}


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2505_18992_gb300 import scenes
    scene = scenes.indoor_room()
    vals = []
    for _ in range(a.warmup):
        oracle_sample(scene, 1)
    last = None
    for _ in range(a.steps):
        last = oracle_sample(scene, max(1, a.cpu_rows // 4))
        vals.append(last["value"])
    v = statistics.median(vals)
    px_step = max(1, a.cpu_rows // 4) * scene.camera.width
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": px_step / (v * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_rows": max(1, a.cpu_rows // 4)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50", "-i", gpu_id,
                                          "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                ts = _dt.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, f))
        except Exception:
            pass
        inside = [f for ts, f in rows if t0 - 0.05 <= ts <= t1 + 0.05]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(f[1]) for f in inside if f[1].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for f in inside:
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(inside[0][2]) if inside[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(inside),
                "power_w_max": max(float(f[3]) for f in inside if f[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------------------
# algorithmic bytes of the hot kernels (per launch)
# ---------------------------------------------------------------------------

def algorithmic_bytes(kernel: str, N: int, Nv: int, M: int, P: int):
    """Minimum DRAM bytes a launch must move, from the unit counts of the frame.

    N Gaussians, Nv visible ones, M tile instances, P pixels."""
    table = {
        # pre-cull: read 56 B of parameters and write a 4 B tile count per Gaussian
        "preprocess_fwd": 60 * N,
        # exact projection: write the 64 B screen record, the 64 B binning record and
        # zero the 40 B of 2D gradient slots per visible Gaussian
        "project": 168 * Nv,
        # gather id + 48 B record per instance; write RGB, depth, alpha, T, count (28 B/px)
        "composite_fwd": 52 * M + 28 * P,
        # same gather, read T, list length and 20 B of upstream gradient per pixel, write 40 B/visible
        "composite_bwd": 52 * M + 28 * P + 40 * Nv,
        # per visible Gaussian: read 40 B of mean / scale / rotation and the 40 B of 2D
        # gradients, zero those slots, add 56 B of parameter gradients
        "preprocess_bwd": 176 * Nv,
        # per pass: read and write one 8-byte (key, value) pair per item
        "radix_onesweep": None,
    }
    return table.get(kernel)


# FP32 flops (FMA = 2) of one pixel-Gaussian pair, counted from the method's
# arithmetic: evaluating alpha (offset 2, whitened form 6, power 4, exp 2,
# opacity 1, clamp 1 = 17) and, for blended pairs, the blend (forward: 1 - alpha,
# T update, weight, 4 accumulations = 11) or the gradient (backward: T recovery 4,
# weight 1, colour/depth grads 8, dalpha 10 (g . c, minus g . B, times T plus
# the alpha term), update of g . B 2, opacity and power 3, mean 4, conic 8 = 40;
# the whitening rows of the mean gradient are applied once per Gaussian).
PAIR_FLOPS = {"eval": 17, "blend_fwd": 11, "blend_bwd": 40}


def alu_peak_tflops(sm_mhz, sms):
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def step_floor_bytes(N: int, Nv: int, M: int, P: int) -> int:
    """Algorithmic DRAM bytes of one fwd+bwd step (recompute form), the floor the
    method must move with a one-pass sort: forward = pre-cull 56 N, projection
    52 Nv, instance keys 12 M, sort 24 M, ranges 8 M, compositing 52 M + 28 P;
    backward = the same projection and binning again (56 N + 52 Nv + 44 M),
    compositing 52 M + 28 P + 40 Nv, preprocess backward 96 Nv + 56 N."""
    fwd = 56 * N + 52 * Nv + (12 + 24 + 8 + 52) * M + 28 * P
    bwd = 56 * N + 52 * Nv + (12 + 24 + 8) * M + 52 * M + 28 * P + 40 * Nv + 96 * Nv + 56 * N
    return fwd + bwd


def _sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "composite_fwd": ["paper_2505_18992_gb300/csrc/render_comp.cu", "paper_2505_18992_gb300/csrc/common.cuh"],
    "composite_bwd": ["paper_2505_18992_gb300/csrc/render_comp.cu", "paper_2505_18992_gb300/csrc/common.cuh"],
    "preprocess_fwd": ["paper_2505_18992_gb300/csrc/render_pre.cu", "paper_2505_18992_gb300/csrc/common.cuh"],
    "project": ["paper_2505_18992_gb300/csrc/render_pre.cu", "paper_2505_18992_gb300/csrc/common.cuh"],
    "preprocess_bwd": ["paper_2505_18992_gb300/csrc/render_pre.cu", "paper_2505_18992_gb300/csrc/common.cuh"],
    "radix_onesweep": ["paper_2505_18992_gb300/csrc/prims.cuh"],
    "scan_lookback": ["paper_2505_18992_gb300/csrc/prims.cuh", "paper_2505_18992_gb300/csrc/render_bin.cu"],
}


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            d = json.load(fh)
        e = d[kernel]
        if e.get("source_sha") != _sha(KERNEL_SOURCES[kernel]):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.build import build
    from paper_2505_18992_gb300.render import Intrinsics, Renderer

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    C.lib()
    dev = torch.device("cuda", local)
    if a.scale == 1.0:
        sc = scenes.indoor_room()
    else:
        sc = scenes.indoor_room(n=int(1_000_000 * a.scale ** 2), width=int(1200 * a.scale),
                                height=int(680 * a.scale) // 2 * 2, f=600.0 * a.scale)
    cam = sc.camera
    H, W, V = cam.height, cam.width, 1
    P = V * H * W
    g = [torch.tensor(x, device=dev).contiguous() for x in sc.arrays()]
    T = torch.tensor(cam.T_cw, dtype=torch.float64, device=dev).contiguous()
    tw, th = (int(x) for x in a.tile.lower().split("x"))
    r = Renderer(Intrinsics(W, H, cam.fx, cam.fy, cam.cx, cam.cy), device=dev,
                 persistent_ctas=a.persistent, tile_w=tw, tile_h=th)
    rng = np.random.default_rng(5)
    g_rgb = torch.tensor(np.sign(rng.normal(size=(1, 3, H, W))) / (3 * P), dtype=torch.float32, device=dev)
    g_d = torch.tensor(np.sign(rng.normal(size=(1, H, W))) / P, dtype=torch.float32, device=dev)
    names = ("means", "scales", "quats", "opacities", "colors")
    grads = {k: torch.zeros_like(t) for k, t in zip(names, g)}
    dpose = torch.zeros((1, 6), dtype=torch.float64, device=dev)
    out = r.forward(*g, T, check=True)  # sizes the instance capacity (host sync, untimed)
    st = r.stats()
    Nv, M = int(st.n_visible), int(st.n_instances)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step(reuse=False):
        # the metric's form: the backward recomputes projection and tile lists
        for t in grads.values():
            t.zero_()
        dpose.zero_()
        r.forward(*g, T, out=out, check=False)
        r.backward(*g, T, out, g_rgb, g_d, None, grads=grads, dpose=dpose, reuse=reuse)

    for _ in range(max(3, a.warmup)):
        step()
    torch.cuda.synchronize()
    C.check(r.stats().status, "warm-up render")

    def timed(fn, k, flush_l2=True):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for e0, e1 in evs:
            if flush_l2:
                flush.fill_(1.0)
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(uuid) if rank == 0 else None
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = C.vpgs_launch_count()
    t_wall0 = time.time()
    ms = timed(step, a.steps)
    t_wall1 = time.time()
    launches = C.vpgs_launch_count() - l0
    ms_step = max_over_ranks(sum(ms) / len(ms), dev)
    if world > 1:
        dist.barrier()
    C.check(r.stats().status, "timed renders")
    value_eager = P * world / (ms_step * 1e-3) / 1e6
    eager = {"value": value_eager, "ms_per_step": ms_step, "ms_p50": statistics.median(ms)}
    # the same step captured once into a CUDA graph and replayed (the library
    # is capturable: no host sync, device-side counts); L2 flushed between replays
    graph_ms = None
    try:
        if a.no_extras:
            raise RuntimeError("skipped (--no-extras)")
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            step()
        for _ in range(3):
            cg.replay()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t_wall0g = time.time()
        g_ms = timed(cg.replay, a.steps)
        t_wall1 = time.time()
        graph_ms = max_over_ranks(sum(g_ms) / len(g_ms), dev)
        C.check(r.stats().status, "graph replays")
    except Exception as exc:  # reported; the eager number stands
        eager["graph_error"] = repr(exc)[:200]
    reuse_ms = None
    if not a.no_extras:
        # opt-in variant (not the metric's form): the backward reuses the forward's lists
        reuse_ms = max_over_ranks(statistics.fmean(timed(lambda: step(reuse=True), min(a.steps, 100))), dev)
        C.check(r.stats().status, "reuse renders")
    if sampler:
        time.sleep(0.2)
        sampler.stop()
    if graph_ms is not None and graph_ms < ms_step:
        ms_step_head, launch = graph_ms, "cuda_graph"
        t_wall0 = t_wall0g  # clocks of the region that gives the headline number
    else:
        ms_step_head, launch = ms_step, "eager"
    value = P * world / (ms_step_head * 1e-3) / 1e6

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step_head, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if a.scale == 1.0 else f"room scaled x{a.scale}",
                       "n_gaussians": sc.n, "width": W, "height": H,
                       "visible": Nv, "instances": M, "tile": a.tile,
                       "persistent_ctas_per_sm": a.persistent,
                       "step": "forward (projection, binning, compositing) + backward recomputing "
                               "projection and tile lists; all Gaussian and pose gradients",
                       "l2": "256 MiB buffer written between timed steps (inputs 56 MB < L2)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "launch": launch},
            "eager": eager, "cuda_graph": {"ms_per_step": graph_ms,
                                           "value": P * world / (graph_ms * 1e-3) / 1e6 if graph_ms else None},
            "gpu_launches": int(launches)}
    if reuse_ms is not None:
        line["reuse_binning"] = {"ms_per_step": reuse_ms, "value": P * world / (reuse_ms * 1e-3) / 1e6,
                                 "note": "opt-in VPGS_RENDER_REUSE_BINNING: backward takes the forward's tile "
                                         "lists (eager; not the metric's recompute form)"}
    if sampler:
        line["clocks"] = sampler.summary(t_wall0, t_wall1)

    if not a.no_extras:
        # per-kernel live timing (CUDA events on the launching stream), same steps again
        C.vpgs_profile_enable(1)
        timed(step, min(a.steps, 50))
        C.vpgs_profile_enable(0)
        prof = C.profile_collect()
        kern = {k: {"launches": n, "ms_total": t, "ms_avg": t / n} for k, (n, t) in prof.items()}
        tot = sum(v["ms_total"] for v in kern.values())
        for v in kern.values():
            v["share"] = v["ms_total"] / tot if tot else 0.0
        top = max(kern, key=lambda k: kern[k]["ms_total"])
        peak, peak_src = _peaks()
        ab = algorithmic_bytes(top, sc.n, Nv, M, P)
        pairs_eval = int(out["n_iter"].to(torch.int64).sum())
        pairs_blend = int(out["n_contrib"].to(torch.int64).sum())
        # tile-level SIMD waste: a tile walks its list as far as its slowest pixel
        ni = out["n_iter"][0].to(torch.float32)
        ph, pw = (-H) % th, (-W) % tw
        nip = torch.nn.functional.pad(ni, (0, pw, 0, ph))
        tmax = torch.nn.functional.max_pool2d(nip[None, None], (th, tw))[0, 0]
        line["config"]["pairs_useful"] = pairs_eval
        line["config"]["pairs_tile_walk"] = int(tmax.sum().item()) * tw * th
        if top in ("composite_fwd", "composite_bwd"):
            blend = PAIR_FLOPS["blend_fwd" if top == "composite_fwd" else "blend_bwd"]
            flops = pairs_eval * PAIR_FLOPS["eval"] + pairs_blend * blend
            mhz = (line.get("clocks") or {}).get("sm_mhz") or 2070.0
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            pk = alu_peak_tflops(mhz, sms)
            ach = flops / (kern[top]["ms_avg"] * 1e-3) / 1e12
            line["roofline"] = {"kernel": top, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                "frac": ach / pk, "traffic": ncu_traffic(top),
                                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz",
                                "algorithmic_flops": flops, "pairs_evaluated": pairs_eval,
                                "pairs_blended": pairs_blend,
                                "hbm": {"algorithmic_bytes": ab,
                                        "achieved_gbs": ab / (kern[top]["ms_avg"] * 1e-3) / 1e9 if ab else None,
                                        "peak_gbs": peak, "peak_source": peak_src}}
        elif ab is not None:
            achieved = ab / (kern[top]["ms_avg"] * 1e-3) / 1e9
            line["roofline"] = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peak,
                                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                                "algorithmic_bytes": ab, "traffic": ncu_traffic(top)}
        else:
            line["roofline"] = {"kernel": top, "bound": "hbm", "achieved": None, "peak": peak,
                                "unit": "GB/s", "frac": None, "traffic": None}
        # the metric's "% HBM roofline": the whole step's algorithmic bytes over its time
        floor = step_floor_bytes(sc.n, Nv, M, P)
        line["roofline"]["step_hbm"] = {
            "algorithmic_bytes": floor, "ms_per_step": ms_step_head,
            "achieved_gbs": floor / (ms_step_head * 1e-3) / 1e9, "peak_gbs": peak, "peak_source": peak_src,
            "frac": floor / (ms_step_head * 1e-3) / 1e9 / peak,
            "formula": "168 N + 240 Nv + 192 M + 56 P bytes (one-pass-sort floor of the fwd+bwd recompute step)"}
        line["kernels"] = {k: {"launches": v["launches"] // min(a.steps, 50), "ms_avg": round(v["ms_avg"], 5),
                               "share": round(v["share"], 4)} for k, v in sorted(kern.items(),
                                                                                  key=lambda kv: -kv[1]["ms_total"])}
    if not a.no_extras and not a.no_rows:
        # end to end through the public API with host buffers
        pin = lambda t: t.detach().cpu().pin_memory()  # noqa: E731
        h_in = [pin(t) for t in g] + [pin(T), pin(g_rgb), pin(g_d)]
        h_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()
                 if k in ("rgb", "depth", "alpha")}
        h_gr = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in grads.items()}
        h_pose = torch.empty((1, 6), dtype=torch.float64).pin_memory()
        d_in = g + [T, g_rgb, g_d]

        side = torch.cuda.Stream(device=dev)
        n_fwd = len(g) + 1  # the Gaussians and the pose feed the forward

        def e2e_step():
            # every copy of the step stays inside it: the upstream gradients
            # (needed by the backward only) go in beside the forward, the
            # images come back beside the backward
            cur = torch.cuda.current_stream()
            for d_t, h_t in zip(d_in[:n_fwd], h_in[:n_fwd]):
                d_t.copy_(h_t, non_blocking=True)
            side.wait_stream(cur)
            with torch.cuda.stream(side):
                for d_t, h_t in zip(d_in[n_fwd:], h_in[n_fwd:]):
                    d_t.copy_(h_t, non_blocking=True)
                grads_in = torch.cuda.Event()
                grads_in.record(side)
            for t in grads.values():
                t.zero_()
            dpose.zero_()
            r.forward(*g, T, out=out, check=False)
            side.wait_stream(cur)
            with torch.cuda.stream(side):
                for k in h_out:
                    h_out[k].copy_(out[k], non_blocking=True)
            cur.wait_event(grads_in)
            r.backward(*g, T, out, g_rgb, g_d, None, grads=grads, dpose=dpose)
            for k in h_gr:
                h_gr[k].copy_(grads[k], non_blocking=True)
            h_pose.copy_(dpose, non_blocking=True)
            cur.wait_stream(side)

        ms_e = timed(e2e_step, min(a.steps, 50))
        e_ms = sum(ms_e) / len(ms_e)
        h2d = sum(t.numel() * t.element_size() for t in h_in)
        d2h = sum(t.numel() * t.element_size() for t in list(h_out.values()) + list(h_gr.values())) + 48
        line["e2e"] = {"value": P * world / (e_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": e_ms,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        # coarse tracking: 50 pose-only iterations, eager vs one captured CUDA graph
        for key, fn in (("tracking", lambda: tracking_rows(sc, g, dev)), ("decode", lambda: decode_rows(dev)),
                        ("batched_keyframes", lambda: batched_rows(dev)), ("fusion", lambda: fusion_rows(dev)),
                        ("mapping", lambda: mapping_rows(sc, g, dev)), ("icp", lambda: icp_rows(dev)),
                        ("anchors", lambda: anchor_rows(dev))):
            try:
                line[key] = fn()
            except Exception as exc:  # reported, not fatal
                line[key] = {"error": repr(exc)[:300]}
    T_icp = line["icp"].pop("_T", None) if isinstance(line.get("icp"), dict) else None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(sc, a.cpu_rows)
        if "icp" in line:
            try:
                line["cpu_baseline"]["icp"] = icp_oracle(T_icp)
            except Exception as exc:  # reported, not fatal
                line["cpu_baseline"]["icp"] = {"error": repr(exc)[:300]}
        if "anchors" in line:
            try:
                line["cpu_baseline"]["anchors"] = anchor_oracle()
            except Exception as exc:  # reported, not fatal
                line["cpu_baseline"]["anchors"] = {"error": repr(exc)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _time_ms(fn, reps=20):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def decode_rows(dev):
    """Anchor decode of 100,000 street anchors: FP32 FMA vs BF16 tensor cores, fwd and bwd."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.decode import Decoder
    sc = scenes.street_anchors()
    t = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device=dev).contiguous()  # noqa: E731
    anchors, feats, scal, offs = t(sc.anchors), t(sc.features), t(sc.scaling), t(sc.offsets)
    params = t(np.concatenate([np.asarray(p, np.float32).reshape(-1)
                               for name in ("opacity", "color", "cov") for p in sc.mlp[name]]))
    T = t(sc.camera.T_cw[0], torch.float64)
    res = {"anchors": sc.n, "k": sc.k,
           "timing": "library calls on preallocated buffers, no host sync inside the timed loop"}
    for name, bf in (("fp32", False), ("bf16", True)):
        d = Decoder(sc.k, bf16=bf, device=dev)
        out = d.forward(anchors, feats, scal, offs, params, sc.camera, T)
        grads = {k: torch.ones_like(out[k]) for k in ("means", "scales", "quats", "opacities", "colors")}
        gres = d.backward(anchors, feats, scal, offs, params, sc.camera, T, out, grads)
        fwd_ms = _time_ms(lambda: d.forward(anchors, feats, scal, offs, params, sc.camera, T, out=out, sync=False))
        bwd_ms = _time_ms(lambda: d.backward(anchors, feats, scal, offs, params, sc.camera, T, out, grads, res=gres))
        # per-kernel device times (CUDA events on the launching stream)
        C.vpgs_profile_enable(1)
        for _ in range(10):
            d.forward(anchors, feats, scal, offs, params, sc.camera, T, out=out, sync=False)
            d.backward(anchors, feats, scal, offs, params, sc.camera, T, out, grads, res=gres)
        torch.cuda.synchronize()
        prof = C.profile_collect()
        C.vpgs_profile_enable(0)
        res[name] = {"fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "gaussians_out": out["n"],
                     "anchors_per_s_fwd": sc.n / (fwd_ms * 1e-3),
                     "kernels_us": {k: round(1000 * t / max(n, 1), 1) for k, (n, t) in prof.items()}}
    return res


def mapping_rows(sc, g, dev, steps=20):
    """Mapping step of Sec. III-A on the room frame: render, the full loss L_m
    (Eq. 7-9: L1 + SSIM colour, L1 depth, volume), backward through the renderer
    (recomputing its tile lists) to every Gaussian parameter.  The target is the
    render from the pose perturbed by 2 cm / 1 degree."""
    import torch

    from paper_2505_18992_gb300.loss import MappingLoss
    from paper_2505_18992_gb300.render import Intrinsics, Renderer
    cam = sc.camera
    W, H = cam.width, cam.height
    r = Renderer(Intrinsics(W, H, cam.fx, cam.fy, cam.cx, cam.cy), device=dev)
    T = torch.tensor(cam.T_cw, dtype=torch.float64, device=dev).contiguous()
    T1 = torch.tensor(sc.extra["T_track0"], dtype=torch.float64, device=dev).reshape(1, 4, 4).contiguous()
    tgt = r.forward(*g, T1, check=True)
    t_rgb, t_depth = tgt["rgb"].clone(), tgt["depth"].clone()
    out = r.forward(*g, T, check=True)
    L = MappingLoss(1, W, H)
    names = ("means", "scales", "quats", "opacities", "colors")
    grads = {k: torch.zeros_like(t) for k, t in zip(names, g)}
    d_rgb = torch.empty_like(out["rgb"])
    d_depth = torch.empty_like(out["depth"])

    def loss_only():
        L(out["rgb"], t_rgb, out["depth"], t_depth, g[1], d_rgb=d_rgb, d_depth=d_depth, d_scales=grads["scales"])

    def step():
        for t in grads.values():
            t.zero_()
        r.forward(*g, T, out=out, check=False)
        loss_only()
        r.backward(*g, T, out, d_rgb, d_depth, None, grads=grads)

    loss_ms = _time_ms(loss_only, steps)
    step_ms = _time_ms(step, steps)
    lv = L.loss.cpu().numpy()
    P = W * H
    # loss kernels: read rgb + target (24 B/px), write A, B, C (36 B/px); read them
    # with rgb + target again (60 B/px), write the colour gradient (12 B/px); depth
    # terms 12 B/px; volume term 24 B per Gaussian
    loss_bytes = 144 * P + 12 * P + 24 * sc.n
    return {"loss_ms": loss_ms, "loss_hbm_gbs": loss_bytes / (loss_ms * 1e-3) / 1e9,
            "loss_algorithmic_bytes": loss_bytes, "step_ms": step_ms,
            "step_mpix_s": P / (step_ms * 1e-3) / 1e6,
            "terms": {"L_m": float(lv[0]), "L_c": float(lv[1]), "L_SSIM": float(lv[2]), "L_d": float(lv[3]),
                      "L_vol": float(lv[4])}}


def batched_rows(dev, steps=10):
    """8 keyframes of a 2M-Gaussian submap: one 8-view call vs 8 one-view calls (fwd+bwd)."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.render import Intrinsics, Renderer
    sc = scenes.batched_keyframes()
    cam = sc.camera
    g = [torch.tensor(x, device=dev).contiguous() for x in sc.arrays()]
    T = torch.tensor(cam.T_cw, dtype=torch.float64, device=dev).contiguous()
    V, H, W = cam.n_views, cam.height, cam.width
    intr = Intrinsics(W, H, cam.fx, cam.fy, cam.cx, cam.cy)
    grads = {k: torch.zeros_like(x) for k, x in zip(("means", "scales", "quats", "opacities", "colors"), g)}
    rb = Renderer(intr, n_views=V, device=dev)
    outb = rb.forward(*g, T, check=True)
    gb = torch.full((V, 3, H, W), 1.0 / (3 * H * W), device=dev)
    dpb = torch.zeros((V, 6), dtype=torch.float64, device=dev)

    def batched():
        rb.forward(*g, T, out=outb, check=False)
        rb.backward(*g, T, outb, gb, None, None, grads=grads, dpose=dpb)

    r1 = Renderer(intr, n_views=1, device=dev)
    Ts = [T[v:v + 1].contiguous() for v in range(V)]
    outs = [r1.forward(*g, Tv, check=True) for Tv in Ts]
    g1 = gb[:1].contiguous()
    dp1 = torch.zeros((1, 6), dtype=torch.float64, device=dev)

    def separate():
        for Tv, o in zip(Ts, outs):
            r1.forward(*g, Tv, out=o, check=False)
            r1.backward(*g, Tv, o, g1, None, None, grads=grads, dpose=dp1)

    mb = _time_ms(batched, steps)
    ms = _time_ms(separate, steps)
    px = V * H * W
    # per-kernel device times of a batched call (CUDA events on the launching stream)
    C.vpgs_profile_enable(1)
    for _ in range(3):
        batched()
    torch.cuda.synchronize()
    prof = C.profile_collect()
    C.vpgs_profile_enable(0)
    row = {"views": V, "gaussians": sc.n, "width": W, "height": H,
           "batched_ms": mb, "separate_ms": ms, "batched_mpix_s": px / (mb * 1e-3) / 1e6,
           "separate_mpix_s": px / (ms * 1e-3) / 1e6,
           "kernels_us_per_call": {k: round(1000 * t / 3, 1) for k, (n, t) in prof.items()}}
    # launch shape picked by the autotuner (tile shape x persistent CTAs x views per call)
    from paper_2505_18992_gb300 import autotune
    del outb, outs
    torch.cuda.empty_cache()
    shapes = autotune.candidates(V, tiles=((8, 16), (16, 16), (16, 8), (8, 8)), persistent=(0, 4),
                                 views_per_call=(8, 4, 1))
    best, timings = autotune.tune(g, T, intr, gb, shapes=shapes, steps=3)
    row["autotuned"] = {"shape": {"tile": f"{best.tile_w}x{best.tile_h}", "persistent_ctas": best.persistent_ctas,
                                  "views_per_call": best.views_per_call},
                        "ms": timings[best], "mpix_s": px / (timings[best] * 1e-3) / 1e6,
                        "candidates": len(timings),
                        "default_ms": timings.get(autotune.LaunchShape(16, 16, 0, V))}
    return row


FUSION_SUBMAPS, FUSION_PAIR = 16, (7, 8)


def fusion_rows(dev, iters=10):
    """Submap fusion by distillation (Sec. III-C, Eq. 14) as an optimisation loop,
    on a 1 km street held as 16 submaps resident on the GPU: submap i holds
    50,000 anchors (k = 10: 500,000 neural Gaussians, 8M in all) over
    [62.5 i - 10, 62.5 (i + 1)] m, so neighbours overlap by 10 m, each with its
    own BF16 decoder.  Every submap is decoded once from a camera at its
    centre.  The loop then works on submaps 7 and 8, with m = 4 keyframes in
    their overlap at 1920x1080: each iteration decodes both, renders the
    keyframes (one 4-view call per submap), takes the squared distillation loss
    between the two renders, runs the render backward (recomputing its tile
    lists) and the decoder backward of both submaps, and takes an Adam step on
    each submap's anchor features and MLP weights."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.decode import Decoder
    from paper_2505_18992_gb300.fusion import Adam, DistillLoss
    from paper_2505_18992_gb300.render import Intrinsics, Renderer
    torch.cuda.reset_peak_memory_stats(dev)
    t = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device=dev).contiguous()  # noqa: E731
    # the whole street, resident: anchors, features, scalings, offsets, decoder
    # weights and the decoded Gaussians of every submap
    street = []
    for i in range(FUSION_SUBMAPS):
        x0 = 62.5 * i - (10.0 if i > 0 else 0.0)
        sc = scenes.street_anchors(n_anchors=50_000, length=62.5 * (i + 1) - x0, x0=x0, seed=20 + i, width=1920,
                                   height=1080, f=1000.0, cam_x=x0 + 2.0, mlp_seed=7)
        params = t(np.concatenate([np.asarray(p, np.float32).reshape(-1)
                                   for name in ("opacity", "color", "cov") for p in sc.mlp[name]]))
        inp = (t(sc.anchors), t(sc.features), t(sc.scaling), t(sc.offsets), params)
        d = Decoder(sc.k, bf16=True, device=dev)
        out = d.forward(*inp, sc.camera, t(sc.camera.T_cw[0], torch.float64))
        street.append({"sc": sc, "inp": inp, "d": d, "out": out})
    resident = [int(s["out"]["n_dev"].item()) for s in street]
    subs = [street[j]["sc"] for j in FUSION_PAIR]
    # keyframes in the 10 m overlap, facing the facade, so both submaps are in view
    kfs = np.stack([scenes.look_at([x, 0.0, 1.7], [x, 10.0, 1.7], [0, 0, 1]) for x in (491.5, 494.0, 496.0, 498.5)])
    m = len(kfs)
    T = t(kfs, torch.float64)
    cam = subs[0].camera
    W, H = cam.width, cam.height
    r = Renderer(Intrinsics(W, H, cam.fx, cam.fy, cam.cx, cam.cy), n_views=m, device=dev)
    dist = DistillLoss(m, W, H)
    state = []
    for j in FUSION_PAIR:
        sc, inp, d = street[j]["sc"], street[j]["inp"], street[j]["d"]
        sc.camera.T_cw = kfs[:1]  # decode culls against the first keyframe
        feats, params = inp[1], inp[4]
        out = d.forward(*inp, sc.camera, T[0], out=street[j]["out"])
        res = {"features": torch.zeros_like(feats), "offsets": torch.zeros_like(inp[3]),
               "scaling": torch.zeros_like(inp[2]), "params": torch.zeros_like(params)}
        opts = [Adam(feats, res["features"], lr=1e-3), Adam(params, res["params"], lr=1e-4)]
        img = r.alloc_images()
        grads = {k: torch.zeros_like(out[k]) for k in ("means", "scales", "quats", "opacities", "colors")}
        state.append({"d": d, "inp": inp, "sc": sc, "out": out, "res": res, "opts": opts, "img": img,
                      "grads": grads, "g_rgb": torch.empty_like(img["rgb"]), "g_d": torch.empty_like(img["depth"])})
    for st in state:  # size the render workspace once (host sync, untimed)
        o = st["out"]
        r.forward(o["means"], o["scales"], o["quats"], o["opacities"], o["colors"], T, n_dev=o["n_dev"],
                  out=st["img"], check=True)
    P = W * H

    def iteration():
        for st in state:
            o = st["d"].forward(*st["inp"], st["sc"].camera, T[0], out=st["out"], sync=False)
            r.forward(o["means"], o["scales"], o["quats"], o["opacities"], o["colors"], T, n_dev=o["n_dev"],
                      out=st["img"], check=False)
        a, b = state
        dist(a["img"]["rgb"], b["img"]["rgb"], a["img"]["depth"], b["img"]["depth"], a["g_rgb"], b["g_rgb"],
             a["g_d"], b["g_d"])
        for st in state:
            o, gr = st["out"], st["grads"]
            for v in gr.values():
                v.zero_()
            r.backward(o["means"], o["scales"], o["quats"], o["opacities"], o["colors"], T, st["img"], st["g_rgb"],
                       st["g_d"], None, grads=gr, n_dev=o["n_dev"])
            st["d"].backward(*st["inp"], st["sc"].camera, T[0], o, gr, res=st["res"])
            for opt in st["opts"]:
                opt.step()

    losses = []
    iteration()
    torch.cuda.synchronize()
    losses.append(float(dist.loss[0]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        iteration()
    e1.record()
    torch.cuda.synchronize()
    losses.append(float(dist.loss[0]))
    ms = e0.elapsed_time(e1) / iters
    # per-kernel device times of an iteration (CUDA events on the launching stream)
    C.vpgs_profile_enable(1)
    for _ in range(2):
        iteration()
    torch.cuda.synchronize()
    prof = C.profile_collect()
    C.vpgs_profile_enable(0)
    return {"submaps_resident": FUSION_SUBMAPS, "anchors_resident": sum(s["sc"].n for s in street),
            "gaussian_capacity_resident": sum(s["sc"].n * s["sc"].k for s in street),
            "gaussians_decoded_per_submap": resident, "fused_pair": list(FUSION_PAIR), "keyframes": m,
            "width": W, "height": H,
            "gaussians_decoded": [int(st["out"]["n_dev"].item()) for st in state],
            "ms_per_iteration": ms, "mpix_s": 2 * m * P / (ms * 1e-3) / 1e6,
            "loss": {"first": losses[0], f"after_{iters + 1}": losses[1]},
            "peak_hbm_gb": torch.cuda.max_memory_allocated(dev) / 1e9,
            "kernels_us_per_iteration": {k: round(1000 * t / 2, 1) for k, (n, t) in prof.items()}}


def icp_rows(dev, reps=20):
    """Fine tracking by voxel-hash ICP (Sec. III-B, Eq. 10-12): one 64-beam
    LiDAR sweep (114k points) of a 200 m street registered against a map of
    1M Gaussian means in 1 m voxels; double downsampling at 0.5 m and 1.5 m,
    tau = 1 m, sigma = 0.3, up to 50 Gauss-Newton steps with eps = 1e-4.
    Times the map build and one registration, eager and as one CUDA graph."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.icp import ICP, VoxelMap
    sc = scenes.street_lidar()
    mp = torch.tensor(sc.map_points, device=dev).contiguous()
    scan = torch.tensor(sc.scan, device=dev).contiguous()
    T0 = torch.tensor(sc.T_init, dtype=torch.float64, device=dev).contiguous()
    vmap = VoxelMap(mp, 1.0)
    build_ms = _time_ms(lambda: vmap.rebuild(), reps)
    icp = ICP(len(sc.scan), 0.5, 1.5, 1.0, 0.3, iterations=50, eps=1e-4)
    T = T0.clone()

    def reg():
        T.copy_(T0)
        icp.register(vmap, scan, T)

    eager_ms = _time_ms(reg, reps)
    rep = icp.report()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        reg()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        reg()
    graph_ms = _time_ms(g.replay, reps)
    T_gpu = T.cpu().numpy()
    C.vpgs_profile_enable(1)
    for _ in range(5):
        reg()
    torch.cuda.synchronize()
    prof = C.profile_collect()
    C.vpgs_profile_enable(0)
    return {"map_points": len(sc.map_points), "scan_points": len(sc.scan), "n_source": rep["n_source"],
            "iterations": rep["iterations"], "stop": rep["stop"], "n_corr": rep["n_corr"],
            "map_build_ms": build_ms, "register_ms_eager": eager_ms, "register_ms_graph": graph_ms,
            "scans_per_s_graph": 1e3 / graph_ms,
            "kernels_us_per_registration": {k: round(1000 * t / 5, 1) for k, (n, t) in prof.items()},
            "trans_err_m_start": float(np.linalg.norm(sc.T_init[:3, 3] - sc.T_true[:3, 3])),
            "trans_err_m": float(np.linalg.norm(T_gpu[:3, 3] - sc.T_true[:3, 3])), "_T": T_gpu}


def icp_oracle(T_gpu):
    """The FP64 oracle's registration of the ICP row's scan (one host core), and
    its distance to the GPU's pose."""
    import importlib
    import time

    from paper_2505_18992_gb300 import scenes
    oracle = importlib.import_module("oracle.icp")
    sc = scenes.street_lidar()
    t0 = time.perf_counter()
    ref = oracle.icp(sc.scan, sc.map_points, sc.T_init, 0.5, 1.5, 1.0, 0.3, iterations=50, eps=1e-4)
    ms = (time.perf_counter() - t0) * 1e3
    out = {"value": ms, "unit": "ms per registration", "cores": 1, "kind": "oracle",
           "sample": "one full registration of the ICP row's scan (cKDTree build included)",
           "iterations": ref["iterations"]}
    if T_gpu is not None:
        out["max_abs_dT_vs_gpu"] = float(np.abs(T_gpu - ref["T"]).max())
    return out


SPAWN = dict(tau_alpha=0.5, delta_depth=0.1, voxel=0.05, rho=0.04, map_voxel=0.05, max_samples=50_000)
ANCHOR_UPDATE = dict(tau_g=2.5e-3, tau_o=0.3, grow_voxel=0.2)


def anchor_rows(dev, reps=20):
    """Submap expansion and anchor maintenance (Sec. III-A): statistics of one
    training step of 100,000 street anchors (500,000 decoded Gaussians),
    pruning + growth from them, and spawning from one 1200x680 room keyframe
    (142k masked pixels, 50,000 samples, 5 cm voxels, rho = 4 cm against
    300,000 Gaussian means)."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.anchors import AnchorStats, AnchorUpdate, Spawner
    from paper_2505_18992_gb300.icp import VoxelMap
    t = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device=dev).contiguous()  # noqa: E731
    stp = scenes.anchor_step()
    A, N = len(stp.anchors), len(stp.src_index)
    src, grads, opac, vis, means = (t(stp.src_index, torch.int32), t(stp.grads), t(stp.opacities),
                                    t(stp.visible, torch.int32), t(stp.means))
    st = AnchorStats(A, device=dev)
    acc_ms = _time_ms(lambda: st.accumulate(stp.k, src, grads, opac, vis), reps)
    st.reset()
    st.accumulate(stp.k, src, grads, opac, vis)
    amap = VoxelMap(t(stp.anchors), ANCHOR_UPDATE["grow_voxel"])
    amap_ms = _time_ms(lambda: amap.rebuild(), reps)
    up = AnchorUpdate(A, N, device=dev, **ANCHOR_UPDATE)
    upd_ms = _time_ms(lambda: up(st, stp.k, src, means, amap), reps)
    keep, grown = up.results()
    fr = scenes.keyframe_spawn()
    gmap = VoxelMap(t(fr.gauss_means), SPAWN["map_voxel"])
    sp = Spawner(fr.width, fr.height, fr.fx, fr.fy, fr.cx, fr.cy, SPAWN["tau_alpha"], SPAWN["delta_depth"],
                 SPAWN["voxel"], SPAWN["rho"], SPAWN["max_samples"], device=dev)
    ins = (t(fr.alpha), t(fr.depth), t(fr.depth_in), t(fr.T_cw, torch.float64))
    spawn_ms = _time_ms(lambda: sp(*ins, gmap), reps)
    new, _ = sp.results()
    C.vpgs_profile_enable(1)
    for _ in range(5):
        st.accumulate(stp.k, src, grads, opac, vis)
        up(st, stp.k, src, means, amap)
        sp(*ins, gmap)
    torch.cuda.synchronize()
    prof = C.profile_collect()
    C.vpgs_profile_enable(0)
    acc_bytes = N * (4 + 12 + 4 + 4)
    return {"anchors": A, "decoded_gaussians": N, "stats_accumulate_ms": acc_ms,
            "stats_accumulate_gbs": acc_bytes / (acc_ms * 1e-3) / 1e9,
            "anchor_map_build_ms": amap_ms, "prune_grow_ms": upd_ms, "kept": int(len(keep)), "grown": int(len(grown)),
            "spawn_ms": spawn_ms, "spawn_pixels": fr.width * fr.height, "spawned": int(len(new)),
            "kernels_us": {k: round(1000 * tt / 5, 1) for k, (n, tt) in prof.items()
                           if k.startswith(("anchor", "spawn"))}}


def anchor_oracle():
    """The FP64 oracle on the anchor row's inputs (one host core): statistics,
    pruning + growth and spawning."""
    import importlib
    import time

    from paper_2505_18992_gb300 import scenes
    O = importlib.import_module("oracle.anchors")
    stp = scenes.anchor_step()
    fr = scenes.keyframe_spawn()
    t0 = time.perf_counter()
    s = O.accumulate_stats(O.new_stats(len(stp.anchors)), stp.src_index, stp.k, stp.grads, stp.opacities, stp.visible)
    t1 = time.perf_counter()
    O.prune(s, ANCHOR_UPDATE["tau_o"])
    O.grow(s, stp.src_index, stp.k, stp.means, ANCHOR_UPDATE["tau_g"], ANCHOR_UPDATE["grow_voxel"], stp.anchors)
    t2 = time.perf_counter()
    new, _ = O.spawn(fr.alpha, fr.depth, fr.depth_in, fr.fx, fr.fy, fr.cx, fr.cy, fr.T_cw, SPAWN["tau_alpha"],
                     SPAWN["delta_depth"], SPAWN["max_samples"], SPAWN["voxel"], SPAWN["rho"], fr.gauss_means)
    t3 = time.perf_counter()
    return {"value": (t3 - t0) * 1e3, "unit": "ms (statistics + prune/grow + spawn)", "cores": 1, "kind": "oracle",
            "sample": "the full anchor row workload", "stats_ms": (t1 - t0) * 1e3, "prune_grow_ms": (t2 - t1) * 1e3,
            "spawn_ms": (t3 - t2) * 1e3, "spawned": int(len(new))}


def tracking_rows(sc, g, dev):
    import torch

    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.render import Intrinsics, Renderer
    from paper_2505_18992_gb300.tracking import Tracker
    cam = sc.camera
    r = Renderer(Intrinsics(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy), device=dev)
    T_true = torch.tensor(cam.T_cw, dtype=torch.float64, device=dev).contiguous()
    ref = r.forward(*g, T_true, check=True)
    tgt_rgb, tgt_d = ref["rgb"].clone(), ref["depth"].clone()
    T0 = torch.tensor(sc.extra["T_track0"], dtype=torch.float64, device=dev).contiguous()
    T = T0.clone()
    tr = Tracker(r, g, T, tgt_rgb, tgt_d, lr=(2e-3, 2e-3))  # the backward reuses the forward's tile lists
    tr.prepare()
    tr.iteration()  # loads every kernel module once before timing
    iters = 50
    tr.reset(T0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tr.run_eager(iters)
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    err0 = float(torch.linalg.norm(T0[0, :3, 3] - T_true[0, :3, 3]))
    err_eager = float(torch.linalg.norm(T[0, :3, 3] - T_true[0, :3, 3]))
    # per-kernel device times of an iteration (CUDA events on the launching stream)
    tr.reset(T0)
    C.vpgs_profile_enable(1)
    tr.run_eager(10)
    torch.cuda.synchronize()
    prof = C.profile_collect()
    C.vpgs_profile_enable(0)
    kernels_us = {k: round(1000 * t / max(n, 1), 1) for k, (n, t) in prof.items()}
    tr.reset(T0)
    tr.capture(iters)
    tr.reset(T0)
    torch.cuda.synchronize()
    e0.record()
    tr.replay()
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    err_graph = float(torch.linalg.norm(T[0, :3, 3] - T_true[0, :3, 3]))
    # the same loop with the backward recomputing projection and tile lists
    r2 = Renderer(Intrinsics(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy), device=dev)
    T2 = T0.clone()
    tr2 = Tracker(r2, g, T2, tgt_rgb, tgt_d, lr=(2e-3, 2e-3), reuse_binning=False)
    tr2.prepare()
    tr2.iteration()
    tr2.reset(T0)
    tr2.capture(iters)
    tr2.reset(T0)
    torch.cuda.synchronize()
    e0.record()
    tr2.replay()
    e1.record()
    torch.cuda.synchronize()
    rec_ms = e0.elapsed_time(e1)
    err_rec = float(torch.linalg.norm(T2[0, :3, 3] - T_true[0, :3, 3]))
    return {"iters": iters, "eager_ms": eager_ms, "graph_ms": graph_ms,
            "ms_per_iter_graph": graph_ms / iters, "trans_err_m_start": err0,
            "trans_err_m_eager": err_eager, "trans_err_m_graph": err_graph,
            "tile_lists": "the backward of an iteration takes the forward's (one pose per iteration)",
            "recompute_binning": {"graph_ms": rec_ms, "ms_per_iter": rec_ms / iters, "trans_err_m": err_rec,
                                  "pose_gap_m": float(torch.linalg.norm(T2[0, :3, 3] - T[0, :3, 3]))},
            "kernels_us_per_launch": kernels_us}


def run_row(a):
    """One secondary row alone, on cuda:0, printed as JSON."""
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300 import vpgs as C
    from paper_2505_18992_gb300.build import build
    build()
    C.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if a.row in ("tracking", "mapping"):
        sc = scenes.indoor_room()
        g = [torch.tensor(x, device=dev).contiguous() for x in sc.arrays()]
        out = tracking_rows(sc, g, dev) if a.row == "tracking" else mapping_rows(sc, g, dev)
    else:
        out = {"decode": decode_rows, "batched_keyframes": batched_rows, "fusion": fusion_rows,
               "icp": icp_rows, "anchors": anchor_rows}[a.row](dev)
    out.pop("_T", None)
    print(json.dumps({"row": a.row, **out}), flush=True)


def main():
    a = _args()
    if a.row:
        run_row(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
