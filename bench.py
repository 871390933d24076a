"""Throughput benchmark of the rasterizer's training step.

Workload (default): 1,000,000 Gaussians (SH degree 3, clustered synthetic
scene), 8 views of uneven sizes (2x 800x800, 3x 1280x720, 2x 1600x1063,
1x 1920x1080) rendered and backpropagated in one batch: gs_preprocess ->
gs_bin_sort -> gs_render_fwd -> L1 loss -> gs_render_bwd, all in libgs.so.

One JSON line on rank 0.  `value` is device-resident fwd+bwd Mpixel/s over
all ranks; `e2e` is the same step with the scene and targets copied from
pinned host memory and the loss and gradients copied back inside the timed
region.  `--impl reference` times the CPU oracle on a bounded sample of the
same workload instead.  Multi-GPU runs (torchrun) render independent
replicas: there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import tempfile
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s and steps/s at 1M Gaussians; serving p50/p99 ms vs one-at-a-time"
WORKLOAD = ("batched fwd+bwd, 1M Gaussians SH3 (64-cluster + shell scene), 8 views "
            "2x800x800 + 3x1280x720 + 2x1600x1063 + 1x1920x1080, L1 loss; emits colour, d^mid depth, "
            "i_max and per-Gaussian accumulated blending weight")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-culling", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1100)
    ap.add_argument("--serve-runs", type=int, default=3)
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
def dist_setup(gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int) -> float:
    """Max over ranks (timing only)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(local_units: float, local_seconds: float, world: int) -> tuple[float, float]:
    """(total units over ranks, max seconds over ranks): whole-job throughput
    is total / max; each rank processes the same replica workload."""
    return local_units * world, reduce_max(local_seconds, world)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gs_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or p[0] != str(device_index):
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our arm
class Step:
    """Resident state of the batched training step (workspaces reused)."""

    def __init__(self, n: int, seed: int):
        import torch
        from paper_2411_12788_gb300 import raster, scenes
        self.torch, self.raster = torch, raster
        self.scene = scenes.cluster_scene(n, 64, seed=seed, sh_degree=3)
        self.cams = scenes.multiview_cameras()
        tg = scenes.target_images(self.cams, seed=1)
        self.g = raster.GaussianTensors.from_scene(self.scene, "cuda")
        self.target = torch.as_tensor(np.concatenate([t.reshape(-1) for t in tg])).cuda()
        self.plan = raster.make_plan(n, self.cams)
        self.cfg = raster.make_config(flags=raster._lib.GS_FLAG_ZERO_ACCUM)
        self.pre_ws = torch.empty(raster.preprocess_workspace_size(self.plan), dtype=torch.uint8, device="cuda")
        self.sort_ws = torch.empty(0, dtype=torch.uint8, device="cuda")
        # the step emits colour, depth, i_max (forward) and the accumulated
        # blending weight I_i, which the backward pass collects as it replays
        # every blended entry
        self.outs = raster.alloc_outputs(self.plan, "cuda", want=("image", "final_T", "n_contrib", "depth",
                                                                  "imax"))
        self.loss = torch.zeros(1, device="cuda")
        self.dL = torch.empty_like(self.outs["image"])
        self.grads = raster.alloc_grads(self.g)
        self.grads["weight_sum"] = torch.zeros(int(self.plan.n_items), device="cuda")
        self.pixels = int(self.plan.total_pixels)

    def run(self, mask=None):
        r = self.raster
        r.preprocess(self.plan, self.g.struct(), self.cfg, self.pre_ws, mask)
        need = r.bin_sort_workspace_size(self.plan)
        if self.sort_ws.numel() < need:
            self.sort_ws = self.torch.empty(int(need * 1.1), dtype=self.torch.uint8, device="cuda")
        r.bin_sort(self.plan, self.pre_ws, self.sort_ws)
        r.render_fwd(self.plan, self.cfg, self.pre_ws, self.sort_ws, self.outs)
        r.loss_l1(self.outs["image"], self.target, self.loss, self.dL)
        r.render_bwd(self.plan, self.g.struct(), self.cfg, self.pre_ws, self.sort_ws, self.dL,
                     self.outs["image"], self.outs["n_contrib"], self.grads)


def kernel_times(collect=True) -> dict:
    from paper_2411_12788_gb300 import _lib
    import ctypes as C
    arr = (_lib.KernelTime * 64)()
    k = _lib.lib().gs_timing_collect(arr, 64)
    out = {}
    for i in range(min(k, 64)):
        out[arr[i].name.decode()] = {"ms": arr[i].ms, "launches": int(arr[i].launches)}
    return out


# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) at this workload,
# valid while the kernel's source file is the one profiled (its SHA-256) and the workload has the same number
# of tile entries; otherwise the traffic is reported as null.
PROFILED_TRAFFIC = {
    "render_bwd": {"bytes": 594.82e6, "entries": 79448137, "source": "paper_2411_12788_gb300/csrc/render.cu",
                   "sha256": "022f3893b1ac2df820a6f7bb1719c7874117dec52fe852828fbb15647ed631f6",
                   "profile": "profiles/render_bwd_1M_8views.md"},
}


def profiled_traffic(name: str, entries: int):
    import hashlib
    rec = PROFILED_TRAFFIC.get(name)
    if rec is None or rec["entries"] != entries:
        return None
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()
    except OSError:
        return None
    return rec["bytes"] if sha == rec["sha256"] else None


def visible_items(st: "Step") -> int:
    """Items with at least one touched tile in the step's preprocess
    workspace (counted on the device)."""
    import ctypes as C
    from paper_2411_12788_gb300 import _lib
    if getattr(st, "_visible", None) is not None:
        return st._visible
    v = _lib.PreprocessView()
    _lib.lib().gs_inspect_preprocess(C.byref(st.plan), C.c_void_p(st.pre_ws.data_ptr()), C.byref(v))
    off = v.tiles - st.pre_ws.data_ptr()
    I = int(st.plan.n_items)
    tiles = st.pre_ws[off: off + 4 * I].view(st.torch.int32)
    st._visible = int((tiles > 0).sum().item())
    return st._visible


def all_rooflines(kt: dict, st: "Step", peaks: dict, clocks: dict) -> dict:
    """Roofline of every kernel with an algorithmic figure (same units as the
    dominant kernel's)."""
    out = {}
    for name in kt:
        r = roofline(kt, st, 0, peaks, clocks, name=name)
        if r.get("achieved"):
            out[name] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    return out


def roofline(kt: dict, st: "Step", steps: int, peaks: dict, clocks: dict, name: str | None = None) -> dict:
    """Roofline of the dominant kernel (largest share of the timed region),
    or of `name`."""
    name = name or max(kt, key=lambda k: kt[k]["ms"])
    ms = kt[name]["ms"] / max(1, kt[name]["launches"])
    E = int(st.plan.n_entries)
    torch = st.torch
    if name in ("render_bwd", "render_fwd"):
        # ALU-bound.  Units: the (pixel, entry) pairs the sequential per-pixel
        # algorithm evaluates up to the last blended entry (sum of n_contrib);
        # the blended ones cost the full per-pair figure, the skipped ones
        # (alpha < 1/255) only the offsets and the exponent
        pc = pair_counts(st)
        full = BWD_FLOPS_PER_BLEND if name == "render_bwd" else FWD_FLOPS_PER_BLEND
        flops = pc["blended"] * full + pc["skipped"] * FLOPS_PER_SKIP
        sms = st.torch.cuda.get_device_properties(st.torch.cuda.current_device()).multi_processor_count
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        ach = flops / (ms * 1e-3) / 1e12
        traffic = profiled_traffic(name, E)
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic,
                "traffic_note": (f"DRAM bytes per launch from ncu ({PROFILED_TRAFFIC[name]['profile']}); "
                                 f"algorithmic {flops / traffic:.0f} flop per byte moved") if traffic else None,
                "units": {"blended_pairs_per_launch": pc["blended"], "skipped_pairs_per_launch": pc["skipped"],
                          "flops_per_blended_pair": full, "flops_per_skipped_pair": FLOPS_PER_SKIP,
                          "flops_per_launch": flops},
                "peak_note": f"FP32 FMA issue: {sms} SMs (device query) x {FP32_LANES_PER_SM} lanes x 2 flop x "
                             f"{sm_mhz:.0f} MHz (median sampled)"}
    # HBM-bound kernels: algorithmic bytes per launch.  V = items with a tile
    # (the rest are culled and write only their count and depth key).
    I = int(st.plan.n_items)
    V = visible_items(st)
    N = st.g.n
    P = int(st.plan.n_pairs)
    per = {"tile_sort_onesweep": 16 * E, "depth_sort_onesweep": 16 * I, "tile_sort_histogram": 4 * E,
           "depth_sort_histogram": 4 * I, "pair_sort_onesweep": 16 * P, "pair_sort_histogram": 4 * P,
           # tile lists: the item id and band size of every position, the 32 B binning record of every
           # visible item, 8 B per pair
           "lists_pairs": 8 * I + 32 * V + 8 * P,
           # the row-sorted pairs in, one item id per entry out
           "lists_entries": 8 * P + 4 * E,
           # item id, tile count and offset of every item; centre and row parameters of visible ones; entries
           "duplicate": 8 * I + 52 * V + 8 * E,
           # attributes of every Gaussian; count and key of every item, 136 B of state per visible item
           "preprocess": 236 * N + 8 * I + 136 * V,
           # attributes and their gradients; the 2-D gradients (36 B) of visible items
           "preprocess_backward": 2 * 236 * N + 36 * V}
    bytes_ = per.get(name, 0)
    ach = bytes_ / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": None}


FP32_LANES_PER_SM = 128
# Algorithmic FP32 operations (an FMA counts 2) per (pixel, entry) pair,
# counted for the plain sequential per-pixel algorithm (no scan or other
# parallelisation overhead).  A blended pair: forward: offsets 2, exponent 8,
# alpha 2, transmittance 2, weight 1, colour 6, blended depth 2, argmax 1 =
# 24; backward: offsets 2, exponent 8, alpha 2, transmittance 2, weight 1,
# c.g 5, running colour sum 2, colour gradient 6, dL/dalpha 4, dL/de 2, conic
# and centre terms 17, I_i 1 = 52.  A pair skipped at alpha < 1/255: offsets
# 2 and exponent 8 = 10.  The forward's evaluations past the last blended
# entry (the stopping entry, or the rest of a list that never stops) are not
# counted, so the figure is a lower bound of the forward's work.  MUFU work
# (ex2, rcp) is not counted.
FWD_FLOPS_PER_BLEND = 24
BWD_FLOPS_PER_BLEND = 52
FLOPS_PER_SKIP = 10


def pair_counts(st: "Step") -> dict:
    """Pairs of the step's last forward: blended (sum of n_blended) and
    skipped before the last blended entry (sum of n_contrib - n_blended).
    One extra forward launch with the n_blended output, outside any timed
    region, on the step's current workspaces."""
    if getattr(st, "_pairs", None) is not None:
        return st._pairs
    torch = st.torch
    outs = dict(st.outs)
    outs["n_blended"] = torch.empty_like(st.outs["n_contrib"])
    st.raster.render_fwd(st.plan, st.cfg, st.pre_ws, st.sort_ws, outs)
    blended = int(outs["n_blended"].to(torch.int64).sum().item())
    evals = int(st.outs["n_contrib"].to(torch.int64).sum().item())
    st._pairs = {"blended": blended, "skipped": evals - blended, "evaluated": evals}
    return st._pairs


def run_ours(args, rank, world):
    import torch
    from paper_2411_12788_gb300 import _lib
    L = _lib.lib()
    st = Step(args.n, seed=0)
    for _ in range(args.warmup):
        st.run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler()
    clocks.start()
    L.gs_timing_enable(1)
    kernel_times()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st.run()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    kt = kernel_times()
    L.gs_timing_enable(0)
    ck = clocks.stop(torch.cuda.current_device())
    sec = e0.elapsed_time(e1) / 1e3
    units, sec_max = aggregate(st.pixels * args.steps, sec, world)
    value = units / sec_max / 1e6
    total_kms = sum(v["ms"] for v in kt.values())
    for v in kt.values():
        v["share"] = v["ms"] / total_kms if total_kms else 0.0
        v["ms_per_launch"] = v["ms"] / max(1, v["launches"])
    launches = sum(v["launches"] for v in kt.values())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {"hbm_gbs": 6800.0, "note": "fallback"}
    rl = roofline(kt, st, args.steps, peaks, ck)
    rls = all_rooflines(kt, st, peaks, ck)

    function_step = run_function_step(st, args)
    strategies = None if args.no_culling else run_strategies(st)
    culling = None if args.no_culling else run_culling(st, args, sec_max * 1e3 / args.steps)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(st, args, world)
    serving = None if args.no_serve else run_serving(st, args)
    dense = None if args.no_dense else run_dense(args)
    c1 = None if args.no_dense else run_c1_step()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(st.scene, st.cams)
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec_max * 1e3 / args.steps,
            "steps_per_s": args.steps / sec_max * world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": args.n, "views": len(st.cams),
                       "pixels_per_step": st.pixels, "entries_per_step": int(st.plan.n_entries),
                       "l2": "inputs larger than L2 (236 MB scene, 1.5 GB workspace)",
                       "parallelism": f"replicas x{world}"},
            "roofline": rl, "rooflines": rls, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches // 1,
            "autograd_function_step": function_step,
            "serving": serving, "dense_phase": dense, "single_view_l1_ssim": c1, "culling": culling,
            "strategies": strategies,
            "clocks": ck, "kernels": kt}
    return line


def run_function_step(st: Step, args) -> dict:
    """The same batched step through the public autograd API:
    raster.rasterize (the torch.autograd.Function) and raster.l1_loss, then
    loss.backward(); once with the sorted lists kept for the backward and
    once with them rebuilt there (recompute_sort).  Workspaces and outputs
    come from the torch caching allocator each step; the gradient buffers
    are dropped between steps.  Events on the current stream, like the
    main step."""
    import torch
    r = st.raster
    ps = [getattr(st.g, k).detach().clone().requires_grad_(True)
          for k in ("means", "scales", "rotations", "opacities", "sh")]
    out = {}
    for recompute in (False, True):
        settings = r.RasterSettings(st.cams, st.g.sh_degree, recompute_sort=recompute)

        def step():
            for p in ps:
                p.grad = None
            img, depth, imax, wsum, area = r.rasterize(*ps, settings)
            r.l1_loss(img, st.target).backward()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out["recompute_sort" if recompute else "keep_sort"] = {"ms_per_step": ms,
                                                               "mpix_per_s": st.pixels / ms / 1e3}
    out["note"] = ("raster.rasterize + raster.l1_loss + backward(): outputs colour, d^mid, i_max, I_i and S_i; "
                   "allocations through the caching allocator")
    return out


def run_culling(st: Step, args, ms_unculled: float) -> dict:
    """Occluded-Gaussian culling (Sec. 5.2): the per-view visibility V_i of
    the step's scene and views from one forward pass (I_i, S_i, i_max, w_max
    -> gs_identify), then the same training step with the invisible (view,
    Gaussian) items masked out in the preprocess.  Reports both step times,
    like the paper's comparison of training with and without culling."""
    import torch
    r = st.raster
    outs = r.alloc_outputs(st.plan, "cuda", want=("image", "final_T", "n_contrib", "imax", "wmax", "weight_sum",
                                                  "max_area"))
    r.preprocess(st.plan, st.g.struct(), st.cfg, st.pre_ws)
    r.bin_sort(st.plan, st.pre_ws, st.sort_ws)
    r.render_fwd(st.plan, st.cfg, st.pre_ws, st.sort_ws, outs)
    entries = int(st.plan.n_entries)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    idr = r.identify(st.plan, outs["weight_sum"], outs["max_area"], outs["imax"], outs["wmax"])
    e1.record(stream)
    torch.cuda.synchronize()
    identify_ms = e0.elapsed_time(e1)
    mask = idr["visible_mask"]
    for _ in range(3):
        st.run(mask)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        st.run(mask)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    culled_entries = int(st.plan.n_entries)
    counts = idr["counts"].cpu().tolist()
    return {"visible_items": int(mask.to(torch.int64).sum().item()), "items": int(st.plan.n_items),
            "per_view_blur_intersect_visible_critical": counts, "identify_ms": identify_ms,
            "ms_per_step_unculled": ms_unculled, "ms_per_step_culled": ms,
            "mpix_per_s_culled": st.pixels / ms / 1e3, "entries_unculled": entries, "entries_culled": culled_entries,
            "note": "visibility: keep quantile 0.99 of the positive I_i per view; the masked step renders only "
                    "the visible (view, Gaussian) items"}


def run_strategies(st: Step, reps: int = 5) -> dict:
    """The kernels of the reorganisation on the step's own outputs: primitive
    sampling of half of the Gaussians with I_i > 0 by P_i ~ I_i (Sec. 4.3;
    I_i summed over the 8 views), depth-reinitialization seeds of 10 % of
    each view's pixels (Sec. 4.2), the fused L1 + D-SSIM loss over the 8
    views and the aggressive clone of the first view's critical Gaussians
    (Sec. 5.1; allocation of the grown scene included).  Mean of `reps`
    calls each, CUDA events."""
    import torch
    r = st.raster
    n = st.g.n
    I = st.grads["weight_sum"].view(len(st.cams), n).sum(0)
    g = torch.Generator(device="cuda").manual_seed(7)
    E = -torch.log(1.0 - torch.rand(n, device="cuda", generator=g))      # Exp(1) draws
    k = int((I > 0).sum().item()) // 2
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r.sample_gaussians(I, E, k)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        kept = r.sample_gaussians(I, E, k)
    e1.record(stream)
    torch.cuda.synchronize()
    sample_ms = e0.elapsed_time(e1) / reps
    us = [1.0 - torch.rand(int(c.width) * int(c.height), device="cuda", generator=g) for c in st.cams]
    ks = [int(c.width) * int(c.height) // 10 for c in st.cams]
    from paper_2411_12788_gb300 import _lib
    kernel_times()                                   # drain earlier records
    _lib.lib().gs_timing_enable(1)
    e0.record(stream)
    drawn = 0
    for _ in range(reps):
        for v in range(len(st.cams)):
            off = int(st.plan.pixel_base[v])
            tgt = st.target[3 * off: 3 * int(st.plan.pixel_base[v + 1])]
            drawn += int(r.depth_points(st.plan, v, st.outs["depth"], st.outs["imax"], tgt, us[v],
                                        ks[v])["points"].shape[0])
    e1.record(stream)
    torch.cuda.synchronize()
    _lib.lib().gs_timing_enable(0)
    depth_dev_ms = sum(v["ms"] for v in kernel_times().values()) / reps
    depth_ms = e0.elapsed_time(e1) / reps
    # fused L1 + D-SSIM loss and gradient over the 8 views (the C1 objective)
    L = torch.zeros(1, device="cuda")
    dL = torch.empty_like(st.outs["image"])
    ws = r.loss_l1_ssim(st.plan, st.outs["image"], st.target, L, dL, 0.2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        r.loss_l1_ssim(st.plan, st.outs["image"], st.target, L, dL, 0.2, ws=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ssim_ms = e0.elapsed_time(e1) / reps
    # aggressive clone of the first view's critical Gaussians (Sec. 5.1)
    outs = r.alloc_outputs(st.plan, "cuda", want=("image", "final_T", "n_contrib", "imax", "wmax", "weight_sum",
                                                  "max_area"))
    r.render_fwd(st.plan, st.cfg, st.pre_ws, st.sort_ws, outs)
    ids = r.identify(st.plan, outs["weight_sum"], outs["max_area"], outs["imax"], outs["wmax"])
    crit = torch.nonzero(ids["flags"][:n] & r.ID_CRITICAL).flatten().to(torch.int32)
    r.clone_gaussians(st.g, crit)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cl = r.clone_gaussians(st.g, crit)
    e1.record(stream)
    torch.cuda.synchronize()
    clone_ms = e0.elapsed_time(e1) / reps
    del cl
    return {"sample_gaussians_ms": sample_ms, "sampled": int(kept.numel()), "of_positive": 2 * k,
            "loss_l1_ssim_ms_8_views": ssim_ms,
            "clone_critical_ms": clone_ms, "cloned": int(crit.numel()),
            "depth_points_ms_8_views": depth_ms, "depth_points_device_ms_8_views": depth_dev_ms,
            "depth_points_per_call": drawn // reps,
            "note": "depth_points_ms includes one host read of the drawn count per view (the Python binding "
                    "slices its outputs); depth_points_device_ms sums the event-timed kernels of those calls"}


def run_c1_step(iters: int = 5) -> dict:
    """The training step of the single-view configuration: 500k Gaussians
    (SH 3, 64-cluster + shell scene), one 1600x1063 ring view, 0.8 L1 +
    0.2 D-SSIM against the seeded target; forward (colour, depth, i_max, I_i),
    fused loss, backward.  Mean of `iters` steps after one warm-up, CUDA
    events."""
    import torch
    from paper_2411_12788_gb300 import raster, scenes
    sc = scenes.cluster_scene(500_000, 64, seed=0, sh_degree=3)
    cam = scenes.ring_camera(0.3, 1600, 1063)
    g = raster.GaussianTensors.from_scene(sc, "cuda")
    y = torch.as_tensor(scenes.target_images([cam], seed=1)[0].reshape(-1)).cuda()
    plan = raster.make_plan(sc.n, [cam])
    cfg = raster.make_config(flags=raster._lib.GS_FLAG_ZERO_ACCUM)
    pre_ws = torch.empty(raster.preprocess_workspace_size(plan), dtype=torch.uint8, device="cuda")
    outs = raster.alloc_outputs(plan, "cuda", want=("image", "final_T", "n_contrib", "depth", "imax"))
    grads = raster.alloc_grads(g)
    grads["weight_sum"] = torch.zeros(int(plan.n_items), device="cuda")
    L = torch.zeros(1, device="cuda")
    dL = torch.empty_like(outs["image"])
    state = {"sort": torch.empty(0, dtype=torch.uint8, device="cuda"), "ws": None}

    def step():
        raster.preprocess(plan, g.struct(), cfg, pre_ws)
        need = raster.bin_sort_workspace_size(plan)
        if state["sort"].numel() < need:
            state["sort"] = torch.empty(int(need * 1.1), dtype=torch.uint8, device="cuda")
        raster.bin_sort(plan, pre_ws, state["sort"])
        raster.render_fwd(plan, cfg, pre_ws, state["sort"], outs)
        state["ws"] = raster.loss_l1_ssim(plan, outs["image"], y, L, dL, 0.2, ws=state["ws"])
        raster.render_bwd(plan, g.struct(), cfg, pre_ws, state["sort"], dL, outs["image"], outs["n_contrib"],
                          grads)
    step()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(iters):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    return {"workload": "500k Gaussians SH3, 1600x1063, 0.8 L1 + 0.2 D-SSIM: fwd + fused loss + bwd",
            "ms_per_step": ms, "mpix_per_s": cam.width * cam.height / ms / 1e3, "entries": int(plan.n_entries),
            "loss": float(L.item())}


def run_e2e(st: Step, args, world) -> dict:
    """The same step with host buffers: every step copies its scene and target
    images in from pinned host memory and its loss and gradients (and I_i)
    back out.  Uploads and downloads run on two more streams (one per
    direction, so both copy directions are busy at once) with two device
    buffer sets, so step k+1's upload and step k's download overlap step k's
    compute; all of them are inside the timed region."""
    import torch
    from paper_2411_12788_gb300 import raster
    names = ("means", "scales", "rotations", "opacities", "sh")
    host_in = {k: getattr(st.g, k).cpu().pin_memory() for k in names}
    host_tg = st.target.cpu().pin_memory()
    sets = []
    for b in range(2):
        g = st.g if b == 0 else raster.GaussianTensors(*(getattr(st.g, k).clone() for k in names), st.g.sh_degree)
        tg = st.target if b == 0 else st.target.clone()
        gr = st.grads if b == 0 else {k: v.clone() for k, v in st.grads.items()}
        loss = st.loss if b == 0 else st.loss.clone()
        out = {k: v.cpu().pin_memory() for k, v in gr.items()}
        sets.append({"g": g, "target": tg, "grads": gr, "loss": loss, "host_out": out,
                     "host_loss": torch.zeros(1).pin_memory()})
    h2d = sum(t.numel() * 4 for t in host_in.values()) + host_tg.numel() * 4
    d2h = sum(t.numel() * 4 for t in sets[0]["host_out"].values()) + 4
    compute = torch.cuda.current_stream()
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]       # set b's inputs are uploaded
    done = [torch.cuda.Event(), torch.cuda.Event()]        # the step using set b has finished
    fetched = [torch.cuda.Event(), torch.cuda.Event()]     # set b's outputs are downloaded
    orig = (st.g, st.target, st.grads, st.loss)

    def upload(b):
        with torch.cuda.stream(copy_in):
            copy_in.wait_event(done[b])              # the step that last read set b is finished
            for k in names:
                getattr(sets[b]["g"], k).copy_(host_in[k], non_blocking=True)
            sets[b]["target"].copy_(host_tg, non_blocking=True)
            ready[b].record(copy_in)

    def run(k):
        b = k % 2
        compute.wait_event(ready[b])
        compute.wait_event(fetched[b])               # the last download of set b's outputs
        st.g, st.target, st.grads, st.loss = sets[b]["g"], sets[b]["target"], sets[b]["grads"], sets[b]["loss"]
        st.run()
        done[b].record(compute)
        with torch.cuda.stream(copy_out):
            copy_out.wait_event(done[b])
            for key, v in sets[b]["grads"].items():
                sets[b]["host_out"][key].copy_(v, non_blocking=True)
            sets[b]["host_loss"].copy_(sets[b]["loss"], non_blocking=True)
            fetched[b].record(copy_out)

    def steps(n):
        upload(0)
        upload(1)
        for k in range(n):
            run(k)
            if k + 2 < n:
                upload(k % 2)                       # inputs of step k+2 go into the set step k used
        compute.wait_stream(copy_in)
        compute.wait_stream(copy_out)               # the last downloads are part of the run

    steps(3)
    torch.cuda.synchronize()
    barrier(world)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(compute)
    steps(args.steps)
    t1.record(compute)
    torch.cuda.synchronize()
    barrier(world)
    st.g, st.target, st.grads, st.loss = orig
    sec = t0.elapsed_time(t1) / 1e3
    units, sec_max = aggregate(st.pixels * args.steps, sec, world)
    return {"value": units / sec_max / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": sec_max * 1e3 / args.steps,
            "overlap": "double-buffered: uploads and downloads on one stream per direction overlap the "
                       "previous/next step"}


def run_serving(st: Step, args) -> dict:
    """Serving loop on the resident 1M scene: Poisson arrivals (seed 3), poses
    on a sphere of radius U[3, 6], resolutions uniform over 640x480 /
    1280x720 / 1920x1080 / 3840x2160, 24 GB admission budget; the first 10 %
    of requests are warm-up.  Batched (3 stream slots with their own worker
    threads, up to 16 views per batch) against the same trace served one
    request at a time, at 200 requests/s and at 600 requests/s (where
    requests contend for the GPU), each repeated `serve_runs` times on the
    same trace so that the gain can be set against the run-to-run spread."""
    import torch
    from paper_2411_12788_gb300 import serve
    n = args.serve_requests
    skip = n // 11
    # the earlier phases' cached blocks go back to the device, so that the
    # servers' buffers are fresh allocations made before their clocks start
    torch.cuda.empty_cache()

    def once(rate, name, streams, views):
        trace = serve.poisson_trace(n, rate=rate, seed=3)
        srv = serve.RenderServer(st.g, budget_bytes=24 << 30, streams=streams, max_views=views)
        srv.serve(trace)
        torch.cuda.synchronize()
        stats = serve.latency_stats(trace, skip=skip)
        stats.update({"batches": srv.batches_run, "mean_views_per_batch": srv.views_run / max(1, srv.batches_run),
                      "peak_reserved_gb": srv.peak_reserved / 2**30})
        return stats

    def compare(rate):
        runs = []
        for _ in range(args.serve_runs):
            runs.append({"batched": once(rate, "batched", 3, 16), "one_at_a_time": once(rate, "one", 1, 1)})
        gains = [r["one_at_a_time"]["p99_ms"] / r["batched"]["p99_ms"] for r in runs]
        b99 = [r["batched"]["p99_ms"] for r in runs]
        o99 = [r["one_at_a_time"]["p99_ms"] for r in runs]
        return {"rate_per_s": rate, "requests_timed": n - skip, "warmup_requests": skip, "budget_gb": 24,
                "scene_gaussians": st.g.n, "runs": runs,
                "p99_ms_batched": b99, "p99_ms_one_at_a_time": o99,
                "p99_speedup_per_run": gains, "p99_speedup_median": statistics.median(gains),
                "p99_spread_batched": (max(b99) - min(b99)) / statistics.median(b99),
                "p99_spread_one_at_a_time": (max(o99) - min(o99)) / statistics.median(o99),
                "mean_views_per_batch": statistics.mean(r["batched"]["mean_views_per_batch"] for r in runs)}
    res = compare(200.0)
    res["at_600_per_s"] = compare(600.0)
    return res


def run_dense(args, iters: int = 3) -> dict:
    """Dense-phase step (MSv2-D): 3M Gaussians (256 clusters, SH 3), one
    1920x1080 view: fwd+bwd with L1, keep the top 25 % by accumulated weight,
    gather them and re-render the sparse set."""
    import torch
    from paper_2411_12788_gb300 import raster, scenes
    sc = scenes.cluster_scene(3_000_000, 256, seed=0, sh_degree=3)
    cam = scenes.ring_camera(0.3, 1920, 1080)
    g = raster.GaussianTensors.from_scene(sc, "cuda")
    target = torch.as_tensor(scenes.target_images([cam], seed=1)[0].reshape(-1)).cuda()
    cfg = raster.make_config(flags=raster._lib.GS_FLAG_ZERO_ACCUM)
    k = math.ceil(0.25 * sc.n)
    loss = torch.zeros(1, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    times = {"fwd_bwd": 0.0, "prune_gather": 0.0, "rerender": 0.0}

    def once(record):
        s = torch.cuda.current_stream()
        if record:
            ev[0].record(s)
        fr = raster.forward(g, [cam], cfg)
        dL = torch.empty_like(fr.outs["image"])
        raster.loss_l1(fr.outs["image"], target, loss, dL)
        raster.backward(g, fr, dL)
        if record:
            ev[1].record(s)
        keep = raster.prune_select(fr.outs["weight_sum"], k)
        h = raster.gather_scene(g, keep)
        if record:
            ev[2].record(s)
        fr2 = raster.forward(h, [cam], cfg)
        if record:
            ev[3].record(s)
            torch.cuda.synchronize()
            times["fwd_bwd"] += ev[0].elapsed_time(ev[1])
            times["prune_gather"] += ev[1].elapsed_time(ev[2])
            times["rerender"] += ev[2].elapsed_time(ev[3])
        return fr, fr2
    once(False)
    torch.cuda.synchronize()
    for _ in range(iters):
        fr, fr2 = once(True)
    ms = {k2: v / iters for k2, v in times.items()}
    total = sum(ms.values())
    pix = cam.width * cam.height
    return {"workload": "3M Gaussians SH3 (256 clusters), 1920x1080: fwd+bwd, top-25% prune, re-render",
            "ms": ms, "ms_total": total, "kept": k, "entries": int(fr.plan.n_entries),
            "entries_after_prune": int(fr2.plan.n_entries), "mpix_per_s": 2 * pix / total / 1e3,
            "note": "each phase allocates its workspaces from the torch caching allocator"}


# ---------------------------------------------------------------- oracle arm
def oracle_view_setup(scene, cam) -> dict:
    """The oracle's per-view work that does not depend on the pixels: the
    projection of every Gaussian (no gradient) and the tile lists (exact
    support, oracle.binning.tile_lists).  Timed."""
    import torch
    from oracle import binning as OB, project as OP
    t0 = time.perf_counter()
    with torch.no_grad():
        pr = OP.project(scene.means, scene.scales, scene.rotations, scene.opacities, scene.sh,
                        scene.sh_degree, cam)
    gg, tt, _, _, _ = OB.tile_lists(pr["mean2d"].numpy(), pr["conic"].numpy(), pr["opacity"].numpy(),
                                     pr["valid"].numpy(), cam.width, cam.height)
    tx, ty = OB.tile_grid(cam.width, cam.height)
    order = np.argsort(tt, kind="stable")
    starts = np.searchsorted(tt[order], np.arange(tx * ty + 1))
    return {"gauss": gg[order], "starts": starts, "tiles": tx * ty, "tiles_x": tx,
            "seconds": time.perf_counter() - t0}


def oracle_tiles_step(scene, cam, setup: dict, tiles) -> tuple[int, float]:
    """float64 oracle fwd+bwd (colour, d^mid, I_i, S_i and the gradients of
    a loss on the colour) of every pixel of the given tiles of one view,
    each tile composited over the Gaussians its list holds.  Returns
    (pixels, seconds)."""
    import torch
    from oracle import project as OP, render as OR
    t0 = time.perf_counter()
    lists = [setup["gauss"][setup["starts"][k]: setup["starts"][k + 1]] for k in tiles]
    sel = np.unique(np.concatenate(lists)) if lists else np.zeros(0, np.int64)
    params = [torch.tensor(np.asarray(a[sel], np.float64), requires_grad=True)
              for a in (scene.means, scene.scales, scene.rotations, scene.opacities, scene.sh)]
    pr = OP.project(*params, scene.sh_degree, cam)
    loss, pixels = 0.0, 0
    for k, lst in zip(tiles, lists):
        ty, tx = divmod(int(k), setup["tiles_x"])
        uu, vv = np.meshgrid(np.arange(16 * tx, min(16 * tx + 16, cam.width)),
                             np.arange(16 * ty, min(16 * ty + 16, cam.height)))
        pix = np.stack([uu.reshape(-1), vv.reshape(-1)], 1)
        view = dict(pr)
        view["valid"] = pr["valid"] & torch.as_tensor(np.isin(sel, lst))
        out = OR.render_view(view, cam, pix=pix, want_depth=True)
        loss = loss + out["colour"].sum()
        pixels += len(pix)
    if pixels and isinstance(loss, torch.Tensor) and loss.requires_grad:
        loss.backward()
    return pixels, time.perf_counter() - t0


def oracle_sample(scene, cams, views, tiles_per_view: int, seed: int) -> dict:
    """Oracle fwd+bwd throughput on a tile sample of the batched workload:
    per view, the projection and binning of all Gaussians, then
    `tiles_per_view` tiles drawn uniformly (seeded).  The per-view work is
    charged by the sampled share of the view's tiles, so the rate is that of
    the oracle rendering whole views."""
    rng = np.random.default_rng(seed)
    pixels, charged, wall0 = 0, 0.0, time.perf_counter()
    for v in views:
        cam = cams[v]
        su = oracle_view_setup(scene, cam)
        tiles = rng.choice(su["tiles"], size=min(tiles_per_view, su["tiles"]), replace=False)
        p, sec = oracle_tiles_step(scene, cam, su, tiles)
        pixels += p
        charged += sec + su["seconds"] * len(tiles) / su["tiles"]
    return {"pixels": pixels, "charged_seconds": charged, "wall_seconds": time.perf_counter() - wall0}


def oracle_full_frame(threads: int | None, backward: bool) -> float:
    """Seconds of the oracle on one full frame of the 1,024-Gaussian 128x128
    scene (SH 0), forward (colour, d^mid, I_i, S_i) or forward + backward,
    on `threads` host threads (None: torch's default)."""
    import torch
    from oracle import project as OP, render as OR
    from paper_2411_12788_gb300 import scenes
    sc = scenes.box_scene(1024, seed=0, sh_degree=0)
    cam = scenes.origin_camera()
    old = torch.get_num_threads()
    if threads:
        torch.set_num_threads(threads)
    try:
        t0 = time.perf_counter()
        params = [torch.tensor(np.asarray(a, np.float64), requires_grad=backward)
                  for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]
        with torch.set_grad_enabled(backward):
            pr = OP.project(*params, sc.sh_degree, cam)
            out = OR.render_view(pr, cam, want_depth=True)
            if backward:
                out["colour"].sum().backward()
        return time.perf_counter() - t0
    finally:
        torch.set_num_threads(old)


def cpu_baseline(scene, cams, tiles_per_view: int = 16, views=(0,)) -> dict:
    """The float64 oracle, as it stands, on the host cores: fwd+bwd Mpix/s on
    a tile sample of the batched workload (the line's metric), plus full
    frames of the small 1,024-Gaussian scene (forward and fwd+bwd on all
    threads, forward on one thread)."""
    import torch
    s = oracle_sample(scene, cams, views, tiles_per_view, seed=11)
    px0 = 128 * 128
    f_all = oracle_full_frame(None, False)
    fb_all = oracle_full_frame(None, True)
    f_one = oracle_full_frame(1, False)
    return {"value": s["pixels"] / s["charged_seconds"] / 1e6, "unit": "Mpix/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": (f"float64 oracle fwd+bwd of {tiles_per_view} random 16x16 tiles of view(s) {list(views)} of "
                       f"the {scene.n}-Gaussian 8-view workload ({s['pixels']} pixels, each tile over its list); the "
                       f"per-view projection and binning of all Gaussians charged by the sampled share of the "
                       f"view's tiles; {s['wall_seconds']:.1f} s wall"),
            "full_frame_1024_gaussians_128x128": {
                "fwd_mpix_s_all_threads": px0 / f_all / 1e6, "fwd_bwd_mpix_s_all_threads": px0 / fb_all / 1e6,
                "fwd_mpix_s_one_thread": px0 / f_one / 1e6, "threads": torch.get_num_threads()}}


def run_reference(args, rank, world):
    """The oracle on the line's workload: each step is fwd+bwd of 8 random
    tiles of one view (round robin over the 8 views), each view's projection
    and binning computed once and charged by the sampled share of its
    tiles."""
    from paper_2411_12788_gb300 import scenes
    if rank != 0:
        return None
    import torch
    scene = scenes.cluster_scene(args.n, 64, seed=0, sh_degree=3)
    cams = scenes.multiview_cameras()
    rng = np.random.default_rng(11)
    per_step = 8
    setups = {}

    def one(k):
        v = k % len(cams)
        if v not in setups:
            setups[v] = oracle_view_setup(scene, cams[v])
        su = setups[v]
        tiles = rng.choice(su["tiles"], size=per_step, replace=False)
        p, sec = oracle_tiles_step(scene, cams[v], su, tiles)
        return p, sec + su["seconds"] * per_step / su["tiles"]
    for k in range(args.warmup):
        one(k)
    done, charged = 0, 0.0
    t0 = time.perf_counter()
    for k in range(args.steps):
        p, sec = one(args.warmup + k)
        done += p
        charged += sec
    wall = time.perf_counter() - t0
    value = done / charged / 1e6
    cpu = {"value": value, "unit": "Mpix/s", "cores": torch.get_num_threads(), "kind": "oracle",
           "sample": f"each step: float64 oracle fwd+bwd of {per_step} random 16x16 tiles of one view (round robin "
                     f"over the 8 views) of the {args.n}-Gaussian workload, each tile over its list; each view's "
                     f"projection and binning of all Gaussians (once per view) charged by the sampled share of "
                     f"its tiles; {wall:.1f} s wall for the timed steps"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": charged * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "gaussians": args.n},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
