#!/usr/bin/env python
"""Benchmark of the 2DGS rasterizer hot path (CityGaussianV2, arXiv
2411.00771): one training step per view = render (preprocess, sort, blend)
+ L1/D-SSIM/depth loss + backward + decomposed densification statistics +
Eq. 2 selection + elongation filter, on a synthetic aerial city block of
1M surfels (SH degree 3) seen at 1600x900.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are launched by torchrun; each
rank renders and differentiates its own view of a replicated scene (no
collective in the step; weak scaling).  ``--impl reference`` times the FP64
CPU oracle on a bounded crop of the same view on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "2DGS fwd+bwd ms/view at 1M surfels 1600x900; served render p50/p99 ms"
UNIT = "ms/view"
N_SURFELS = 1_000_000
WEIGHTS = (0.8, 0.2, 0.5)          # L1, D-SSIM, depth (first-iteration depth weight)
OMEGA, GRAD_THR, ETA_THR = 0.9, 0.0002, 0.1
# algorithmic FP32 work (FMA = 2 FLOPs), see the design notes
FLOP_EVAL = 25       # per list entry evaluated (ray-splat, low-pass max, alpha)
FLOP_BLEND = 26      # per blended pair (composite of 12 planes)
FLOP_BWD_PAIR = 140  # per blended pair in the backward (adjoints + chain)
SM_COUNT, FP32_LANES, SM_MAX_HZ = 152, 128, 2.07e9
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_HZ / 1e12
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peak(key):
    """A peak from the measured-peaks file at the repository root, else the
    earlier single GB300 measurement."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return FALLBACK_PEAKS[key]

# DRAM bytes (read + write) of one blend_bwd launch on this workload, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass, the
# full-size view); valid only for the kernel sources it was taken on.
BLEND_BWD_TRAFFIC = {"bytes": 173498880 + 12352256,
                     "sources_sha256": "1cd9e09a91486b181251c0e18ac59717778c8cb85654a43281f1d093b2313cd1"}


def blend_sources_sha256():
    """SHA-256 of blend.cu followed by gs2d_internal.cuh."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for f in ("blend.cu", "gs2d_internal.cuh"):
        with open(os.path.join(here, "paper_2411_00771_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def blend_bwd_traffic():
    """The captured traffic if blend.cu + gs2d_internal.cuh are unchanged, else None."""
    ok = blend_sources_sha256() == BLEND_BWD_TRAFFIC["sources_sha256"]
    return BLEND_BWD_TRAFFIC["bytes"] if ok else None


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--width", type=int, default=1600, help="view width (smaller views for ncu captures)")
    ap.add_argument("--height", type=int, default=900)
    ap.add_argument("--no-training", action="store_true", help="skip the 4M-surfel training-step measurement")
    ap.add_argument("--no-vq", action="store_true", help="skip the vector-quantisation measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        self.cmd = cmd

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) == len(self.FIELDS):
                self.rows.append(p)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------
def workload_config(W: int, H: int, views: int) -> dict:
    """The config object of the JSON line (the same for both arms)."""
    return {"workload": f"aerial city block, 1M surfels SH3, {W}x{H}, fwd+bwd+loss+densify",
            "surfels": N_SURFELS, "width": W, "height": H, "sh_degree": 3, "views_per_step": views,
            "l2": "inputs larger than L2 (232 MB surfel parameters, 69 MB render planes per view)"}


def rank_env():
    """(world size, rank, local rank) of this process (torchrun's variables;
    1, 0, 0 when run alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_azimuth(rank: int) -> float:
    """Each rank renders its own view of the replicated scene (weak scaling:
    views are independent, no collective in the step): azimuths 45 degrees
    apart, rank 0 the single-GPU view."""
    return -90.0 + 360.0 * rank / 8.0


def max_over_ranks(value: float, world: int, dist=None, device="cpu") -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_view(ms_step_max: float, world: int, views_per_rank: int = 1) -> float:
    """Whole-job ms per view: every rank finishes views_per_rank views per step,
    the step ends when the slowest rank does."""
    return ms_step_max / (world * views_per_rank)


def city_workload(rank: int, width: int = 1600, height: int = 900):
    from paper_2411_00771_gb300 import synthetic as syn
    scene, info = syn.city_scene(n=N_SURFELS)
    cam = syn.aerial_camera(width=width, height=height, azimuth_deg=rank_azimuth(rank))
    tgt, tinv = syn.city_targets(info, cam)
    return scene, cam, tgt, tinv


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2411_00771_gb300 import binding as B

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    scene_np, cam, tgt_np, tinv_np = city_workload(rank, args.width, args.height)
    P = {k: torch.from_numpy(np.ascontiguousarray(scene_np[k], np.float32)).to(dev)
         for k in ("mu", "quat", "scale", "opacity", "sh")}
    sc = B.Scene(P["mu"], P["quat"], P["scale"], P["opacity"], P["sh"], scene_np["sh_degree"])
    H, W = cam["height"], cam["width"]
    n = scene_np["mu"].shape[0]
    out = torch.empty((12, H, W), device=dev)
    adj_t = torch.zeros((11, H, W), device=dev)
    adj_s = torch.zeros((11, H, W), device=dev)
    adj_l = torch.zeros((11, H, W), device=dev)
    losses = torch.empty(4, device=dev)
    # the gradients and screen gradients live in one buffer: one fill per step
    sizes = [v.numel() for v in P.values()] + [3 * n * 2]
    flat = torch.zeros(sum(sizes), device=dev)
    views = list(torch.split(flat, sizes))
    grads = {k: views[i].view(v.shape) for i, (k, v) in enumerate(P.items())}
    screen = views[-1].view(3, n, 2)
    stats = torch.zeros((n, 4), device=dev)
    tgt = torch.from_numpy(tgt_np).to(dev)
    tinv = torch.from_numpy(tinv_np).to(dev)
    masks = [0x7 | (1 << 5), 0x7, 0x7]
    keep_frame = [None]

    def step(keep=False, tgt_in=None, tinv_in=None):
        o, frame = sc.render(cam, out=out)
        B.loss(o, tgt if tgt_in is None else tgt_in, tinv if tinv_in is None else tinv_in, WEIGHTS,
               adj_total=adj_t, adj_ssim=adj_s, adj_l1=adj_l, losses=losses)
        flat.zero_()
        sc.backward(frame, [adj_t, adj_s, adj_l], masks, grads, screen)
        sc.densify_accumulate(frame, screen, stats)
        mask, _, _ = B.densify_select(stats, P["scale"], OMEGA, GRAD_THR, ETA_THR)
        B.elongation_filter(P["scale"], ETA_THR)
        if keep:
            keep_frame[0] = frame
        else:
            frame.release()
        return mask

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_uuid(local))
    barrier()
    torch.cuda.synchronize()
    l0 = B.kernel_launches()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = B.kernel_launches() - l0
    ms_step = ev0.elapsed_time(ev1) / args.steps
    # stage times and per-launch kernel times from a separate pass with the
    # library's profiling events on (they are not part of the timed steps)
    B.profile_read()
    B.profile_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    B.profile_enable(False)
    prof = B.profile_read()
    ms_step_max = max_over_ranks(ms_step, world, dist, dev)

    # end to end through the public API: host targets in, losses and the
    # densification mask out, every step
    tgt_h = torch.from_numpy(tgt_np).pin_memory()
    tinv_h = torch.from_numpy(tinv_np).pin_memory()
    loss_h = torch.empty(4).pin_memory()
    mask_h = torch.empty(n, dtype=torch.uint8).pin_memory()
    e2e_steps = max(3, args.steps // 2)

    # inputs double-buffered: the next step's targets are copied on a second
    # stream while the current step computes (as a training loop prefetches)
    tgt_d, tinv_d = [tgt, torch.empty_like(tgt)], [tinv, torch.empty_like(tinv)]
    copy_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]

    def prefetch(b):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(free[b])  # the step that last read buffer b is done
            tgt_d[b].copy_(tgt_h, non_blocking=True)
            tinv_d[b].copy_(tinv_h, non_blocking=True)
            ready[b].record(copy_stream)

    def step_e2e(i):
        b = i % 2
        torch.cuda.current_stream().wait_event(ready[b])
        mask = step(tgt_in=tgt_d[b], tinv_in=tinv_d[b])
        free[b].record()
        prefetch(1 - b)
        loss_h.copy_(losses, non_blocking=True)
        mask_h.copy_(mask, non_blocking=True)

    prefetch(0)
    step_e2e(0)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    prefetch(0)
    for i in range(e2e_steps):
        step_e2e(i)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, world, dist, dev)

    # work counts of this view (deterministic per step) for the roofline
    step(keep=True)
    info = keep_frame[0].info()
    keep_frame[0].release()
    E, Bl, R = info["pairs_evaluated"], info["pairs_blended"], info["bwd_pairs_evaluated"]
    work = {"blend_fwd": FLOP_EVAL * E + FLOP_BLEND * Bl,
            "blend_bwd": FLOP_EVAL * R + FLOP_BWD_PAIR * Bl}
    per_launch = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in prof.items()}
    dom = max(("blend_fwd", "blend_bwd"), key=lambda k: prof[k][0])
    achieved = work[dom] / (per_launch[dom] * 1e-3) / 1e12
    roofline = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
                "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                "traffic": (blend_bwd_traffic() if dom == "blend_bwd" and W == 1600 and H == 900 else None),
                "ms_per_launch": round(per_launch[dom], 4),
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and max clock)"}
    # per step: a group may record several scopes per step (the sort group
    # covers every scan, radix pass, emit and range pass of a render)
    breakdown = {k: round(v[0] / args.steps, 4) for k, v in prof.items()}

    contribution = measure_contribution(sc, cam, n, dev, args)
    visibility = measure_visibility(scene_np, dev, args)
    training, vq = (None, None) if args.no_training else measure_training(dev, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene_np, cam, tgt_np, tinv_np, budget_s=20.0)
    serving = None
    if not args.no_serving:
        del grads, screen, flat, views, stats, adj_t, adj_s, adj_l
        torch.cuda.empty_cache()
        serving = run_serving(args, dev, sc, P, rank)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(job_ms_per_view(ms_step_max, world), 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": round(ms_step_max, 4), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(W, H, world),
            "e2e": {"value": round(job_ms_per_view(e2e_ms, world), 4), "unit": UNIT,
                    "h2d_bytes_per_step": int(tgt_h.numel() * 4 + tinv_h.numel() * 4) * world,
                    "d2h_bytes_per_step": int(16 + n) * world},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "stage_ms": breakdown,
            "work": {"instances": info["n_instances"], "visible": info["n_visible"],
                     "pairs_evaluated": E, "pairs_blended": Bl, "bwd_pairs_replayed": R,
                     "bwd_warp_steps": info["bwd_warp_entries"],
                     "bwd_lanes_per_step": round(info["bwd_warp_lanes"] / max(1, info["bwd_warp_entries"]), 2)},
            "clocks": clk,
            "cpu_baseline": cpu,
            "contribution": contribution,
            "visibility": visibility,
            "training": training,
            "vq": vq,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_contribution(sc, cam, n, dev, args):
    """Trim contribution (Sec. 3.3, Eq. 3) of the same view, accumulated with
    weight 1 (Eq. 4's sum), and the percentile prune at the paper's ratio, each
    timed with CUDA events over repeated calls after warm-up."""
    import torch
    from paper_2411_00771_gb300 import binding as B
    contrib = torch.zeros(n, device=dev)
    reps = max(3, min(args.steps, 20))
    for _ in range(3):
        sc.contribution(cam, gamma=0.5, weight=1.0, contrib=contrib)
    torch.cuda.synchronize()
    l0 = B.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sc.contribution(cam, gamma=0.5, weight=1.0, contrib=contrib)
    e1.record()
    torch.cuda.synchronize()
    ms_view = e0.elapsed_time(e1) / reps
    launches = (B.kernel_launches() - l0) / reps
    for _ in range(3):
        B.prune_by_contribution(contrib, 0.025)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        keep, bound = B.prune_by_contribution(contrib, 0.025)
    e1.record()
    torch.cuda.synchronize()
    return {"ms_per_view": round(ms_view, 4), "gamma": 0.5, "launches_per_view": launches,
            "prune_ms": round(e0.elapsed_time(e1) / reps, 4), "prune_ratio": 0.025,
            "pruned": int(n - int(keep.sum().item()))}


def measure_training(dev, args):
    """The training step of the 4M-surfel configuration: 4 views at 1600x900
    from random poses on an orbit 200 m up, the full loss (L1, SSIM, depth,
    normal consistency, distortion), the hand backward with the preprocess
    recomputed, densification statistics and the FP32 Adam update, timed with
    CUDA events: through torch.autograd (activate, render and loss as
    autograd Functions, one backward()) and by the direct calls."""
    import numpy as np
    import torch
    from paper_2411_00771_gb300 import synthetic as syn
    from paper_2411_00771_gb300 import training as T
    scene, info = syn.city_scene(seed=20241101 + 3, n=4_000_000)
    rng = np.random.default_rng(20241101 + 4)
    views = []
    for _ in range(4):
        cam = syn.orbit_camera(rng, 1600, 900, radius=rng.uniform(150.0, 250.0), altitude=200.0)
        tgt, tinv = syn.city_targets(info, cam)
        views.append((cam, torch.from_numpy(tgt).to(dev), torch.from_numpy(tinv).to(dev)))
    P = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev) for k in ("mu", "quat", "scale",
                                                                                          "opacity", "sh")}
    tr = T.Trainer(P["mu"], P["quat"], torch.log(P["scale"]), torch.logit(P["opacity"].clamp(1e-6, 1 - 1e-6)),
                   P["sh"], scene["sh_degree"], w_normal=0.0125, w_dist=0.01)
    del P
    reps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = {}
    for mode in ("autograd", "direct"):
        for _ in range(3):
            tr.step(views, autograd=mode == "autograd")
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            L = tr.step(views, autograd=mode == "autograd")
        e1.record()
        torch.cuda.synchronize()
        ms[mode] = e0.elapsed_time(e1) / reps
    out = {"surfels": tr.n, "views_per_step": 4, "resolution": [1600, 900], "step": "autograd.Function",
           "ms_per_step": round(ms["autograd"], 3), "steps_per_s": round(1e3 / ms["autograd"], 2),
           "ms_per_step_direct": round(ms["direct"], 3), "steps": reps,
           "loss_total": round(float(L[3]) / 4, 5)}
    vq = None if args.no_vq else measure_vq(tr, views, dev, args)
    del tr, views
    torch.cuda.empty_cache()
    return out, vq


VQ_K, VQ_RATIO, VQ_ITERS = 8192, 0.4, 10


def measure_vq(tr, views, dev, args):
    """Contribution-based vector quantisation of the 4M-surfel scene (Sec.
    3.3; Appendix C: 8192 entries, ratio 0.4): the contribution over the 4
    views (Eq. 4), then quantised set, Lloyd's K-means (10 steps, tensor
    cores) and the compressed layout, timed end to end; the assignment
    kernel alone through the library's profiling events (tensor roofline:
    2 m K C FLOPs per launch against the measured dense 16-bit peak); and the
    render of the compressed scene against the FP32 one."""
    import torch
    from paper_2411_00771_gb300 import binding as B
    n = tr.n
    B.activate(tr.raw["scale"], tr.raw["opacity"], tr.scale, tr.opacity)
    contrib = torch.zeros(n, device=dev)
    for cam, _, _ in views:
        tr.scene.contribution(cam, gamma=0.5, weight=1.0 / len(views), contrib=contrib)
    params = (tr.raw["mu"].detach(), tr.raw["quat"].detach(), tr.scale, tr.opacity, tr.raw["sh"].detach())
    u = torch.rand(VQ_K, device=dev, generator=torch.Generator(device=dev).manual_seed(20241101))
    B.compress(params, 3, contrib, VQ_RATIO, VQ_K, 1, u, method=1)  # warm-up
    torch.cuda.synchronize()
    B.profile_read()
    B.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    comp, info = B.compress(params, 3, contrib, VQ_RATIO, VQ_K, VQ_ITERS, u, method=1)
    e1.record()
    torch.cuda.synchronize()
    B.profile_enable(False)
    compress_ms = e0.elapsed_time(e1)
    prof = B.profile_read()
    t_assign, n_assign = prof["vq_assign"]
    m = info["m"]
    C = 48
    flops = 2.0 * m * VQ_K * C
    ms_launch = t_assign / max(n_assign, 1)
    peak = measured_peak("bf16_tflops")
    achieved = flops / (ms_launch * 1e-3) / 1e12
    obj = info["objective"].cpu().numpy()
    # renders: compressed against FP32, the 4 views
    csc = B.CompressedScene(comp)
    res = {}
    for name, scn in (("fp32", tr.scene), ("compressed", csc)):
        for _ in range(3):
            for cam, _, _ in views:
                scn.render(cam, save=False)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            for cam, _, _ in views:
                scn.render(cam, save=False)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / (5 * len(views))
    rows = comp["sh_table"].shape[0]
    bytes_fp32 = n * (3 + 4 + 2 + 1 + C) * 4
    bytes_comp = n * (12 + 8 + 4 + 2 + 4) + rows * C * 2
    csc.close()
    return {"surfels": n, "quantised": m, "K": VQ_K, "ratio": VQ_RATIO, "iters": VQ_ITERS,
            "compress_ms": round(compress_ms, 2), "assign_launches": n_assign,
            "objective_first": float(obj[0]), "objective_last": float(obj[-1]),
            "render_ms_per_view_fp32": round(res["fp32"], 4),
            "render_ms_per_view_compressed": round(res["compressed"], 4),
            "bytes_fp32": bytes_fp32, "bytes_compressed": bytes_comp,
            "roofline": {"kernel": "vq_assign_tc_kernel", "bound": "tensor", "achieved": round(achieved, 2),
                         "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "ms_per_launch": round(ms_launch, 4),
                         "peak_source": "measured dense bf16 (binary16 has the same nominal tensor rate)"}}


VIS_POINTS, VIS_VIEWS = 31_400_000, 958


def measure_visibility(scene_np, dev, args):
    """Visible frequency of points (Sec. 4 crop volume estimation) at the
    paper's scale: 31.4M points on the city block's surfaces (the surfel
    centres repeated with a jitter of half their spacing) and 958 views at
    1920x1080 on 150-250 m orbits, each point an isotropic Gaussian of 0.1 m.
    Timed with CUDA events after one warm-up call."""
    import numpy as np
    import torch
    from paper_2411_00771_gb300 import binding as B
    from paper_2411_00771_gb300 import synthetic as syn
    rng = np.random.default_rng(20241101 + 9)
    mu = torch.from_numpy(np.ascontiguousarray(scene_np["mu"], np.float32)).to(dev)
    reps = -(-VIS_POINTS // mu.shape[0])
    pts = mu.repeat(reps, 1)[:VIS_POINTS]
    g = torch.Generator(device=dev).manual_seed(20241101 + 10)
    pts += (torch.rand(pts.shape, device=dev, generator=g) - 0.5) * 0.5
    cams = [syn.orbit_camera(rng, 1920, 1080, radius=rng.uniform(150, 250), altitude=rng.uniform(150, 250))
            for _ in range(VIS_VIEWS)]
    counts = torch.zeros(VIS_POINTS, dtype=torch.int32, device=dev)
    B.visibility_count(pts, 0.1, cams, counts=counts)
    torch.cuda.synchronize()
    counts.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    B.visibility_count(pts, 0.1, cams, counts=counts)
    keep, zr = B.visibility_bounds(pts, counts, 3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pv = VIS_POINTS * VIS_VIEWS
    out = {"points": VIS_POINTS, "views": VIS_VIEWS, "resolution": [1920, 1080], "ms": round(ms, 3),
           "point_views_per_s": round(pv / (ms * 1e-3), 1), "mean_views_per_point": round(float(counts.float().mean()), 2),
           "kept_at_3": int(keep.sum().item()), "height_range": [round(float(v), 3) for v in zr.cpu()]}
    del pts, counts, keep
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
SERVE_RES = [(256, 256), (800, 600), (1600, 900), (1920, 1080), (3840, 2160)]


def run_serving(args, dev, scene1m, params1m, rank):
    """Served renders: 3 resident city scenes (1M, 4M, 10M surfels, SH 3),
    requests from 64 client threads with Poisson arrivals, each a random pose
    on a 150-250 m orbit and a resolution drawn from SERVE_RES.  Reports the
    one-request-at-a-time throughput on the same request stream, then the
    continuous-batching server at 0.5x, 0.9x and 1.2x that rate and
    saturated, with p50/p99 latency from submission to completion."""
    import numpy as np
    import torch

    from paper_2411_00771_gb300 import binding as B
    from paper_2411_00771_gb300 import synthetic as syn

    rng = np.random.default_rng(20241101 + 4)
    scenes = [scene1m]
    keep = [params1m]
    for n, ext, nb in ((4_000_000, (500.0, 500.0), 200), (10_000_000, (1000.0, 1000.0), 800)):
        s_np, _ = syn.city_scene(seed=20241101 + 40 + n // 1_000_000, n=n, extent=ext, n_boxes=nb)
        Pn = {k: torch.from_numpy(np.ascontiguousarray(s_np[k], np.float32)).to(dev)
              for k in ("mu", "quat", "scale", "opacity", "sh")}
        keep.append(Pn)
        scenes.append(B.Scene(Pn["mu"], Pn["quat"], Pn["scale"], Pn["opacity"], Pn["sh"], 3))
        del s_np

    def make_req():
        sid = int(rng.integers(3))
        W, H = SERVE_RES[int(rng.integers(len(SERVE_RES)))]
        az = rng.uniform(0, 2 * math.pi)
        r = rng.uniform(150.0, 250.0)
        ext = 250.0 if sid < 2 else 500.0
        tgt = (rng.uniform(-0.3, 0.3) * ext, rng.uniform(-0.3, 0.3) * ext, 0.0)
        cam = syn.look_at((tgt[0] + r * math.cos(az), tgt[1] + r * math.sin(az), rng.uniform(150.0, 250.0)),
                          tgt, W, H, 0.5 * W / math.tan(math.radians(30.0)))
        return sid, cam

    reqs = [make_req() for _ in range(400)]
    outs = {}

    def out_for(key, cam):
        if key not in outs:
            outs[key] = torch.empty((12, cam["height"], cam["width"]), device=dev)
        return outs[key]

    # one request at a time: render, wait, next
    for sid, cam in reqs[:5]:
        scenes[sid].render(cam, out=out_for(("seq", cam["width"]), cam), save=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_lat = []
    nseq = 0
    for sid, cam in reqs:
        a = time.perf_counter()
        scenes[sid].render(cam, out=out_for(("seq", cam["width"]), cam), save=False)
        torch.cuda.synchronize()
        seq_lat.append((time.perf_counter() - a) * 1e3)
        nseq += 1
        if time.perf_counter() - t0 > args.serving_seconds:
            break
    seq_vps = nseq / (time.perf_counter() - t0)

    free, _ = torch.cuda.mem_get_info(dev)
    srv = B.Server(budget_bytes=int(0.7 * free), max_slots=8)
    ids = [srv.add_scene(s) for s in scenes]

    def run(rate, duration, clients=64):
        stop_at = time.perf_counter() + duration
        srv.stats(reset=True)
        done = [0]
        lock = threading.Lock()

        def client(c):
            crng = np.random.default_rng(1000 + c)
            i = c
            while time.perf_counter() < stop_at:
                if rate:
                    time.sleep(crng.exponential(clients / rate))
                sid, cam = reqs[i % len(reqs)]
                i += clients
                t = srv.submit(ids[sid], cam, out_for(("c", c, cam["width"]), cam))
                srv.wait(t, 600000)
                with lock:
                    done[0] += 1

        th = [threading.Thread(target=client, args=(c,)) for c in range(clients)]
        a = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        el = time.perf_counter() - a
        st = srv.stats()
        return {"offered_views_per_s": round(rate, 2) if rate else None,
                "views_per_s": round(done[0] / el, 2), "completed": done[0],
                "p50_ms": round(st["latency_p50_ms"], 3), "p99_ms": round(st["latency_p99_ms"], 3),
                "views_per_blend_launch": round(st["batched_views"] / max(1, st["batches"]), 2)}

    runs = {"saturated": run(None, args.serving_seconds)}
    for f in (0.5, 0.9, 1.2):
        runs[f"{f}x"] = run(f * seq_vps, args.serving_seconds / 2)
    srv.close()
    seq_sorted = sorted(seq_lat)
    return {"scenes_surfels": [1_000_000, 4_000_000, 10_000_000], "resolutions": SERVE_RES,
            "clients": 64, "one_at_a_time": {"views_per_s": round(seq_vps, 2),
                                             "p50_ms": round(seq_sorted[len(seq_sorted) // 2], 3),
                                             "p99_ms": round(seq_sorted[int(0.99 * (len(seq_sorted) - 1))], 3)},
            "served": runs, "p50_ms": runs["0.9x"]["p50_ms"], "p99_ms": runs["0.9x"]["p99_ms"],
            "speedup_saturated": round(runs["saturated"]["views_per_s"] / seq_vps, 3)}


# ---------------------------------------------------------------------------
def crop_camera(cam, y0, h):
    c = dict(cam)
    c["cy"] = cam["cy"] - y0
    c["height"] = h
    return c


def time_oracle_crop(scene, cam, tgt, tinv, rows):
    """fwd + loss + bwd of the oracle on rows [y0, y0 + rows) of the view."""
    import numpy as np

    import oracle
    H = cam["height"]
    y0 = (H - rows) // 2
    cc = crop_camera(cam, y0, rows)
    t0 = time.perf_counter()
    r = oracle.render(scene, cc)
    L = oracle.loss(r["out"], np.ascontiguousarray(tgt[:, y0:y0 + rows]),
                    np.ascontiguousarray(tinv[y0:y0 + rows]), WEIGHTS)
    oracle.backward(scene, cc, L["adj"])
    return time.perf_counter() - t0


def time_oracle_per_surfel(scene, cam):
    import oracle
    t0 = time.perf_counter()
    oracle.preprocess(scene, cam)
    return time.perf_counter() - t0


def cpu_baseline(scene, cam, tgt, tinv, budget_s=15.0):
    """The oracle as it stands on the host cores: whole views of the workload
    (render + loss + backward), repeated until about budget_s seconds of CPU
    work; the mean per view.  If one view would take far longer than the
    budget (a slow host), a crop of the view is timed instead and scaled to
    the full view (per-pixel work by the row count, the per-surfel
    preprocess, which the oracle runs twice per step, once)."""
    import statistics as st

    import oracle
    H = cam["height"]
    t_pre = time_oracle_per_surfel(scene, cam)
    t8 = time_oracle_crop(scene, cam, tgt, tinv, 8)
    per_row = max((t8 - 2 * t_pre) / 8, 1e-6)
    if 2 * t_pre + per_row * H <= 2 * budget_s:
        times = [time_oracle_crop(scene, cam, tgt, tinv, H)]
        while sum(times) < budget_s and len(times) < 8:
            times.append(time_oracle_crop(scene, cam, tgt, tinv, H))
        v = st.mean(times)
        return {"value": round(v * 1e3, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"FP64 oracle render+loss+backward of {len(times)} whole {cam['width']}x{H} views "
                          f"({sum(times):.1f} s), mean per view"}
    rows2 = int(min(H, max(8, (budget_s - 2 * t_pre) / per_row)))
    t2 = time_oracle_crop(scene, cam, tgt, tinv, rows2)
    per_row = max((t2 - 2 * t_pre) / rows2, 1e-6)
    est = 2 * t_pre + per_row * H
    return {"value": round(est * 1e3, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle render+loss+backward on a {cam['width']}x{rows2} crop of the "
                      f"{cam['width']}x{H} view ({t2:.1f} s); per-pixel work scaled x{H / rows2:.1f}, "
                      f"per-surfel preprocess ({t_pre:.2f} s, run twice) counted once each"}


def run_reference(args):
    world, rank, _ = rank_env()
    if rank != 0:  # the oracle runs once, on rank 0; the other ranks have no work
        return
    import oracle
    scene, cam, tgt, tinv = city_workload(0)
    H = cam["height"]
    total_budget = 150.0
    per_step = total_budget / (args.steps + max(args.warmup, 3))
    t_pre = time_oracle_per_surfel(scene, cam)
    t8 = time_oracle_crop(scene, cam, tgt, tinv, 8)
    per_row = max((t8 - 2 * t_pre) / 8, 1e-6)
    rows = int(min(H, max(1, (per_step - 2 * t_pre) / per_row)))
    vals = []
    for i in range(max(args.warmup, 3) + args.steps):
        t = time_oracle_crop(scene, cam, tgt, tinv, rows)
        if i >= max(args.warmup, 3):
            vals.append((2 * t_pre + max(t - 2 * t_pre, 0.0) / rows * H) * 1e3)
    v = statistics.mean(vals)
    sample = (f"FP64 oracle render+loss+backward on a {cam['width']}x{rows} crop per step, per-pixel "
              f"work scaled x{H / rows:.1f} to the {cam['width']}x{H} view")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cam["width"], H, world),
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
