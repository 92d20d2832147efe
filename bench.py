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
CPU oracle on whole views of the same workload on the host cores.
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
FP32_LANES = 128     # FP32 lanes per SM (Blackwell: 4 sub-partitions x 32)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}


def fp32_peak_tflops(sm_count, sm_max_mhz):
    """FP32 issue peak from unit counts and the clock: SMs (read from the
    device) x 128 FP32 lanes x 2 FLOPs (an FMA) x the maximum SM clock (the
    measured-peaks file's, else GB300's 2070 MHz)."""
    return sm_count * FP32_LANES * 2 * sm_max_mhz * 1e6 / 1e12


def stage_bytes(N, C, V, K, ntiles, npix, sh_coeffs=16, n_sets=3):
    """Algorithmic (compulsory) DRAM bytes per view of the HBM-bound stages,
    from the view's counts: N surfels, C candidates (kept by the cull), V
    visible surfels, K (surfel, tile) instances, npix pixels.
      preprocess: every surfel reads mu, q, s (36 B) and writes its tile rect
        and count (12 B); every candidate reads opacity and SH (4 + 12 k B for
        k SH coefficients per channel) and writes its blend record (112 B),
        footprint shape (56 B), depth key and index (8 B);
      order: per candidate 4 depth-sort passes of (key, value) read and
        written (64 B), the count gather and scan (16 B) and the emission's
        reads (order, offset, rect, footprint: 72 B); per instance the
        emitted (key, value) (8 B), 2 tile-sort passes (32 B) and the range
        scan's read (4 B); per tile the range (8 B) and the launch order
        (12 B);
      loss: per pixel the colour and inverse depth of the render and the
        target read (32 B), the total set's colour and inverse-depth
        adjoints and the SSIM and L1 sets' colour adjoints written (40 B);
      preprocess_bwd: per candidate its index and count (8 B); per visible
        surfel its gradient record (64 B) and parameters (232 B at degree 3)
        read and the five gradient arrays read and written (2 x 232 B);
      densify: per surfel the accumulation (rect 8 B, n_sets screen gradients
        8 B each, statistics read and written 32 B), the Eq. 2 selection
        (statistics read twice 32 B, scales 8 B, mask 1 B, g 4 B) and the
        elongation filter (scales 8 B, keep 1 B)."""
    P = 36 + 4 + 12 * sh_coeffs
    return {
        "preprocess": N * 48 + C * (4 + 12 * sh_coeffs + 112 + 56 + 8),
        "sort": C * (64 + 16 + 72) + K * (8 + 32 + 4) + ntiles * 20,
        "loss": npix * 72,
        "preprocess_bwd": C * 8 + V * (64 + 3 * P),
        "densify": N * (8 + 8 * n_sets + 32 + 32 + 8 + 1 + 4 + 8 + 1),
    }


def stage_roofline(info, stage_ms, n, npix, sm_count, sm_max_mhz, hbm_gbs):
    """Achieved rate of every stage of the step against its roofline: GB/s of
    algorithmic bytes against the measured HBM copy bandwidth for the
    HBM-bound stages, algorithmic FLOP/s against the FP32 issue peak for the
    two blends."""
    C, V, K = info["n_candidates"], info["n_visible"], info["n_instances"]
    ntiles = info["tiles_x"] * info["tiles_y"]
    out = {}
    for k, b in stage_bytes(n, C, V, K, ntiles, npix).items():
        ms = stage_ms.get(k, 0.0)
        if ms > 0:
            gbs = b / (ms * 1e-3) / 1e9
            out[k] = {"bound": "hbm", "bytes": int(b), "ms": round(ms, 4), "achieved": round(gbs, 1),
                      "unit": "GB/s", "peak": hbm_gbs, "frac": round(gbs / hbm_gbs, 4)}
    peak = fp32_peak_tflops(sm_count, sm_max_mhz)
    E, Bl, R = info["pairs_evaluated"], info["pairs_blended"], info["bwd_pairs_evaluated"]
    work = {"blend_fwd": FLOP_EVAL * E + FLOP_BLEND * Bl, "blend_bwd": FLOP_EVAL * R + FLOP_BWD_PAIR * Bl}
    for k, f in work.items():
        ms = stage_ms.get(k, 0.0)
        if ms > 0:
            tf = f / (ms * 1e-3) / 1e12
            out[k] = {"bound": "alu", "flops": int(f), "ms": round(ms, 4), "achieved": round(tf, 3),
                      "unit": "TFLOP/s", "peak": round(peak, 2), "frac": round(tf / peak, 4)}
    return out


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
BLEND_BWD_TRAFFIC = {"bytes": 182110720 + 11200000,
                     "sources_sha256": "9e2ec483cf2f2ccf617b3be5632442872007dd758d5f2653c7ac9ce78650129b"}


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
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1M-25M surfel 4K sweep")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
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

    def wait_first(self, timeout_s=20.0):
        """Block until the sampler has produced its first row (or timeout)."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.rows and time.perf_counter() - t0 < timeout_s:
            if self.proc.poll() is not None:
                break
            time.sleep(0.02)
        return bool(self.rows)

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


def step_time_summary(per_step_ms, host_ms):
    """Per-step device times (CUDA events at every step boundary) and the
    host's wall time of the same loop, per step."""
    xs = sorted(per_step_ms)
    n = len(xs)
    return {"median_ms": round(xs[n // 2], 4) if n else None, "min_ms": round(xs[0], 4) if n else None,
            "max_ms": round(xs[-1], 4) if n else None,
            "host_wall_ms_per_step": round(host_ms / n, 4) if n else None}


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

    # the clock sampler starts (and has taken its first sample, so that
    # nvidia-smi's start-up is over) before the warm-up: nothing starts
    # inside the timed region
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    clocks.wait_first(timeout_s=20.0)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    l0 = B.kernel_launches()
    # one event per step boundary: the per-step times show a stall, if any
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    t_host = time.perf_counter()
    evs[0].record()
    for i in range(args.steps):
        step()
        evs[i + 1].record()
    torch.cuda.synchronize()
    host_ms = (time.perf_counter() - t_host) * 1e3
    barrier()
    clk = clocks.stop()
    launches = B.kernel_launches() - l0
    ms_step = evs[0].elapsed_time(evs[-1]) / args.steps
    step_times = step_time_summary([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)], host_ms)
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
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = measured_peak("sm_max_mhz")
    fp32_peak = fp32_peak_tflops(sm_count, sm_max_mhz)
    achieved = work[dom] / (per_launch[dom] * 1e-3) / 1e12
    roofline = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4),
                "traffic": (blend_bwd_traffic() if dom == "blend_bwd" and W == 1600 and H == 900 else None),
                "ms_per_launch": round(per_launch[dom], 4),
                "peak_source": f"{sm_count} SMs (device) x {FP32_LANES} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz "
                               f"(unit counts and the maximum SM clock)"}
    # per step: a group may record several scopes per step (the sort group
    # covers every scan, radix pass, emit and range pass of a render)
    breakdown = {k: round(v[0] / args.steps, 4) for k, v in prof.items()}
    stages = stage_roofline(info, {k: v[0] / args.steps for k, v in prof.items()}, n, W * H, sm_count,
                            sm_max_mhz, measured_peak("hbm_gbs"))

    contribution = measure_contribution(sc, cam, n, dev, args)
    sweep = None if args.no_sweep else measure_sweep(dev, args)
    visibility = measure_visibility(scene_np, dev, args)
    training, vq = (None, None) if args.no_training else measure_training(dev, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene_np, cam, tgt_np, tinv_np, budget_s=20.0)
        # the same oracle on one core (a crop, scaled), and the small case
        # (2,000 surfels at 128x128) on all cores and on one
        cpu["one_core"] = oracle_child("city:48", 1)
        cpu["small_case"] = {"all_cores": oracle_child("small", os.cpu_count() or 1),
                             "one_core": oracle_child("small", 1)}
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
            "step_times": step_times,
            "roofline": roofline,
            "stage_ms": breakdown,
            "stage_roofline": stages,
            "work": {"instances": info["n_instances"], "visible": info["n_visible"],
                     "pairs_evaluated": E, "pairs_blended": Bl, "bwd_pairs_replayed": R,
                     "bwd_warp_steps": info["bwd_warp_entries"],
                     "bwd_lanes_per_step": round(info["bwd_warp_lanes"] / max(1, info["bwd_warp_entries"]), 2)},
            "clocks": clk,
            "cpu_baseline": cpu,
            "contribution": contribution,
            "visibility": visibility,
            "large_scene": sweep,
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


SWEEP_N = (1_000_000, 2_000_000, 4_000_000, 8_000_000, 16_000_000, 25_000_000)


def measure_sweep(dev, args):
    """Large-scene stress: the city distribution on a 500 m x 2 km strip
    (800 buildings, 25M surfels, SH 3) seen at 3840x2160 from 250 m.  Forward
    renders of its 1M..25M prefixes (a prefix of the area-sampled surfels is a
    uniform subsample): ms/view timed with CUDA events (profiling off), then a
    profiling pass for the per-stage times and their roofline fractions, and
    contributors per pixel; and the training step (render, loss, backward,
    densification statistics and filters) of the whole 25M scene at 4K, with
    seeded uniform targets (the analytic ray cast of 800 buildings at 4K costs
    minutes of host time)."""
    import numpy as np
    import torch
    from paper_2411_00771_gb300 import binding as B
    from paper_2411_00771_gb300 import synthetic as syn
    scene, _ = syn.city_scene(n=SWEEP_N[-1], extent=(500.0, 2000.0), n_boxes=800)
    cam = syn.aerial_camera(width=3840, height=2160, altitude=250.0, azimuth_deg=-90.0)
    P = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
         for k in ("mu", "quat", "scale", "opacity", "sh")}
    del scene
    H, W = cam["height"], cam["width"]
    out = torch.empty((12, H, W), device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    rows = []
    for n in SWEEP_N:
        sc = B.Scene(P["mu"][:n], P["quat"][:n], P["scale"][:n], P["opacity"][:n], P["sh"][:n], 3)
        for _ in range(2):
            sc.render(cam, out=out, save=False)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sc.render(cam, out=out, save=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        B.profile_read()
        B.profile_enable(True)
        for _ in range(reps):
            sc.render(cam, out=out, save=False)
        torch.cuda.synchronize()
        B.profile_enable(False)
        prof = {k: v[0] / reps for k, v in B.profile_read().items()}
        _, fr = sc.render(cam, out=out)
        info = fr.info()
        fr.release()
        st = stage_roofline(info, prof, n, W * H, sm_count, measured_peak("sm_max_mhz"), measured_peak("hbm_gbs"))
        rows.append({"surfels": n, "ms_per_view": round(ms, 4), "visible": info["n_visible"],
                     "instances": info["n_instances"],
                     "contributors_per_pixel": round(info["pairs_blended"] / (W * H), 2),
                     "evaluated_per_pixel": round(info["pairs_evaluated"] / (W * H), 2),
                     "stages": {k: {"ms": v["ms"], "achieved": v["achieved"], "unit": v["unit"], "frac": v["frac"]}
                                for k, v in st.items() if k in ("preprocess", "sort", "blend_fwd")}})
        sc.close()
    # fwd + bwd of the whole scene at 4K
    n = SWEEP_N[-1]
    sc = B.Scene(P["mu"], P["quat"], P["scale"], P["opacity"], P["sh"], 3)
    g = torch.Generator(device=dev).manual_seed(20241101 + 5)
    tgt = torch.rand((3, H, W), device=dev, generator=g)
    tinv = torch.rand((H, W), device=dev, generator=g) * 0.01
    adj = [torch.zeros((11, H, W), device=dev) for _ in range(3)]
    losses = torch.empty(4, device=dev)
    grads = {k: torch.zeros_like(v) for k, v in P.items()}
    screen = torch.zeros((3, n, 2), device=dev)
    stats = torch.zeros((n, 4), device=dev)

    def step():
        o, fr = sc.render(cam, out=out)
        B.loss(o, tgt, tinv, WEIGHTS, adj_total=adj[0], adj_ssim=adj[1], adj_l1=adj[2], losses=losses)
        for v in grads.values():
            v.zero_()
        screen.zero_()
        sc.backward(fr, adj, [0x7 | (1 << 5), 0x7, 0x7], grads, screen)
        sc.densify_accumulate(fr, screen, stats)
        B.densify_select(stats, P["scale"], OMEGA, GRAD_THR, ETA_THR)
        B.elongation_filter(P["scale"], ETA_THR)
        return fr

    for _ in range(2):
        step().release()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        step().release()
    e1.record()
    torch.cuda.synchronize()
    fb = e0.elapsed_time(e1) / 3
    fr = step()
    info = fr.info()
    fr.release()
    sc.close()
    del P, grads, screen, stats, adj, out
    torch.cuda.empty_cache()
    return {"scene": "city strip 500 m x 2 km, 800 buildings, SH 3", "resolution": [W, H],
            "forward": rows,
            "fwd_bwd_25m": {"ms_per_view": round(fb, 3), "contributors_per_pixel": round(info["pairs_blended"] / (W * H), 2),
                            "bwd_pairs_replayed": info["bwd_pairs_evaluated"], "targets": "seeded uniform"}}


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


class FifoRenderer:
    """One request at a time: a FIFO queue served by one thread that renders
    each request to completion (gs_render, then a stream synchronise) before
    taking the next; the same submit/wait interface as the server."""

    def __init__(self, scenes):
        import queue
        self.scenes = scenes
        self.q = queue.Queue()
        self.lat = []
        self.lock = threading.Lock()
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        import torch
        while True:
            item = self.q.get()
            if item is None:
                return
            sid, cam, out, t_sub, ev = item
            self.scenes[sid].render(cam, out=out, save=False)
            torch.cuda.synchronize()
            with self.lock:
                self.lat.append((time.perf_counter() - t_sub) * 1e3)
            ev.set()

    def submit(self, sid, cam, out):
        ev = threading.Event()
        self.q.put((sid, cam, out, time.perf_counter(), ev))
        return ev

    def wait(self, ev, timeout_ms):
        ev.wait(timeout_ms / 1e3)

    def stats(self, reset=False):
        with self.lock:
            xs = sorted(self.lat)
            if reset:
                self.lat = []
        n = len(xs)
        return {"latency_p50_ms": xs[n // 2] if n else 0.0,
                "latency_p99_ms": xs[int(0.99 * (n - 1))] if n else 0.0,
                "batched_views": n, "batches": n}

    def close(self):
        self.q.put(None)
        self.th.join(timeout=10)


def run_serving(args, dev, scene1m, params1m, rank):
    """Served renders: 3 resident city scenes (1M, 4M, 10M surfels, SH 3),
    requests from 64 client threads, each a random pose on a 150-250 m orbit
    and a resolution drawn from SERVE_RES.  Every client loops: an
    exponentially distributed think time (mean 64 / rate, so that 64 clients
    offer `rate` views/s when answers are instant), submit, wait.  The same
    client population runs against one-request-at-a-time rendering (a FIFO
    served by one thread, FifoRenderer) and against the continuous-batching
    server, at 0.5x, 0.9x and 1.2x the one-at-a-time capacity (its rate with
    no think time) and saturated (no think time); both report completed
    views/s and p50/p99 latency from submission to completion.  The server's
    batched blend launches are also timed through the library's profiling
    events for their FP32 roofline."""
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

    # capacity of one-at-a-time rendering: the request stream back to back
    for sid, cam in reqs[:5]:
        scenes[sid].render(cam, out=out_for(("seq", cam["width"]), cam), save=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nseq = 0
    for sid, cam in reqs:
        scenes[sid].render(cam, out=out_for(("seq", cam["width"]), cam), save=False)
        torch.cuda.synchronize()
        nseq += 1
        if time.perf_counter() - t0 > args.serving_seconds / 2:
            break
    seq_vps = nseq / (time.perf_counter() - t0)

    def run(srv, ids, rate, duration, clients=64):
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
                "views_per_blend_launch": round(st["batched_views"] / max(1, st["batches"]), 2),
                "_pairs": (st.get("pairs_evaluated", 0), st.get("pairs_blended", 0))}

    loads = [("saturated", None), ("0.5x", 0.5), ("0.9x", 0.9), ("1.2x", 1.2)]
    fifo = FifoRenderer(scenes)
    one = {}
    for name, f in loads:
        one[name] = run(fifo, [0, 1, 2], f * seq_vps if f else None, args.serving_seconds / 2)
    fifo.close()

    free, _ = torch.cuda.mem_get_info(dev)
    srv = B.Server(budget_bytes=int(0.7 * free), max_slots=16)
    ids = [srv.add_scene(s) for s in scenes]
    runs = {}
    for name, f in loads:
        if name == "saturated":
            B.profile_read()
            B.profile_enable(True)
        runs[name] = run(srv, ids, f * seq_vps if f else None, args.serving_seconds if f is None else
                         args.serving_seconds / 2)
        if name == "saturated":
            B.profile_enable(False)
            prof = B.profile_read()
    srv.close()
    t_blend, n_blend = prof.get("blend_fwd", (0.0, 0))
    E, Bl = runs["saturated"]["_pairs"]
    for r in list(one.values()) + list(runs.values()):
        r.pop("_pairs", None)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sm_count, measured_peak("sm_max_mhz"))
    tf = (FLOP_EVAL * E + FLOP_BLEND * Bl) / max(t_blend * 1e-3, 1e-12) / 1e12
    return {"scenes_surfels": [1_000_000, 4_000_000, 10_000_000], "resolutions": SERVE_RES,
            "clients": 64, "capacity_one_at_a_time_views_per_s": round(seq_vps, 2),
            "one_at_a_time": one, "served": runs,
            "p50_ms": runs["0.9x"]["p50_ms"], "p99_ms": runs["0.9x"]["p99_ms"],
            "speedup": {k: round(runs[k]["views_per_s"] / max(one[k]["views_per_s"], 1e-9), 3) for k, _ in loads},
            "saturated_blend_launches": {"launches": n_blend, "ms": round(t_blend, 2),
                                         "ms_per_launch": round(t_blend / max(n_blend, 1), 4)},
            "roofline": {"kernel": "blend_fwd_batched (saturated run)", "bound": "alu", "achieved": round(tf, 3),
                         "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(tf / peak, 4),
                         "pairs_evaluated": int(E), "pairs_blended": int(Bl)}}


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
    """The oracle as it stands, on the host cores, on the same workload: each
    step renders, takes the loss of and differentiates one whole 1600x900
    view.  Only if whole views would not fit about five minutes for the
    whole run (a slow host) is a crop timed per step and scaled to the
    view, which the line then says."""
    world, rank, _ = rank_env()
    if rank != 0:  # the oracle runs once, on rank 0; the other ranks have no work
        return
    import oracle
    scene, cam, tgt, tinv = city_workload(0)
    H = cam["height"]
    warm = max(args.warmup, 3)
    total_budget = 300.0
    t0 = time.perf_counter()
    t_first = time_oracle_crop(scene, cam, tgt, tinv, H)  # the first warm-up step
    vals = []
    if t_first * (warm + args.steps) <= total_budget:
        for i in range(1, warm + args.steps):
            t = time_oracle_crop(scene, cam, tgt, tinv, H)
            if i >= warm:
                vals.append(t * 1e3)
        sample = f"FP64 oracle render+loss+backward of one whole {cam['width']}x{H} view per step"
    else:
        per_step = max(total_budget - (time.perf_counter() - t0), 30.0) / (warm + args.steps)
        t_pre = time_oracle_per_surfel(scene, cam)
        per_row = max((t_first - 2 * t_pre) / H, 1e-6)
        rows = int(min(H, max(1, (per_step - 2 * t_pre) / per_row)))
        for i in range(1, warm + args.steps):
            t = time_oracle_crop(scene, cam, tgt, tinv, rows)
            if i >= warm:
                vals.append((2 * t_pre + max(t - 2 * t_pre, 0.0) / rows * H) * 1e3)
        sample = (f"FP64 oracle render+loss+backward on a {cam['width']}x{rows} crop per step, per-pixel "
                  f"work scaled x{H / rows:.1f} to the {cam['width']}x{H} view (whole views would not fit "
                  f"the run's time)")
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": warm,
            "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cam["width"], H, world),
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line), flush=True)


def oracle_sample(spec):
    """Child-process leg of the CPU baseline (run with OMP_NUM_THREADS set by
    the parent): times the oracle on one sample and prints one JSON object.
    spec "city:<rows>" = render+loss+backward of a centred crop of <rows>
    rows of the 1600x900 city view, scaled to the whole view; "small" = the
    2,000-surfel 128x128 case (fwd + L1 loss + bwd), whole."""
    import numpy as np

    import oracle
    from paper_2411_00771_gb300 import synthetic as syn
    if spec == "small":
        scene, cam, tgt, _ = syn.tiny_scene()
        times = []
        t_all = time.perf_counter()
        while time.perf_counter() - t_all < 2.0 or len(times) < 3:
            a = time.perf_counter()
            r = oracle.render(scene, cam)
            L = oracle.loss(r["out"], tgt, None, (1.0, 0.0, 0.0))
            oracle.backward(scene, cam, L["adj"][:1])
            times.append(time.perf_counter() - a)
        res = {"ms_per_view": round(1e3 * statistics.median(times), 3), "views": len(times),
               "sample": "2,000 surfels, 128x128, SH 0, L1 loss: render+loss+backward, whole view"}
    else:
        rows = int(spec.split(":")[1])
        scene, cam, tgt, tinv = city_workload(0)
        H = cam["height"]
        t_pre = time_oracle_per_surfel(scene, cam)
        t = time_oracle_crop(scene, cam, tgt, tinv, rows)
        est = 2 * t_pre + max(t - 2 * t_pre, 0.0) / rows * H
        res = {"ms_per_view": round(est * 1e3, 1),
               "sample": f"a {cam['width']}x{rows} crop ({t:.1f} s), per-pixel work scaled x{H / rows:.1f}, "
                         f"the per-surfel preprocess ({t_pre:.2f} s, run twice per step) counted once each"}
    res["cores"] = oracle.num_threads()
    print(json.dumps(res), flush=True)


def oracle_child(spec, threads, timeout_s=300):
    """Run oracle_sample(spec) in a fresh process with `threads` OpenMP threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec], env=env,
                           capture_output=True, text=True, timeout=timeout_s)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the baseline is context
        return {"error": f"{type(e).__name__}: {e}"[:200]}


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(args.oracle_sample)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
