"""Throughput benchmark of the stitching path on GB300.

One step = one frame set of the workload stitched through the C ABI (warp, feather weights,
pyramids, blend, collapse, uint8 output).  Frames are distinct, device-resident buffers of a
seeded synthetic sequence (every frame set is larger than L2).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 8x4k|4x1080p|2cam]
                    [--path fused|plain] [--fp16-bands] [--impl ours|reference]

N > 1 runs under torchrun: the path does not exchange data, so every rank stitches its own copy of
the workload (replicas) and ``value`` sums all ranks' output over the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle on host cores on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    "8x4k": lambda frames: synth.config_8x4k(frames=frames),
    "4x1080p": lambda frames: synth.config_4x1080p(frames=frames),
    "2cam": lambda frames: synth.config_2cam(),
}
DEFAULT_FRAMES = {"8x4k": 30, "4x1080p": 60, "2cam": 1}
METRIC = "stitched output MPix/s and frames/s on 1 GB300; % of HBM roofline vs plain path"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def compulsory_bytes(cfg) -> int:
    """Algorithmic bytes of one frame set: every source pixel read once (3 B) and every canvas pixel
    written once (3 B, uint8 RGB)."""
    src = sum(c.width * c.height * 3 for c in cfg.cameras)
    return src + cfg.canvas_w * cfg.canvas_h * 3


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(cfg, frames0, budget_s: float = 15.0):
    """Time the FP64 oracle on host cores on square windows of the workload's canvas (bounded)."""
    import oracle
    wins = []
    side = 256
    Wc, Hc = cfg.canvas_w, cfg.canvas_h
    rng = np.random.default_rng(0)
    t_total, px_total = 0.0, 0
    while t_total < budget_s and len(wins) < 64:
        s = min(side, Wc, Hc)
        w = (int(rng.integers(0, Wc - s + 1)), int(rng.integers(0, Hc - s + 1)), s, s)
        t0 = time.perf_counter()
        oracle.forward(cfg.cameras, frames0, Wc, Hc, cfg.levels, window=w)
        t_total += time.perf_counter() - t0
        px_total += s * s
        wins.append(w)
    return {"value": px_total / 1e6 / t_total, "unit": "MPix/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{len(wins)} windows of {side}x{side} canvas px of the {cfg.name} rig "
                      f"(each with its full pyramid dependency region), {t_total:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cfg = WORKLOADS[args.workload](1)
    frames0 = cfg.frame(0)
    # one step = a bounded sample of the workload: one 256x256 canvas window per step
    side = min(256, cfg.canvas_w, cfg.canvas_h)
    rng = np.random.default_rng(1)

    def step():
        w = (int(rng.integers(0, cfg.canvas_w - side + 1)), int(rng.integers(0, cfg.canvas_h - side + 1)), side, side)
        oracle.forward(cfg.cameras, frames0, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=w)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    mpix = side * side / 1e6
    value = mpix * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MPix/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg.name, "canvas": [cfg.canvas_w, cfg.canvas_h], "cameras": len(cfg.cameras),
                   "levels": cfg.levels, "step_sample": f"{side}x{side} canvas window"},
        "cpu_baseline": {"value": value, "unit": "MPix/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"one {side}x{side} window of the {cfg.name} canvas per step"},
        "e2e": {"value": value, "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="8x4k", choices=sorted(WORKLOADS))
    ap.add_argument("--frames", type=int, default=None, help="distinct frame sets (default: the sequence length)")
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--fp16-bands", action="store_true")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison run")
    ap.add_argument("--e2e-steps", type=int, default=5)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1810_03988_gb300 import Rig

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    nfr = args.frames or DEFAULT_FRAMES[args.workload]
    cfg = WORKLOADS[args.workload](nfr)
    t0 = time.perf_counter()
    host_frames = [cfg.frame(t) for t in range(nfr)]
    gen_s = time.perf_counter() - t0
    dframes = [[torch.from_numpy(f).to(dev) for f in fs] for fs in host_frames]
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(rig, out, steps, warmup, profile):
        for k in range(warmup):
            rig.stitch(dframes[k % nfr], out)
        torch.cuda.synchronize()
        if profile:
            rig.set_profiling(True)
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(steps):
            rig.stitch(dframes[(warmup + k) % nfr], out)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1) / steps
        kt = rig.kernel_times() if profile else {}
        if profile:
            rig.set_profiling(False)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, kt

    rig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=args.fp16_bands, path=args.path,
              device=local)
    info = rig.info()
    out = rig.new_output()
    clocks = ClockSampler(local)
    # warm-up and an unprofiled timing pass, then the profiled timed region that is reported
    timed(rig, out, max(1, min(args.steps, 5)), args.warmup, False)
    clocks.start()
    ms, kt = timed(rig, out, args.steps, 3, True)
    clk = clocks.stop()

    mpix = cfg.canvas_w * cfg.canvas_h / 1e6
    value = world * mpix / (ms / 1e3)
    fps = 1e3 / ms
    hbm_peak, peak_kind = _peaks()
    cbytes = compulsory_bytes(cfg)

    # dominant kernel and its roofline
    dom = max(kt.items(), key=lambda kv: kv[1][0]) if kt else None
    roof = None
    if dom:
        name, (tot_ms, launches) = dom
        per_launch_ms = tot_ms / launches
        alg = kernel_algorithmic_bytes(name, cfg, info, launches // args.steps if args.steps else 1)
        achieved = alg / (per_launch_ms / 1e3) / 1e9 if alg else None
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None, "traffic": None,
                "peak_source": f"{peak_kind} hbm_gbs (copy)", "avg_launch_ms": per_launch_ms,
                "launches_per_step": launches / args.steps,
                "share": tot_ms / sum(v[0] for v in kt.values()),
                "algorithmic_bytes_per_launch": alg}
    step_roof = {"achieved": cbytes / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "frac": cbytes / (ms / 1e3) / 1e9 / hbm_peak, "compulsory_bytes_per_step": cbytes}

    plain = None
    if args.path == "fused" and not args.no_plain:
        prig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path="plain", device=local)
        pms, _ = timed(prig, out, max(3, min(args.steps, 10)), 3, False)
        plain = {"value": world * mpix / (pms / 1e3), "ms_per_step": pms,
                 "hbm_frac": cbytes / (pms / 1e3) / 1e9 / hbm_peak, "speedup_fused_over_plain": pms / ms}
        prig.close()

    # end to end through the host-buffer entry point: H2D of the frames, stitch, D2H of the canvas
    pinned = [[torch.from_numpy(f).pin_memory() for f in fs] for fs in host_frames[:min(nfr, 4)]]
    hout = torch.empty((cfg.canvas_h, cfg.canvas_w, 3), dtype=torch.uint8).pin_memory()
    rig.stitch_host(pinned[0], hout)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        rig.stitch_host(pinned[k % len(pinned)], hout)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = sum(c.width * c.height * 3 for c in cfg.cameras)
    d2h = cfg.canvas_w * cfg.canvas_h * 3
    e2e = {"value": world * mpix / e2e_s, "unit": "MPix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_s * 1e3, "steps": args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, host_frames[0])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MPix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "frames_per_s": world * fps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg.name, "cameras": len(cfg.cameras),
                       "camera_size": [cfg.cameras[0].width, cfg.cameras[0].height],
                       "canvas": [cfg.canvas_w, cfg.canvas_h], "levels": cfg.levels, "sequence_frames": nfr,
                       "path": args.path, "bands": "fp16" if args.fp16_bands else "fp32", "output": "uint8 RGB",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: each frame set is a distinct device buffer "
                             f"({cbytes / 1e6:.0f} MB compulsory traffic per step)"},
            "roofline": roof, "step_roofline": step_roof, "plain_path": plain, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk, "gpu_launches": info["num_kernels"] * args.steps,
            "rig": {"scratch_bytes": info["scratch_bytes"], "roi_pixels": info["roi_pixels"],
                    "kernels_per_step": info["num_kernels"], "tiles": info["tiles"]},
            "kernel_times_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in kt.items()},
            "frame_generation_s": gen_s,
        }
        print(json.dumps(line))
    rig.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def kernel_algorithmic_bytes(name: str, cfg, info: dict, launches_per_step: int) -> float | None:
    """Algorithmic (compulsory) bytes of one launch of a kernel: the source pixels it must read and
    the canvas pixels it must write, split evenly over its launches in a step.  Kernels that only
    move intermediates have no compulsory bytes of their own and report the step's compulsory bytes
    over their launches (a lower bound on what the path must move)."""
    cb = compulsory_bytes(cfg)
    return cb / max(1, launches_per_step)


if __name__ == "__main__":
    sys.exit(main())
