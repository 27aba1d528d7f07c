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
    "cyl4x720p": lambda frames: synth.config_cyl(frames=frames),
}
DEFAULT_FRAMES = {"8x4k": 30, "4x1080p": 60, "2cam": 1, "cyl4x720p": 30}
METRIC = "stitched output MPix/s and frames/s on 1 GB300; % of HBM roofline vs plain path"


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time: every rank contributes its value, all receive the maximum."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def frame_percentiles(ms) -> dict:
    """Median, 10th and 90th percentile (nearest rank) of per-frame times in ms."""
    s = sorted(ms)
    if not s:
        return {}
    rank = lambda q: s[min(len(s) - 1, max(0, int(np.ceil(q * len(s))) - 1))]
    return {"p10": rank(0.1), "median": statistics.median(s), "p90": rank(0.9), "frames": len(s)}


def job_value(units_per_step_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes the same units per step (replicas), over the
    slowest rank's step time."""
    return world * units_per_step_per_rank / (ms_per_step / 1e3)


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
        self.begin = self.end = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0:  # wait for the first sample
            time.sleep(0.02)

    def mark_begin(self):
        self.begin = len(self.lines)

    def mark_end(self):
        time.sleep(0.05)  # let samples taken inside the region arrive
        self.end = len(self.lines)

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
        sel = self.lines[self.begin:self.end] if self.begin is not None and self.end is not None else []
        in_region = len(sel)
        if not sel:
            sel = self.lines[-3:]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in sel:
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
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": in_region}


def cpu_baseline(cfg, frames0, budget_s: float = 10.0):
    """Time the FP64 oracle on host cores on square windows of the workload's canvas, about
    `budget_s` seconds of oracle work."""
    import oracle
    wins = []
    side = 256
    Wc, Hc = cfg.canvas_w, cfg.canvas_h
    rng = np.random.default_rng(0)
    t_total, px_total = 0.0, 0
    while t_total < budget_s and len(wins) < 4096:
        s = min(side, Wc, Hc)
        w = (int(rng.integers(0, Wc - s + 1)), int(rng.integers(0, Hc - s + 1)), s, s)
        t0 = time.perf_counter()
        oracle.forward(cfg.cameras, frames0, Wc, Hc, cfg.levels, window=w, canvas=cfg.canvas)
        t_total += time.perf_counter() - t0
        px_total += s * s
        wins.append(w)
    return {"value": px_total / 1e6 / t_total, "unit": "MPix/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{len(wins)} windows of {side}x{side} canvas px of the {cfg.name} rig "
                      f"(each with its full pyramid dependency region), {t_total:.1f} s"}


def measure_lorb(torch, dframes, hframes, device: int, points: int = 500, reps: int = 20):
    """L-ORB on every view of one frame set (whole views as detection areas): ms per frame set and
    input MPix/s on the GPU (CUDA events, after warm-up), and the integer oracle on one view."""
    import oracle
    from paper_1810_03988_gb300 import LORB
    pat = synth.brief_pattern(0)
    H, W = dframes[0].shape[:2]
    areas = [(0, 0, W, H)]
    with LORB(W, H, points, device) as ctx:
        for _ in range(3):
            for f in dframes:
                ctx.detect(f, areas, pat, 20, 0, points)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            for f in dframes:
                ctx.detect(f, areas, pat, 20, 0, points)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    mpix = sum(f.shape[0] * f.shape[1] for f in dframes) / 1e6
    t0 = time.perf_counter()
    oracle.lorb(hframes[0], areas, pat, 20, 0, points)
    cpu_s = time.perf_counter() - t0
    return {"value": mpix / (ms / 1e3), "unit": "MPix/s", "ms_per_frame_set": ms, "views": len(dframes),
            "points_per_view": points, "cpu_oracle": {"value": (W * H / 1e6) / cpu_s, "unit": "MPix/s",
                                                      "cores": oracle.threads(), "sample": "one view"}}


def measure_accuracy(torch, Rig, cfg, frames0, dframes0, out_u8, device: int, n_random: int = 16):
    """Error of the stitched canvas against the FP64 oracle on sampled 256x256 windows of frame 0:
    the windows centred between neighbouring cameras (blended regions) plus seeded random ones.
    FP32 bands (uint8 output: `out_u8` holds frame 0; float output from an out_float rig) and
    FP16 bands (float output)."""
    import oracle
    side = min(256, cfg.canvas_w, cfg.canvas_h)
    wins = []
    cx = []
    for c in cfg.cameras:
        if cfg.canvas is None:
            p = np.asarray(c.H, dtype=np.float64) @ [c.width / 2.0, c.height / 2.0, 1.0]
            cx.append(p[0] / p[2])
    cx.sort()
    for a, b in zip(cx[:-1], cx[1:]):
        x0 = int(min(max((a + b) / 2 - side / 2, 0), cfg.canvas_w - side))
        wins.append((x0, (cfg.canvas_h - side) // 2, side, side))
    rng = np.random.default_rng(7)
    for _ in range(n_random):
        wins.append((int(rng.integers(0, cfg.canvas_w - side + 1)), int(rng.integers(0, cfg.canvas_h - side + 1)),
                     side, side))
    ref = [oracle.forward(cfg.cameras, frames0, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=w, canvas=cfg.canvas)
           for w in wins]
    res = {"windows": len(wins), "window": f"{side}x{side}", "frame": 0,
           "placement": "one between each pair of neighbouring camera centres, the rest seeded random"}
    u8 = out_u8.cpu().numpy()
    d8 = [np.abs(u8[y:y + h, x:x + w].astype(np.int32) - r["u8"].astype(np.int32)) for (x, y, w, h), r in zip(wins, ref)]
    for fp16 in (False, True):
        frig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=fp16, out_float=True, device=device,
                   canvas=cfg.canvas)
        fo = frig.stitch(dframes0).cpu().numpy()
        torch.cuda.synchronize()
        frig.close()
        df = [float(np.abs(fo[y:y + h, x:x + w].astype(np.float64) - r["out"]).max()) for (x, y, w, h), r in zip(wins, ref)]
        key = "fp16_bands" if fp16 else "fp32"
        res[key] = {"max_abs_float": max(df), "bound_float": 1e-3 if fp16 else 2e-4}
        del fo
    res["fp32"].update({"u8_max_lsb": int(max(int(d.max()) for d in d8)),
                        "u8_frac_differing": float(sum(int((d > 0).sum()) for d in d8) / sum(d.size for d in d8)),
                        "bound_u8_lsb": 1})
    return res


def measure_backward(torch, device: int, reps: int = 20):
    """S7 on the differentiation workload (4 cameras 1920x1080, canvas 5200x1300, corners perturbed
    by +-3 px, gains in U[0.8, 1.2], camera 0 fixed): the backward call (overlap loss and the 9
    gradient entries of every camera) timed with CUDA events after warm-up, then 50 Adam steps of
    the refinement through it (wall clock, loss and corner error before and after).  The oracle's
    loss and gradient on the whole canvas at the same parameters, timed once on the host."""
    import oracle
    from paper_1810_03988_gb300 import Rig
    from paper_1810_03988_gb300.autograd import corners_of, params_from_corners, refine
    cfg = synth.config_refine()
    frames = cfg.frame(0)
    dev = [torch.from_numpy(f).to(f"cuda:{device}") for f in frames]
    n = len(cfg.cameras)
    rng = np.random.default_rng(7)
    true = np.stack([corners_of(c.H, c.width, c.height) for c in cfg.cameras])
    start = true.copy()
    start[1:] += rng.uniform(-3, 3, start[1:].shape)
    gains = np.ones(n)
    gains[1:] = rng.uniform(0.8, 1.2, n - 1)
    sizes = [(c.width, c.height) for c in cfg.cameras]
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, device=device) as rig:
        signs = [float(rig.camera_map(i)[0][2, 2]) for i in range(n)]
        p = params_from_corners(torch.tensor(start), torch.tensor(gains), sizes, signs)
        pd = p.to(f"cuda:{device}").contiguous()
        for _ in range(3):
            rig.backward(dev, pd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            loss, grad = rig.backward(dev, pd)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        t0 = time.perf_counter()
        corners, g, hist = refine(rig, dev, start, gains, steps=50)
        torch.cuda.synchronize()
        refine_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.loss_grad([c.width for c in cfg.cameras], [c.height for c in cfg.cameras], p.numpy(), frames,
                     (0, 0, cfg.canvas_w, cfg.canvas_h), a33=signs)
    cpu_s = time.perf_counter() - t0
    mpix = cfg.canvas_w * cfg.canvas_h / 1e6
    err = lambda c: float(np.abs(c - true)[1:].mean())
    return {"value": mpix / (ms / 1e3), "unit": "canvas MPix/s", "ms_per_call": ms,
            "workload": "4x1080p refinement rig (5200x1300 canvas), loss + 9 gradient entries per camera",
            "refine": {"steps": 50, "seconds": refine_s, "loss_start": hist[0], "loss_end": hist[-1],
                       "corner_error_px_start": err(start), "corner_error_px_end": err(corners),
                       "gain_error_start": float(np.abs(gains[1:] - 1).mean()),
                       "gain_error_end": float(np.abs(g[1:] - 1).mean())},
            "cpu_oracle": {"value": mpix / cpu_s, "unit": "canvas MPix/s", "cores": oracle.threads(),
                           "sample": "one loss + gradient over the whole canvas"}}


def measure_match(torch, dframes, hframes, device: int, points: int = 1000, iters: int = 1000, reps: int = 20):
    """Registration of the first two views (Sec. 4.2): GPU L-ORB features of each (whole views),
    then Multi-Probe LSH matching (8 tables x 16 bits) and PROSAC (T iterations) on the GPU, timed
    with CUDA events after warm-up; the oracle on the same feature sets beside it."""
    import oracle
    from paper_1810_03988_gb300 import LORB, Matcher
    pat, bits = synth.brief_pattern(0), synth.lsh_bits(0)
    rnd = synth.prosac_words(0, iters)
    H, W = dframes[0].shape[:2]
    areas = [(0, 0, W, H)]
    with LORB(W, H, points, device) as la, LORB(W, H, points, device) as lb, Matcher(points, iters, device) as m:
        fa = la.detect(dframes[0], areas, pat, 20, 0, points)
        fb = lb.detect(dframes[1], areas, pat, 20, 0, points)
        rw = torch.from_numpy(rnd.view(np.int32)).to(dframes[0].device)
        args = (fa[0], fa[2], fa[3], fb[0], fb[2], fb[3], bits, rw)
        for _ in range(3):
            m.match(*args)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            m.match(*args)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        n_matches, n_inl = int(m.n_matches.cpu()[0]), int(m.n_inliers.cpu()[0])
        ha = [t[:int(fa[3].cpu()[0])].cpu().numpy() for t in (fa[0], fa[2])]
        hb = [t[:int(fb[3].cpu()[0])].cpu().numpy() for t in (fb[0], fb[2])]
    t0 = time.perf_counter()
    oracle.match_prosac(ha[0], ha[1], hb[0], hb[1], bits, rnd)
    cpu_s = time.perf_counter() - t0
    return {"value": 1e3 / ms, "unit": "view pairs/s", "ms_per_pair": ms, "points_per_view": points,
            "prosac_iters": iters, "tables": int(bits.shape[0]), "bits": int(bits.shape[1]),
            "matches": n_matches, "inliers": n_inl,
            "cpu_oracle": {"value": 1.0 / cpu_s, "unit": "view pairs/s", "cores": 1, "sample": "the same pair"}}


def measure_batch(Rig, dev, torch, args, n_rigs: int = 16):
    """The 16-rig batching workload: every rig stitched by its own launch sequence, then the batch
    with the schedule its tuner picks, and each schedule forced (the persistent launch and the
    staged launches, both replayed from a CUDA graph, and the per-rig streams).  Device-timed, 3
    warm-up calls each; batch calls are asynchronous, so the timed region holds no host sync."""
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(n_rigs, seed=0)
    rigs = [Rig(c.cameras, c.canvas_w, c.canvas_h, c.levels, device=dev.index) for c in cfgs]
    frames = [[torch.from_numpy(f).to(dev) for f in c.frame(0)] for c in cfgs]
    outs = [r.new_output() for r in rigs]
    mpix = sum(c.canvas_w * c.canvas_h for c in cfgs) / 1e6
    steps = max(3, min(args.steps, 10))
    stream = torch.cuda.current_stream()

    def run(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def per_rig():
        for r, f, o in zip(rigs, frames, outs):
            r.stitch(f, o)

    per_ms = run(per_rig)
    res = {}
    prev = os.environ.get("STITCH_TUNE")
    for mode in ("auto", "persistent", "staged", "streams"):
        if mode == "auto":
            os.environ.pop("STITCH_TUNE", None)
        else:
            os.environ["STITCH_TUNE"] = mode
        with Batch(rigs) as b:
            b.stitch(frames, outs)  # first call: autotune + graph build
            b.sync()
            ms = run(lambda: b.stitch(frames, outs))
            b.sync()
            res[mode] = {"ms": ms, "value": mpix / (ms / 1e3), "unit": "MPix/s", "speedup_over_per_rig": per_ms / ms,
                         "schedule": b.schedule()}
    if prev is None:
        os.environ.pop("STITCH_TUNE", None)
    else:
        os.environ["STITCH_TUNE"] = prev
    for r in rigs:
        r.close()
    return {"rigs": n_rigs, "cameras": sum(len(c.cameras) for c in cfgs), "canvas_mpix": mpix,
            "per_rig_launches": {"ms": per_ms, "value": mpix / (per_ms / 1e3), "unit": "MPix/s"},
            "batched_launch": res["auto"], "speedup": per_ms / res["auto"]["ms"], "schedule": res["auto"]["schedule"],
            "persistent_launch": res["persistent"], "staged_launches": res["staged"], "per_rig_streams": res["streams"]}


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
        oracle.forward(cfg.cameras, frames0, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=w, canvas=cfg.canvas)

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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="8x4k", choices=sorted(WORKLOADS))
    ap.add_argument("--frames", type=int, default=None, help="distinct frame sets (default: the sequence length)")
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--fp16-bands", action="store_true")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison run")
    ap.add_argument("--e2e-steps", type=int, default=100,
                    help="frames of the end-to-end run (pipeline fill and drain included once)")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-band comparison run")
    ap.add_argument("--no-seam", action="store_true", help="skip the seam-weight run")
    ap.add_argument("--no-lorb", action="store_true", help="skip the L-ORB feature-extraction run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-per-rig comparison")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the error measurement against the oracle")
    ap.add_argument("--no-backward", action="store_true", help="skip the backward (S7) and refinement run")
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

    frame_stats = {}

    def timed(rig, out, steps, warmup, profile, sampler=None):
        for k in range(warmup):
            rig.stitch(dframes[k % nfr], out)
        torch.cuda.synchronize()
        if profile:
            rig.set_profiling(True)
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_begin()
        # the profiled pass also records one event per frame, for the spread of frame times
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps)] if profile else []
        ev0.record(stream)
        for k in range(steps):
            rig.stitch(dframes[(warmup + k) % nfr], out)
            if evs:
                evs[k].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_end()
        barrier()
        ms = ev0.elapsed_time(ev1) / steps
        if evs:
            frame_stats.update(frame_percentiles([a.elapsed_time(b) for a, b in zip([ev0] + evs[:-1], evs)]))
        kt = rig.kernel_times() if profile else {}
        if profile:
            rig.set_profiling(False)
        ms = max_over_ranks(ms, dist if world > 1 else None, dev)
        return ms, kt

    rig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=args.fp16_bands, path=args.path,
              device=local, canvas=cfg.canvas)
    info = rig.info()
    out = rig.new_output()
    clocks = ClockSampler(local)
    # the reported timed region runs without per-kernel events (clocks sampled during it); a
    # second, profiled pass of the same steps gives the per-kernel times and shares
    clocks.start()
    ms, _ = timed(rig, out, args.steps, args.warmup, False, clocks)
    clk = clocks.stop()
    _, kt = timed(rig, out, args.steps, 3, True)

    mpix = cfg.canvas_w * cfg.canvas_h / 1e6
    value = job_value(mpix, world, ms)
    fps = 1e3 / ms
    hbm_peak, peak_kind = _peaks()
    cbytes = compulsory_bytes(cfg)

    # dominant kernel and its roofline: the fused kernels are issue-bound (FP32 sample arithmetic),
    # so the bound is the FP32 ALU peak at the clock measured during the timed region
    dom = max(kt.items(), key=lambda kv: kv[1][0]) if kt else None
    dominant = dom[0] if dom else None
    if dom and kernel_algorithmic_flops(dom[0], cfg, info) is None:
        # small rigs: the largest kernel with an operation model (down1, up_full) stands in
        modelled = [kv for kv in kt.items() if kernel_algorithmic_flops(kv[0], cfg, info) is not None]
        dom = max(modelled, key=lambda kv: kv[1][0]) if modelled else dom
    roof = None
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if dom:
        name, (tot_ms, launches) = dom
        per_launch_ms = tot_ms / launches
        flops = kernel_algorithmic_flops(name, cfg, info)
        peak_tf = fp32_peak_tflops(clk.get("sm_mhz"), sms)
        achieved = flops / (per_launch_ms / 1e3) / 1e12 if flops else None
        traffic, traffic_src = profiled_traffic(name, args.workload)
        roof = {"kernel": name, "dominant_kernel": dominant, "bound": "alu", "achieved": achieved, "peak": peak_tf,
                "unit": "TFLOP/s",
                "frac": (achieved / peak_tf) if achieved else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x median SM clock under load",
                "avg_launch_ms": per_launch_ms, "launches_per_step": launches / args.steps,
                "share": tot_ms / sum(v[0] for v in kt.values()), "algorithmic_flops_per_launch": flops,
                "hbm_achieved_gbs_compulsory": cbytes / (ms / 1e3) / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_peak_source": f"{peak_kind} hbm_gbs (copy)"}
    # the whole step against both roofs: HBM on the compulsory bytes, FP32 ALU on the method's
    # operation count per step (see STEP_FLOPS_* below) at the clock sampled in the timed region
    step_flops = info["roi_pixels"] * STEP_FLOPS_PER_CAMERA_PX + cfg.canvas_w * cfg.canvas_h * STEP_FLOPS_PER_CANVAS_PX
    alu_peak = fp32_peak_tflops(clk.get("sm_mhz"), sms)
    alu_floor_ms = step_flops / (alu_peak * 1e12) * 1e3
    hbm_floor_ms = cbytes / (hbm_peak * 1e9) * 1e3
    step_roof = {"achieved": cbytes / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "frac": cbytes / (ms / 1e3) / 1e9 / hbm_peak, "compulsory_bytes_per_step": cbytes,
                 "hbm_floor_ms": hbm_floor_ms,
                 "algorithmic_flops_per_step": step_flops, "alu_peak_tflops": alu_peak,
                 "alu_achieved_tflops": step_flops / (ms / 1e3) / 1e12,
                 "alu_floor_ms": alu_floor_ms, "alu_frac": alu_floor_ms / ms,
                 "floor_ms": max(alu_floor_ms, hbm_floor_ms), "floor_frac": max(alu_floor_ms, hbm_floor_ms) / ms,
                 "flops_model": f"{STEP_FLOPS_PER_CAMERA_PX} per planned camera level-0 pixel (warp 40, REDUCE 40, "
                                f"EXPAND 35, blend 13) + {STEP_FLOPS_PER_CANVAS_PX} per canvas pixel (collapse)"}

    plain = None
    if args.path == "fused" and not args.no_plain:
        prig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path="plain", device=local,
                   canvas=cfg.canvas)
        pms, _ = timed(prig, out, max(3, min(args.steps, 10)), 3, False)
        plain = {"value": world * mpix / (pms / 1e3), "ms_per_step": pms,
                 "hbm_frac": cbytes / (pms / 1e3) / 1e9 / hbm_peak, "speedup_fused_over_plain": pms / ms}
        prig.close()

    # error against the FP64 oracle on sampled windows of frame 0, FP32 and FP16 bands
    accuracy = None
    if rank == 0 and not args.no_accuracy and args.path == "fused" and not args.fp16_bands:
        rig.stitch(dframes[0], out)
        torch.cuda.synchronize()
        accuracy = measure_accuracy(torch, Rig, cfg, host_frames[0], dframes[0], out, local)

    # FP16 storage of pyramid data between kernels (arithmetic still FP32), same frames
    fp16 = None
    if not args.fp16_bands and not args.no_fp16:
        hrig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=True, device=local,
                   canvas=cfg.canvas)
        hms, _ = timed(hrig, out, max(3, min(args.steps, 10)), 3, False)
        fp16 = {"value": world * mpix / (hms / 1e3), "ms_per_step": hms}
        hrig.close()

    # seam weights (binary owner masks): the masks are decided in FP64 when the rig is created,
    # the per-frame work is that of feather weights
    seam = None
    if not args.no_seam:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        srig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=args.fp16_bands, path=args.path,
                   device=local, weights="seam", canvas=cfg.canvas)
        torch.cuda.synchronize()
        create_ms = (time.perf_counter() - t0) * 1e3
        sms, _ = timed(srig, out, max(3, min(args.steps, 10)), 3, False)
        seam = {"value": world * mpix / (sms / 1e3), "ms_per_step": sms, "rig_create_ms": create_ms}
        srig.close()

    # L-ORB feature extraction (the registration step): every camera view of a frame set, whole
    # view as the detection area, 500 points per view; the oracle on the host for one view.  Then
    # matching and PROSAC on the first two views' features (1000 points each)
    lorb = match = None
    if not args.no_lorb and rank == 0:
        lorb = measure_lorb(torch, dframes[0], host_frames[0], local)
        match = measure_match(torch, dframes[0], host_frames[0], local)

    # S7: the backward (overlap loss and parameter gradient) and the refinement through it
    backward = None
    if not args.no_backward and rank == 0:
        backward = measure_backward(torch, local)

    # batching: 16 uneven rigs, one launch sequence per rig against one persistent launch
    batched = None
    if not args.no_batch:
        batched = measure_batch(Rig, dev, torch, args)

    # end to end through the overlapped host-buffer entry point: every step uploads its frames from
    # pinned host memory, stitches and downloads the canvas into pinned host memory; the upload of
    # step k+1 and the download of step k-1 overlap the stitch of step k; one sync at the end, so
    # the first upload and the last download (pipeline fill and drain) are inside the timed region
    pinned = [[torch.from_numpy(f).pin_memory() for f in fs] for fs in host_frames[:min(nfr, 4)]]
    houts = [torch.empty((cfg.canvas_h, cfg.canvas_w, 3), dtype=torch.uint8).pin_memory() for _ in range(2)]
    for k in range(2):
        rig.stitch_host_async(pinned[k % len(pinned)], houts[k])
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        rig.stitch_host_async(pinned[k % len(pinned)], houts[k & 1])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist if world > 1 else None, dev)
    h2d = sum(c.width * c.height * 3 for c in cfg.cameras)
    d2h = cfg.canvas_w * cfg.canvas_h * 3
    # the same through the blocking entry point (copies and stitch serialised), for comparison
    t0 = time.perf_counter()
    for k in range(3):
        rig.stitch_host(pinned[k % len(pinned)], houts[0])
    serial_ms = (time.perf_counter() - t0) / 3 * 1e3
    e2e = {"value": world * mpix / e2e_s, "unit": "MPix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_s * 1e3, "steps": args.e2e_steps, "entry_point": "stitch_frames_host_async",
           "includes": "pipeline fill and drain (first upload, last download)",
           "serial_ms_per_step": serial_ms}

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
            "roofline": roof, "step_roofline": step_roof, "plain_path": plain, "fp16_bands": fp16,
            "seam_weights": seam, "lorb": lorb, "match": match, "accuracy": accuracy, "backward": backward,
            "batched": batched, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk, "gpu_launches": info["num_kernels"] * args.steps,
            "rig": {"scratch_bytes": info["scratch_bytes"], "roi_pixels": info["roi_pixels"],
                    "kernels_per_step": info["num_kernels"], "tiles": info["tiles"]},
            "kernel_times_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in kt.items()},
            "frame_ms": dict(frame_stats, source="per-frame CUDA events of the profiled pass (same frames)"),
            "frame_generation_s": gen_s,
        }
        print(json.dumps(line))
    rig.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# Algorithmic FP32 operations (FMA = 2) per unit of work, counted from the method's definition:
#   warp sample: homography numerator/denominator (6 FMA = 12), perspective divide (3), bilinear
#     RGB (9 lerps = 18), gain/255 (3), feather weight and its normalisation (8)          -> 44
#   REDUCE to level 1 per level-0 pixel: 4 channels x (5-tap horizontal at half the columns
#     + 5-tap vertical at a quarter) x 2                                                    -> 30
#   blend + collapse per canvas pixel and camera at levels 0-1 (EXPAND 3ch x ~3 taps x 2 x 2
#     levels, weighted sum 8, divide/clamp 6)                                              -> 50
FLOPS_WARP = 44
FLOPS_REDUCE1 = 30
FLOPS_BLEND = 50
# The whole step, as the scope's measurement plan counts it: per planned camera level-0 pixel warp
# 40 + REDUCE 40 + EXPAND 35 + blend 13 (~130, across all levels), per canvas pixel collapse 35.
STEP_FLOPS_PER_CAMERA_PX = 130
STEP_FLOPS_PER_CANVAS_PX = 35

PROFILES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles")
KERNEL_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1810_03988_gb300", "csrc",
                             "fused.cu")


def code_digest(path: str) -> str:
    """SHA-256 of a C/C++/CUDA source with its comments removed and runs of whitespace collapsed:
    edits to comments or layout leave it unchanged, any change to the code changes it."""
    import hashlib
    src = open(path, encoding="utf-8").read()
    out, i, n = [], 0, len(src)
    while i < n:
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif src[i] in "\"'":
            j = i + 1
            while j < n and src[j] != src[i]:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(src[i])
            i += 1
    return hashlib.sha256(" ".join("".join(out).split()).encode()).hexdigest()


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) of one launch of `kernel` on `workload` from the committed ncu
    summaries under profiles/ (a `traffic:` line), or None when there is none or the kernel
    source's code has changed since the capture (the line records its code_digest)."""
    import glob
    import re
    try:
        digest = code_digest(KERNEL_SOURCE)
    except OSError:
        return None, None
    pat = re.compile(r"^traffic: kernel=(\S+) workload=(\S+) bytes_per_launch=(\d+) code_sha256=([0-9a-f]+)")
    for f in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(f):
            m = pat.match(line.strip())
            if m and m.group(1) == kernel and m.group(2) == workload:
                if m.group(4) != digest:
                    return None, f"profiles/{os.path.basename(f)} (stale: kernel source changed since the capture)"
                return int(m.group(3)), f"profiles/{os.path.basename(f)} (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    return None, None


def kernel_algorithmic_flops(name: str, cfg, info: dict) -> float | None:
    """Algorithmic FP32 operations of one launch of the named fused kernel (see the table above);
    the level-0 samples counted are the cameras' planned level-0 regions (roi_pixels), not the
    halo samples the tiling adds."""
    roi = info["roi_pixels"]
    t = info["tiles"]
    if name == "fused_down1":
        return roi * (FLOPS_WARP + FLOPS_REDUCE1)
    if name == "fused_up_full":
        # the level-0 samples come from down1: blend and collapse only
        px = t["full2"] * 64 * 32
        return px * 2 * FLOPS_BLEND
    return None


def fp32_peak_tflops(sm_mhz: float | None, sms: int) -> float:
    """FP32 peak from unit counts and clock: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    mhz = sm_mhz or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


if __name__ == "__main__":
    sys.exit(main())
