#!/usr/bin/env python
"""Benchmark of the LiteGS training-step hot path on GB300.

Workload (default): 3,000,000 Gaussians of SH degree 3 from the uniform-box
generator (means in [-1,1]^3 four units in front of the camera, log-scales
N(-3.5, 0.5), opacity logits N(0, 1), seed 2), one 1297 x 840 pinhole camera
(fx = fy = 1297), 16 x 16 tiles, L1 loss against a uniform random target.
One step = one training iteration a2..a10 on the Morton-sorted scene:
cluster cull + compaction, preprocess, binning + sort, forward
rasterisation, L1 loss gradient, backward rasterisation with the
opacity-gradient moments, variance metric, fused preprocess backward + Adam.
The Morton re-sort of parameters and Adam moments (a1) runs at fixed
intervals and after densification (Sec. 3.2.1); it is timed on its own and
reported beside the line, with the rate it would give if run every step.
The line also carries the mixed-precision steps, batched views (8 cameras,
one CUDA graph) and the served-render latency.

Metric: training iterations per second (whole job; N GPUs run N independent
replicas, weak scaling). Inputs stay resident (the 2.1 GB parameter + moment
state and the target exceed the 129 MB L2, so no flush is needed).

--impl reference times the CPU oracle on a bounded sample of the same
workload instead (see cpu_step_sample()).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd iters/s @3M Gaussians 1.1MP (plain vs mixed); served render p50/p99 ms"
UNIT = "iters/s"
N_GAUSS = 3_000_000
SH_DEG = 3
SEED = 2
W_IMG, H_IMG = 1297, 840
TILE = (16, 16)
WORKLOAD = ("3M Gaussians SH3 surface scene (the config-1 generator: 90% of the means on 32 "
            "planes and 32 spheres, 10% on a radius-20 shell; seed 2, Morton-sorted), 1297x840 "
            "orbit camera (radius 4, elevation 0.3 rad, fx=fy=0.78 W), 16x16 tiles, training "
            "iteration a2-a10 (cluster cull/compact + preprocess + bin sort + raster fwd + L1 + "
            "raster bwd + variance + fused preprocess-bwd/Adam); the periodic Morton re-sort a1 "
            "is timed separately")


def bench_config(world: int = 1) -> dict:
    """The workload description both arms print (`config`)."""
    return {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "sh_degree": SH_DEG,
            "resolution": f"{W_IMG}x{H_IMG}", "tile": f"{TILE[0]}x{TILE[1]}",
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (2.1 GB resident state), no flush"}


def make_workload(seed_offset: int = 0, n: int | None = None, width: int = W_IMG,
                  height: int = H_IMG):
    from paper_2503_01199_gb300 import scenegen
    return scenegen.surface_scene(n or N_GAUSS, SH_DEG, SEED + seed_offset, width, height)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        rows = [r.split(", ") for r in self.lines if r.count(",") >= 9]
        if self.bus_id:
            mine = [r for r in rows if self.bus_id.endswith(r[1].lower()[-12:]) or
                    r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[6 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def traffic_record() -> dict:
    """ncu DRAM bytes per launch of kernels, from profiles/traffic.json, with
    the library build they were captured on (stale entries read as null)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# sources each recorded kernel is compiled from: its recorded DRAM traffic
# stays valid while these are unchanged (profiles/traffic.json carries the
# digest and the list)
FUSED_SOURCES = ("paper_2503_01199_gb300/csrc/preprocess.cu",
                 "paper_2503_01199_gb300/csrc/lgs_internal.cuh", "include/lgs.h")
RASTER_SOURCES = ("paper_2503_01199_gb300/csrc/raster.cu",
                  "paper_2503_01199_gb300/csrc/lgs_internal.cuh", "include/lgs.h")


def source_digest(files=FUSED_SOURCES) -> str:
    """Digest of the code of `files` (comments and whitespace removed)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, name), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(name.encode() + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, units: float | None = None) -> int | None:
    """DRAM bytes of one launch of the recorded kernel `key`: bytes_per_unit
    x units for a kernel whose traffic scales with its units, or the
    bytes of a launch captured at the bench workload itself; None when the
    kernel's sources changed since the capture or nothing was recorded."""
    rec = traffic_record().get(key, {})
    files = tuple(rec.get("source_files", FUSED_SOURCES))
    if not rec or rec.get("source") != source_digest(files):
        return None
    if "bytes_per_unit" in rec and units is not None:
        return round(rec["bytes_per_unit"] * units)
    if "bytes_per_launch" in rec and units is None:
        return int(rec["bytes_per_launch"])
    return None


def recorded_count(key: str) -> int | None:
    """An ncu event count of one launch of the recorded kernel `key` at the
    bench workload (count_per_launch); None when its sources changed since
    the capture or nothing was recorded."""
    rec = traffic_record().get(key, {})
    files = tuple(rec.get("source_files", FUSED_SOURCES))
    if not rec or rec.get("source") != source_digest(files) or "count_per_launch" not in rec:
        return None
    return int(rec["count_per_launch"])


def max_over_ranks(values, device) -> list:
    """Elementwise maximum of every rank's values (the slowest rank's times),
    over the initialised process group; the values themselves with none."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in values]
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_rate(world: int, steps: int, ms: float) -> float:
    """Whole-job iterations/s: the iterations of all ranks (independent
    replicas) over the slowest rank's time."""
    return world * steps / (ms / 1e3)


MV_RES = ((640, 360), (960, 540), (1297, 840), (1600, 1063)) * 2


def run_multiview(tr, steps: int, warmup: int) -> dict:
    """fwd + bwd of the 3M scene for 8 orbit cameras: one CUDA-graph replay
    of the batched sequence (per-view front end, one persistent raster
    forward and backward over all views' tiles) against the same work as 8
    sequential plain launch sequences."""
    import torch
    from paper_2503_01199_gb300 import pipeline as PL
    from paper_2503_01199_gb300 import scenegen
    dev = tr.params.device
    cams = scenegen.orbit_cameras(4, list(MV_RES), radius=4.0, elevation=0.3)
    rng = np.random.default_rng(4)
    tgts = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)).to(dev)
            for w, h in MV_RES]
    mv = PL.MultiView(tr.params, tr.n, tr.sh_degree, cams, tgts, pair_capacity=128_000_000)
    stream = torch.cuda.current_stream(dev)
    out = {}

    def timed(name, fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms_per_batch"] = round(e0.elapsed_time(e1) / steps, 4)

    # the graph with the views' front ends on one stream, then on the side
    # streams (the batched path), then the sequential plain launches
    slots = mv.n_slots
    mv.n_slots = 1
    mv.capture()
    timed("graph_one_stream", mv.replay)
    mv.n_slots = slots
    mv.capture()
    timed("graph", mv.replay)
    timed("sequential", mv.run_sequential)
    pairs = [int(v["d_P"].item()) for v in mv.views]
    del mv
    torch.cuda.empty_cache()
    return {"workload": ("3M Gaussians SH3 (same scene), 8 orbit cameras (radius 4 around the "
                         "origin) at 640x360, 960x540, 1297x840, 1600x1063, two each: "
                         "per-view cull/preprocess/binning (on "
                         f"{slots} side streams in the graph), batched raster fwd, L1, batched "
                         "raster bwd, preprocess bwd summed over views"),
            **out, "views_per_s": round(8 * 1e3 / out["graph_ms_per_batch"], 1),
            "speedup_vs_sequential": round(out["sequential_ms_per_batch"] /
                                           out["graph_ms_per_batch"], 3),
            "pairs_per_view": pairs}


def run_ccc_ablation(steps: int = 24, warmup: int = 3) -> dict:
    """Iteration time (a2-a10) with Cluster-Cull-Compact on / off and with
    Morton-sorted / randomly shuffled storage (Sec. 3.2; the E3/E6 analogue),
    on the 500K surface scene with its orbit camera and on interior scenes
    (a camera inside a cube of side 12, about a tenth of it in view) of 500K
    and 3M Gaussians."""
    import torch
    from paper_2503_01199_gb300 import binding as B
    from paper_2503_01199_gb300 import pipeline as PL
    from paper_2503_01199_gb300 import scenegen
    cases = {}
    d2 = scenegen.surface_scene(500_000, SH_DEG, 1, W_IMG, H_IMG)
    cases["surface_500k_1297x840"] = (d2["scene"], d2["camera"], d2["target"])
    for n, label in ((500_000, "500k"), (3_000_000, "3m")):
        d = scenegen.interior_scene(n, SH_DEG, 5, W_IMG, H_IMG)
        cases[f"interior_{label}_1297x840"] = (d["scene"], d["camera"], d["target"])
    out = {}
    for name, (sc, cam, tgt) in cases.items():
        n = sc["mean"].shape[0]
        perm = np.random.default_rng(9).permutation(n)
        shuffled = {k: (np.asarray(v)[perm] if k != "sh_degree" else v) for k, v in sc.items()}
        res = {}
        for order, scene in (("morton", sc), ("shuffled", shuffled)):
            for ccc in (True, False):
                tr = PL.Trainer(scene, cam["width"], cam["height"],
                                PL.StepConfig(tile=TILE, pair_capacity=128_000_000, ccc=ccc))
                if order == "morton":
                    tr.morton_reorder()
                target = torch.from_numpy(tgt).to(tr.dev)
                cs = B.camera_struct(cam)
                for _ in range(warmup):
                    tr.step(cs, target, reorder=False)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
                ev[0].record()
                for k in range(steps):
                    tr.step(cs, target, reorder=False)
                    ev[k + 1].record()
                torch.cuda.synchronize()
                per = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(steps)])
                V = int(tr.d_V.item()) if ccc else n
                res[f"{order}_{'ccc' if ccc else 'no_ccc'}"] = {
                    "ms_per_iter": round(float(per.mean()), 4),
                    "ms_p10": round(float(np.percentile(per, 10)), 4),
                    "ms_p90": round(float(np.percentile(per, 90)), 4),
                    "steps": steps, "rows_processed": V}
                del tr
                torch.cuda.empty_cache()
        out[name] = res
    return out


def run_extra_configs(steps: int, warmup: int) -> dict:
    """The other single-GPU configurations, each a whole a2-a10 iteration
    through the pipeline on Morton-sorted state: the 3M scene with its
    1600x1063 camera (plain and mixed blend), and the 500K surface scene
    (seed 1) with its 1297x840 camera."""
    import torch
    from paper_2503_01199_gb300 import binding as B
    from paper_2503_01199_gb300 import pipeline as PL
    from paper_2503_01199_gb300 import scenegen
    out = {}
    cases = (("3m_1600x1063", lambda: make_workload(width=1600, height=1063),
              (("fp32", B.LGS_FP32), ("fp16", B.LGS_MIXED_FP16), ("bf16", B.LGS_MIXED_BF16))),
             ("500k_1297x840", lambda: scenegen.surface_scene(500_000, SH_DEG, 1, W_IMG, H_IMG),
              (("fp32", B.LGS_FP32),)))
    for name, make, precs in cases:
        d = make()
        cam = d["camera"]
        tr = PL.Trainer(d["scene"], cam["width"], cam["height"],
                        PL.StepConfig(tile=TILE, pair_capacity=128_000_000))
        tr.morton_reorder()
        cs = B.camera_struct(cam)
        target = torch.from_numpy(d["target"]).to(tr.dev)
        res = {"n_gaussians": int(d["scene"]["mean"].shape[0]),
               "resolution": f"{cam['width']}x{cam['height']}"}
        for pname, prec in precs:
            tr.cfg.precision = prec
            for _ in range(warmup):
                tr.step(cs, target, reorder=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                tr.step(cs, target, reorder=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            res[pname] = {"iters_per_s": round(1e3 / ms, 2), "ms_per_iter": round(ms, 4)}
        res["visible_gaussians"] = int(tr.d_V.item())
        res["pairs"] = int(tr.d_P.item())
        out[name] = res
        del tr, target
        torch.cuda.empty_cache()
    return out


# a8 (the densification metric) is written by the fused a9 + a10 call from
# the gradient rows it reads, so its time is part of "a9a10_bwd_adam"
STAGES = ["a1_morton", "a2_cull", "a3_preprocess", "a4_bin_sort", "a5_raster_fwd", "a6_loss",
          "a7_raster_bwd", "a9a10_bwd_adam"]


def measure_unit_peaks(dev, n_sms: int, reps: int = 5) -> dict:
    """Unit rates of this GPU from the library's own microbenchmarks
    (lgs_peak_*; outside every timed region): the special-function unit's
    ex2, FP32 FMA in the scalar and the packed two-lane form, and float
    reductions into global memory in the backward's pattern (12 lanes into
    one 64-byte row) on 64 MB of rows (L2-resident) and on 192 MB (larger
    than L2, the size class of the 3M scene's 175 MB of gradient rows).
    Each rate is the operation count of `reps` calls over their CUDA-event
    time, after one untimed call."""
    import torch
    from paper_2503_01199_gb300 import binding as B
    blocks = n_sms * 8
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(blocks * B.PEAK_THREADS, dtype=torch.float32, device=dev)
    rows_l2 = torch.zeros((1 << 20, 16), dtype=torch.float32, device=dev)
    rows_big = torch.zeros((3 << 20, 16), dtype=torch.float32, device=dev)

    def rate(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = sum(fn() for _ in range(reps))
        e1.record(stream)
        torch.cuda.synchronize()
        return n / (e0.elapsed_time(e1) * 1e-3)

    res = {"ex2_per_s": rate(lambda: B.lgs_peak_ex2(out, blocks, 256)),
           "ffma_per_s": rate(lambda: B.lgs_peak_ffma(out, blocks, 1024, False)),
           "ffma2_fma_per_s": rate(lambda: B.lgs_peak_ffma(out, blocks, 1024, True)),
           "red_l2_per_s": rate(lambda: B.lgs_peak_red(rows_l2, rows_l2.shape[0], blocks, 1024)),
           "red_192mb_per_s": rate(lambda: B.lgs_peak_red(rows_big, rows_big.shape[0], blocks,
                                                           1024))}
    del out, rows_l2, rows_big
    return {**{k: float(f"{v:.4g}") for k, v in res.items()}, "blocks": blocks,
            "method": "lgs_peak_ex2 / lgs_peak_ffma / lgs_peak_red, CUDA events, "
                      f"{reps} calls after one untimed call"}


def run_gpu(args) -> dict | None:
    import torch
    import torch.distributed as dist
    from paper_2503_01199_gb300 import binding as B
    from paper_2503_01199_gb300 import pipeline as PL

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.load()
    d = make_workload(rank, args.n_gaussians)
    sc, cam, tgt_np = d["scene"], d["camera"], d["target"]
    morton = args.storage == "morton"
    if not morton:  # rows in a random order, never re-sorted (profiling evidence only)
        perm = np.random.default_rng(9).permutation(sc["mean"].shape[0])
        sc = {k: (np.asarray(v)[perm] if k != "sh_degree" else v) for k, v in sc.items()}
    # the profiling case's pair capacity scales with its scene, so that a
    # capture of it holds a small device footprint (22.1M pairs at 3M)
    cap = 128_000_000 if not args.n_gaussians else max(16_000_000, 16 * args.n_gaussians)
    tr = PL.Trainer(sc, W_IMG, H_IMG, PL.StepConfig(tile=TILE, pair_capacity=cap),
                    device=str(dev))
    del sc
    cs = B.camera_struct(cam)
    target = torch.from_numpy(tgt_np).to(dev)
    stream = torch.cuda.current_stream(dev)

    det_ws = None

    def step(events=None, precision=B.LGS_FP32, reorder=False, deterministic=False):
        nonlocal det_ws
        def mark(i):
            if events is not None:
                events[i].record(stream)
        mark(0)
        if reorder:  # a1 runs at intervals (Sec. 3.2.1), timed on its own below
            tr.morton_reorder()
        mark(1)
        g = tr.gaussians()
        B.lgs_cluster_cull_compact(g, cs, tr.cfg.cluster, None, tr.cluster_visible, tr.rowmap,
                                   tr.d_V, tr.ws_ccc)
        mark(2)
        B.lgs_preprocess(g, tr.rowmap, tr.d_V, cs, TILE[0], TILE[1], tr.splats)
        mark(3)
        B.lgs_bin_sort(tr.splats, tr.d_V, tr.n, cs, TILE[0], TILE[1], tr.vals, tr.d_P, tr.ranges,
                       tr.ws_bin)
        mark(4)
        B.lgs_raster_fwd(tr.splats, tr.vals, tr.ranges, cs, TILE[0], TILE[1], tr.image,
                         tr.finalT, tr.last, precision=precision)
        mark(5)
        B.lgs_loss_l1(tr.image, target, tr.dLdI, tr.loss)
        mark(6)
        if deterministic:  # bit-reproducible accumulation (fixed-point limbs)
            if det_ws is None:
                det_ws = torch.empty(B.lgs_raster_bwd_det_workspace_size(tr.gacc.shape[0]),
                                     dtype=torch.uint8, device=dev)
            B.lgs_raster_bwd_deterministic(tr.splats, tr.vals, tr.ranges, cs, TILE[0], TILE[1],
                                           tr.finalT, tr.last, tr.dLdI, tr.gacc, det_ws,
                                           precision=precision)
        else:
            B.lgs_raster_bwd(tr.splats, tr.vals, tr.ranges, cs, TILE[0], TILE[1], tr.finalT,
                             tr.last, tr.dLdI, tr.gacc, precision=precision)
        mark(7)
        tr.step_count += 1
        # a9 + a10, and the a8 metric from the same gradient rows
        B.lgs_preprocess_bwd_adam(tr.gaussians(), tr.m, tr.v, tr.rowmap, tr.d_V, cs, tr.gacc,
                                  tr.lr, tr.cfg.beta1, tr.cfg.beta2, tr.cfg.eps, tr.step_count,
                                  splats=tr.splats, metric=tr.metric)
        mark(8)

    for w in range(args.warmup):
        step(reorder=(w == 0 and morton))  # the timed steps run on Morton-sorted state
    torch.cuda.synchronize()
    overflow = B.lgs_get_overflow()
    if overflow:
        raise RuntimeError(f"pair capacity too small: {overflow} pairs needed")
    V = int(tr.d_V.item())
    P = int(tr.d_P.item())
    # fragments up to each pixel's last composited splat (the raster's unit of
    # work): the sum of last_contrib over the image, the same every iteration
    F = int(tr.last.sum(dtype=torch.int64).item())
    # ---- timed region: device throughput with per-stage events
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except AttributeError:
        pass
    clocks = ClockSampler(bus)
    clocks.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = B.lgs_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    launches = B.lgs_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    stage_ms = {s: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)]))
                for i, s in enumerate(STAGES) if s != "a1_morton"}
    # ---- a1 alone: Morton codes, sort and the gather of params, m and v
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(args.steps):
        tr.morton_reorder()
    m1.record(stream)
    torch.cuda.synchronize()
    morton_ms = m0.elapsed_time(m1) / args.steps
    # ---- end to end: target from pinned host memory, step, loss back to host
    pinned = torch.from_numpy(tgt_np).pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        target.copy_(pinned, non_blocking=True)
        step()
        loss_host.copy_(tr.loss, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    # ---- the same step with the mixed-precision raster (FP16 / BF16 blend)
    mixed = {}
    sh_types = {"fp16": torch.float16, "bf16": torch.bfloat16}
    # every variant starts from the same parameters and moments (the steps
    # train, and a drifting scene would change the work between variants)
    snapshot = tr.state[tr.cur].clone()
    step_count0 = tr.step_count
    for name, prec, dm, sh in (
            ("fp32", B.LGS_FP32, False, None),
            ("fp16", B.LGS_MIXED_FP16, False, None), ("bf16", B.LGS_MIXED_BF16, False, None),
            ("fp16_sh16", B.LGS_MIXED_FP16, False, "fp16"),
            ("bf16_sh16", B.LGS_MIXED_BF16, False, "bf16"),
            ("fp32_warp_reduce_int", B.LGS_FP32 | B.LGS_WARP_REDUCE_INT, False, None),
            ("fp32_deterministic", B.LGS_FP32, True, None),
            ("fp32_warp_reduce_int_deterministic", B.LGS_FP32 | B.LGS_WARP_REDUCE_INT, True,
             None)):
        tr.state[tr.cur].copy_(snapshot)
        tr.step_count = step_count0
        if sh:  # colour coefficients read in 16 bits (the fused Adam keeps the copy)
            tr.sh16 = torch.zeros((tr.np_ - 11, tr.stride), dtype=sh_types[sh], device=dev)
            tr._round_sh16()
        for _ in range(2):
            step(precision=prec, deterministic=dm)
        mev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        for k in range(args.steps):
            step(mev[k], precision=prec, deterministic=dm)
        m1.record(stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1)
        mixed[name] = {
            "value": round(world * args.steps / (mms / 1e3), 2), "unit": UNIT,
            "ms_per_step": round(mms / args.steps, 4),
            "a5_raster_fwd_ms": round(float(np.mean([mev[k][4].elapsed_time(mev[k][5])
                                                     for k in range(args.steps)])), 4),
            "a7_raster_bwd_ms": round(float(np.mean([mev[k][6].elapsed_time(mev[k][7])
                                                     for k in range(args.steps)])), 4),
            "a3_preprocess_ms": round(float(np.mean([mev[k][2].elapsed_time(mev[k][3])
                                                     for k in range(args.steps)])), 4),
            "a9a10_bwd_adam_ms": round(float(np.mean([mev[k][7].elapsed_time(mev[k][8])
                                                      for k in range(args.steps)])), 4)}
        tr.sh16 = None
    tr.state[tr.cur].copy_(snapshot)
    tr.step_count = step_count0
    del snapshot
    multiview = (run_multiview(tr, max(args.steps // 2, 3), 2)
                 if world == 1 and not args.n_gaussians else None)
    clk = clocks.stop()
    loss_val = float(loss_host.item())
    if world > 1:
        ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev)
        dist.destroy_process_group()
    if rank != 0:
        return None
    ms_step = ms / args.steps
    value = job_rate(world, args.steps, ms)
    e2e_value = job_rate(world, args.steps, e2e_ms)
    # ---- rooflines. The two largest items of the iteration, about 28% of
    # the launch list each, are the fused preprocess backward + Adam and the
    # backward raster; `roofline` takes whichever ran longer. The backward
    # raster (k_raster_bwd, a7) is bound by FP32
    # arithmetic: about 30 FP32 operations per fragment up to `last` (the
    # per-pixel gradient terms; an FMA counts as one operation) against the
    # FP32 lanes' rate, 152 SMs x 128 lanes x 2.07 GHz = 40.3 T operations/s.
    # The lane rate is SMs (queried) x 128 FP32 lanes x the SM clock: the
    # median sampled during the timed region (else the maximum, 2070 MHz).
    # The forward (a5): about 9 per fragment. The largest HBM-bound call is
    # the fused preprocess backward + Adam (k_bwd_adam_rec), 1484 B per
    # visible Gaussian at SH3: params, m, v read and written (6 x 59 x 4 B),
    # the 9 gradients + S, M, C of its grad row (48 B), its map entry (4 B),
    # the 3 colours of its splat record (12 B) and the a8 metric it writes
    # (4 B).
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float((clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = n_sms * 128 * clk_mhz * 1e6 / 1e12  # T operations/s, an FMA as one
    ops_bwd, ops_fwd = 30, 9
    bwd_t = F * ops_bwd / (stage_ms["a7_raster_bwd"] * 1e-3) / 1e12
    fwd_t = F * ops_fwd / (stage_ms["a5_raster_fwd"] * 1e-3) / 1e12
    units = measure_unit_peaks(dev, n_sms)
    # the raster's other units: one ex2 per fragment in each pass (the
    # backward adds a reciprocal on the same unit), and the backward's float
    # reductions (12 per contributing (quadrant warp, splat), counted by ncu
    # on the bench workload; null when the raster sources changed since)
    a5_s, a7_s = stage_ms["a5_raster_fwd"] * 1e-3, stage_ms["a7_raster_bwd"] * 1e-3
    red_instr = (recorded_count("a7_raster_bwd_red")
                 if not args.n_gaussians and morton else None)
    red_per_s = 12 * red_instr / a7_s if red_instr else None
    unit_rates = {
        "measured": units,
        "a5_ex2": {"per_launch": F, "achieved_per_s": float(f"{F / a5_s:.4g}"),
                   "frac": round(F / a5_s / units["ex2_per_s"], 4)},
        "a7_mufu": {"per_launch": 2 * F, "achieved_per_s": float(f"{2 * F / a7_s:.4g}"),
                    "frac": round(2 * F / a7_s / units["ex2_per_s"], 4),
                    "note": "ex2 and the reciprocal of 1 - alpha per fragment"},
        "a7_red": {"per_launch": 12 * red_instr if red_instr else None,
                   "achieved_per_s": float(f"{red_per_s:.4g}") if red_per_s else None,
                   "frac_of_l2": round(red_per_s / units["red_l2_per_s"], 4) if red_per_s else None,
                   "frac_of_192mb": (round(red_per_s / units["red_192mb_per_s"], 4)
                                     if red_per_s else None)},
        "fp32_lane_rate_vs_measured_ffma": round(fp32_peak * 1e12 / units["ffma_per_s"], 4),
    }
    peak_src = (f"derived: {n_sms} SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz (sampled SM clock), "
                "one operation per lane per cycle (an FMA as one operation)")
    raster_bwd = {"kernel": "lgs_raster_bwd (k_raster_bwd<0>)", "bound": "alu",
                "achieved": round(bwd_t, 3), "peak": round(fp32_peak, 2), "unit": "T ops/s",
                "peak_source": peak_src,
                "frac": round(bwd_t / fp32_peak, 4),
                "frac_of_fma_flop_peak": round(bwd_t / (2.0 * fp32_peak), 4),
                "traffic": (recorded_traffic("a7_raster_bwd")
                            if not args.n_gaussians and morton else None),
                "algorithmic_ops": int(F * ops_bwd), "fragments": F,
                "ops_per_fragment": ops_bwd}
    npl = B.num_planes(SH_DEG)
    per_unit = {"a9a10_bwd_adam": 6 * npl * 4 + 48 + 4 + 12 + 4,
                "a3_preprocess": npl * 4 + 4 + 48 + 4 + 4}  # params + map in; record, depth, radius out
    dom = "a9a10_bwd_adam"
    achieved = V * per_unit[dom] / (stage_ms[dom] * 1e-3) / 1e9
    traffic = recorded_traffic(dom, V)
    pre_gbs = V * per_unit["a3_preprocess"] / (stage_ms["a3_preprocess"] * 1e-3) / 1e9
    bwd_adam = {"kernel": "lgs_preprocess_bwd_adam (k_bwd_adam_rec<3>, with the a8 metric)",
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "peak_source": "measured" if hbm else "fallback",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes": int(V * per_unit[dom]),
                "bytes_per_visible_gaussian": per_unit[dom]}
    # `roofline` is the kernel with the larger live time of the two largest
    # items (the fused optimizer or the backward raster); the other goes to
    # `roofline_other` with the forward raster and the preprocess
    bwd_first = stage_ms["a7_raster_bwd"] >= stage_ms["a9a10_bwd_adam"]
    roofline = raster_bwd if bwd_first else bwd_adam
    other = {("a9a10_bwd_adam" if bwd_first else "a7_raster_bwd"):
             (bwd_adam if bwd_first else raster_bwd),
             "a5_raster_fwd": {"kernel": "lgs_raster_fwd (k_raster_fwd<0>)", "bound": "alu",
                               "achieved": round(fwd_t, 3), "peak": round(fp32_peak, 2),
                               "unit": "T ops/s", "frac": round(fwd_t / fp32_peak, 4),
                               "ops_per_fragment": ops_fwd},
             "a3_preprocess": {"bound": "hbm", "achieved": round(pre_gbs, 1),
                               "frac": round(pre_gbs / peak, 4)}}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(world),
        "counts": {"visible_gaussians": V, "pairs": P, "fragments": F},
        "roofline": roofline,
        "roofline_other": other,
        "unit_rates": unit_rates,
        "mixed": mixed,
        "batched_views": multiview,
        "a1_morton_resort": {
            "ms": round(morton_ms, 4),
            "note": ("the Morton re-sort of params, m and v runs at fixed intervals and after "
                     "densification (Sec. 3.2.1), so an iteration is a2-a10 and a1 is timed "
                     "on its own"),
            "iters_per_s_if_every_step": round(1e3 / (ms_step + morton_ms), 2)},
        "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(tgt_np.nbytes), "d2h_bytes_per_step": 4},
        "gpu_launches": int(launches),
        "clocks": clk,
        "loss": loss_val,
    }
    return out


# ---------------------------------------------------------------------------
# served renders: resident scenes, Poisson request stream, slots by HBM budget
# ---------------------------------------------------------------------------
SERVE_SCENES = ((500_000, 10), (1_000_000, 11), (2_000_000, 12), (3_000_000, 13))
SERVE_RES = ((640, 360), (1280, 720), (1920, 1080))
SERVE_RATE = 200.0
SERVE_PAIR_CAPACITY = 128_000_000  # 1920x1080 class; largest seen: 97.7M pairs (3M, 1920x1080)
SERVE_BUDGET_LARGE = 4.2  # budget: 4.2 x a 1920x1080 slot (about 14 GB), deliberately small
SERVE_SWEEP = (500.0, 1000.0, 2000.0, 4000.0)
SERVE_SWEEP_SECONDS = 2.0
SERVE_SIDE_SECONDS = 20.0  # the grouped executor and the plain loop at the configured rate


def run_serving(seconds: float) -> dict:
    import gc

    import torch
    from paper_2503_01199_gb300 import scenegen
    from paper_2503_01199_gb300 import serving as SV
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    scenes = [SV.ResidentScene(scenegen.surface_scene(n, SH_DEG, seed, 64, 64)["scene"])
              for n, seed in SERVE_SCENES]
    origin = (0.0, 0.0, 0.0)
    max_n = max(n for n, _ in SERVE_SCENES)
    classes = [(w, h, SV.class_capacity(w, h, max_n, 1920, 1080, SERVE_PAIR_CAPACITY))
               for w, h in SERVE_RES]
    budget = int(SERVE_BUDGET_LARGE * SV.slot_bytes(max_n, 1920, 1080, SERVE_PAIR_CAPACITY))
    res = list(SERVE_RES)

    def stream(seed, secs, rate):
        return scenegen.render_requests(seed, secs, rate, len(scenes), res, center=origin)

    def run(kind, reqs):
        gc.collect()
        torch.cuda.empty_cache()
        if kind == "plain_loop":
            return SV.plain_loop(scenes, reqs, res, SERVE_PAIR_CAPACITY)["stats"]
        out = SV.serve(scenes, reqs, budget, res, SERVE_PAIR_CAPACITY, classes=classes,
                       grouped=(kind == "grouped"))
        st = out["stats"]
        del out
        return st

    keys = ("p50_ms", "p99_ms", "mean_ms", "frames_per_s", "requests", "pair_overflow")
    run("per_request_graphs", stream(21, 1.0, SERVE_RATE))   # discarded warm-up stream
    st = run("per_request_graphs", stream(20, seconds, SERVE_RATE))
    side = min(seconds, SERVE_SIDE_SECONDS)
    gst = run("grouped", stream(20, side, SERVE_RATE))
    plain = run("plain_loop", stream(20, side, SERVE_RATE))
    sweep = []
    for i, rate in enumerate(SERVE_SWEEP):
        row = {"rate_req_per_s": rate, "seconds": SERVE_SWEEP_SECONDS}
        for kind in ("per_request_graphs", "grouped", "plain_loop"):
            r = run(kind, stream(40 + i, SERVE_SWEEP_SECONDS, rate))
            row[kind] = {k: r[k] for k in ("p50_ms", "p99_ms", "frames_per_s", "requests")}
            if kind != "plain_loop":
                row[kind]["retries"] = r["retries"]
        sweep.append(row)
    return {"workload": ("4 resident scenes (config-1 surface generator, SH3, BF16 colour + "
                         "FP32 geometry): 0.5M/1M/2M/3M Gaussians, seeds 10-13; Poisson arrivals "
                         f"at {SERVE_RATE:g} req/s for {seconds:g} s, resolution uniform over "
                         "640x360/1280x720/1920x1080, orbit cameras around the origin; forward "
                         "render + image to pinned host"),
            "hbm_budget_bytes": budget, "slot_classes": st["slot_classes"],
            **{k: st[k] for k in keys}, "slots": st["slots"], "max_inflight": st["max_inflight"],
            "retries": st["retries"],
            "grouped_batched_raster": {**{k: gst[k] for k in keys}, "seconds": side,
                                       "max_group": gst["max_group"]},
            "plain_loop": {**{k: plain[k] for k in keys}, "seconds": side},
            "load_sweep": sweep}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def cpu_step_sample(d, row_frac: int = 2, n_blocks: int = 150, seed: int = 0) -> dict:
    """Time the oracle's step on a bounded sample and scale it to one step.

    Per-Gaussian stages (Morton codes + sort, cluster cull, preprocess,
    variance, preprocess backward, Adam) run on every row_frac-th Gaussian
    and are scaled by row_frac. Per-tile stages (binning, forward, loss,
    backward) run on n_blocks blocks of 4 x 4 tiles drawn from the tile grid,
    each on exactly its own splats (camera cropped to the block, OpenMP over
    its 16 tiles), and are scaled by (number of tiles) / (sampled tiles).
    """
    import oracle
    sc, cam, tgt = d["scene"], d["camera"], d["target"]
    n = sc["mean"].shape[0]
    rows = np.arange(0, n, row_frac)
    sub = {k: (np.asarray(v)[rows] if k != "sh_degree" else v) for k, v in sc.items()}
    t = {}

    def timed(name, fn):
        a = time.perf_counter()
        r = fn()
        t[name] = time.perf_counter() - a
        return r

    timed("a1", lambda: oracle.morton_reorder(sub))
    timed("a2", lambda: oracle.cluster_cull(sub, cam, 128))
    timed("a3", lambda: oracle.preprocess(sub, cam, TILE))
    # per-tile work needs every splat of a block: project the full scene once
    # (untimed setup; its cost is counted by the a3 sample above)
    full = oracle.preprocess(sc, cam, TILE)
    gx, gy = -(-cam["width"] // TILE[0]), -(-cam["height"] // TILE[1])
    rect = full["rect"]
    live = full["radius"] > 0
    rng = np.random.default_rng(seed)
    bs = 4
    tile_time, tiles_done = 0.0, 0
    for _ in range(n_blocks):
        bx, by = int(rng.integers(0, gx - bs + 1)), int(rng.integers(0, gy - bs + 1))
        sel = np.flatnonzero(live & (rect[:, 0] < bx + bs) & (rect[:, 2] > bx) &
                             (rect[:, 1] < by + bs) & (rect[:, 3] > by))
        spt = {k: full[k][sel] for k in ("uv", "conic", "opacity", "rgb", "depth", "radius",
                                         "tau")}
        spt["uv"] = spt["uv"] - np.array([bx * TILE[0], by * TILE[1]], np.float64)
        bw_, bh_ = bs * TILE[0], bs * TILE[1]
        ccam = dict(cam, width=bw_, height=bh_)
        tg = np.zeros((3, bh_, bw_), np.float32)
        part = tgt[:, by * TILE[1]:by * TILE[1] + bh_, bx * TILE[0]:bx * TILE[0] + bw_]
        tg[:, :part.shape[1], :part.shape[2]] = part
        a = time.perf_counter()
        vals, ranges, P = oracle.bin_splats(spt["uv"][:, 0], spt["uv"][:, 1], spt["radius"],
                                            spt["depth"], bw_, bh_, TILE, conic=spt["conic"],
                                            tau=spt["tau"])
        fw = oracle.render_fwd(spt, vals, ranges, ccam, TILE)
        L, dL = oracle.l1_loss(fw["image"], tg)
        oracle.render_bwd(spt, vals, ranges, ccam, dL, TILE)
        tile_time += time.perf_counter() - a
        tiles_done += bs * bs
    g9 = np.random.default_rng(1).standard_normal((rows.size, 9)) * 1e-6
    timed("a8", lambda: oracle.opacity_variance(np.abs(g9[:, 0]), g9[:, 1],
                                                np.ones(rows.size, np.int64)))
    grads = timed("a9", lambda: oracle.preprocess_bwd(sub, cam, g9))
    planes = oracle.scene_planes(sub)
    gp = oracle.grad_planes(grads)
    m, v = np.zeros_like(planes), np.zeros_like(planes)
    from paper_2503_01199_gb300 import pipeline as PL
    lr = np.asarray(PL.lr_per_plane(SH_DEG), np.float64)
    timed("a10", lambda: oracle.adam(planes, gp, m, v, lr, 1, np.arange(rows.size, dtype=np.uint32)))
    # an iteration is a2..a10 (the Morton re-sort a1 runs at intervals)
    per_row = sum(v for k, v in t.items() if k != "a1") * row_frac
    per_tile = tile_time / max(1, tiles_done) * (gx * gy)
    return {"seconds_per_step": per_row + per_tile, "sampled_seconds": sum(t.values()) + tile_time,
            "row_frac": row_frac, "tiles": tiles_done, "n_tiles": gx * gy,
            "a1_seconds": t["a1"] * row_frac}


def oracle_iteration(d) -> float:
    """Seconds of one whole oracle iteration a2-a10 (cluster cull, preprocess,
    binning, forward, L1, backward, variance, preprocess backward, Adam) on
    workload d; the Morton re-sort (a1, run at intervals) is untimed setup."""
    import oracle
    from paper_2503_01199_gb300 import pipeline as PL
    sc, cam, tgt = d["scene"], d["camera"], d["target"]
    _, perm = oracle.morton_reorder(sc)
    sc = {k: (np.asarray(v, np.float64)[perm] if k != "sh_degree" else v) for k, v in sc.items()}
    planes = oracle.scene_planes(sc)
    m, v = np.zeros_like(planes), np.zeros_like(planes)
    lr = np.asarray(PL.lr_per_plane(sc["sh_degree"]), np.float64)
    a = time.perf_counter()
    cc = oracle.cluster_cull(sc, cam, 128)
    rows = cc["map"]
    sub = {k: (v_[rows] if k != "sh_degree" else v_) for k, v_ in sc.items()}
    r = oracle.render_scene(sub, cam, TILE)
    _, dL = oracle.l1_loss(r["image"], tgt)
    bw = oracle.render_bwd(r["splats"], r["vals"], r["ranges"], cam, dL, TILE)
    oracle.opacity_variance(bw["S"], bw["M"], bw["C"])
    g = oracle.grad_planes(oracle.preprocess_bwd(sub, cam, bw["grad9"]))
    gp = np.zeros_like(planes)
    gp[:, rows] = g
    oracle.adam(planes, gp, m, v, lr, 1, rows.astype(np.uint32))
    return time.perf_counter() - a


def cpu_baseline(d) -> dict:
    """The oracle on the host cores: whole iterations of the 4,096-Gaussian
    128x128 case (1 core and all cores) and of the 500K 1297x840 surface
    scene (all cores), measured; and the bench workload itself from a
    bounded sample scaled to one iteration (`value`, marked extrapolated)."""
    import oracle
    from paper_2503_01199_gb300 import scenegen
    oracle.build()
    full = {}
    small = scenegen.uniform_box_scene(4096, 0, 0, 128, 128)
    for name, cores in (("4096_sh0_128x128_1_core", 1), ("4096_sh0_128x128_all_cores", None)):
        oracle.set_threads(cores)
        secs = min(oracle_iteration(small) for _ in range(3))
        full[name] = {"cores": oracle.threads(), "seconds": round(secs, 4),
                      "iters_per_s": round(1.0 / secs, 3)}
    oracle.set_threads(None)
    secs = oracle_iteration(scenegen.surface_scene(500_000, SH_DEG, 1, W_IMG, H_IMG))
    full["500k_sh3_1297x840_all_cores"] = {"cores": oracle.threads(), "seconds": round(secs, 3),
                                           "iters_per_s": round(1.0 / secs, 4)}
    # every Gaussian for the per-Gaussian stages, 300 random 4x4-tile blocks
    # (about 4,800 tile visits for 4,346 tiles) for the per-tile ones
    r = cpu_step_sample(d, row_frac=1, n_blocks=300)
    rows = ("all Gaussians" if r["row_frac"] == 1 else
            f"1 of every {r['row_frac']} Gaussians (x{r['row_frac']})")
    return {"value": round(1.0 / r["seconds_per_step"], 5), "unit": UNIT,
            "cores": oracle.threads(), "kind": "oracle", "extrapolated": True,
            "sample": (f"oracle iteration a2-a10 at the bench workload, extrapolated: per-Gaussian "
                       f"stages on {rows}, per-tile stages (binning, forward, loss, backward) on "
                       f"{r['tiles']} tile visits in random 4x4-tile blocks scaled to the "
                       f"{r['n_tiles']} tiles; {r['sampled_seconds']:.1f} s of CPU work"),
            "full_iterations": full}


def run_reference(args):
    """The oracle as the reference arm: each step times the oracle on a
    bounded sample of the bench workload (1 of every 300 Gaussians for the
    per-Gaussian stages, 4 random 4x4-tile blocks for the per-tile ones);
    `ms_per_step` is the sampled time actually spent per step and `value` the
    full iteration rate extrapolated from the samples (`extrapolated`)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    d = make_workload()
    for _ in range(args.warmup):
        cpu_step_sample(d, row_frac=600, n_blocks=1)
    full_s, spent_s = [], []
    samp = None
    for k in range(args.steps):
        r = cpu_step_sample(d, row_frac=300, n_blocks=4, seed=k)
        full_s.append(r["seconds_per_step"])
        spent_s.append(r["sampled_seconds"])
        samp = r
    value = 1.0 / float(np.mean(full_s))
    sample = (f"each step: the oracle's a2-a10 iteration on 1 of every {samp['row_frac']} "
              f"Gaussians and {samp['tiles']} of the {samp['n_tiles']} tiles, scaled to the full "
              f"iteration")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(spent_s)), 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": bench_config(1),
           "extrapolated": True,
           "extrapolation": {"full_iteration_ms": round(1e3 * float(np.mean(full_s)), 1),
                             "full_iteration_ms_std": round(1e3 * float(np.std(full_s)), 1),
                             "sampled_ms_per_step": round(1e3 * float(np.mean(spent_s)), 2),
                             "row_fraction": f"1/{samp['row_frac']}",
                             "tiles_per_step": samp["tiles"], "n_tiles": samp["n_tiles"]},
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": oracle.threads(),
                            "kind": "oracle", "extrapolated": True, "sample": sample},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-gaussians", type=int, default=None,
                    help="smaller scene for profiling captures (not a bench line)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served-render request stream (0: skip)")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the Cluster-Cull-Compact / storage-order ablation")
    ap.add_argument("--storage", default="morton", choices=["morton", "shuffled"],
                    help="row order of the scene: Morton-sorted (the bench line) or shuffled "
                         "and never re-sorted (profiling evidence for the re-sort)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)
    out = run_gpu(args)
    if out is None:
        return
    if args.storage != "morton":
        out["config"]["workload"] = ("storage-order case (rows shuffled, never re-sorted): " +
                                     out["config"]["workload"].replace(", Morton-sorted", ""))
    if args.n_gaussians:
        out["config"]["n_gaussians"] = args.n_gaussians
        out["config"]["workload"] = "profiling case: " + out["config"]["workload"].replace(
            "3M Gaussians", f"{args.n_gaussians} Gaussians")
    out["serving"] = (run_serving(args.serve_seconds)
                      if args.serve_seconds > 0 and not args.n_gaussians else None)
    out["ccc_ablation"] = (run_ccc_ablation()
                           if not args.no_ablation and not args.n_gaussians else None)
    out["other_configs"] = (run_extra_configs(args.steps, args.warmup)
                            if not args.n_gaussians else None)
    if out["n_gpus"] == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(make_workload())
    else:
        out["cpu_baseline"] = None
    print(json.dumps(out))


if __name__ == "__main__":
    main()
