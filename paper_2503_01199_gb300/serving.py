"""Continuous-batching render server over resident scenes (forward renders).

Scenes stay resident on the device: the geometric planes 0..10 in float32,
the colour coefficients in BF16 (LGS_SH_BF16), each scene Morton-sorted once
at load (Sec. 3.2.1) so that the cluster cull works on compact clusters.

Admission is by HBM budget: the server holds as many slots as the budget
pays for, each with scratch for the largest scene at the largest
resolution, its own CUDA stream, a pinned pose buffer and a pinned image
buffer. Per slot and per (scene, resolution) one CUDA graph holds a whole
request: pose upload, cluster cull + compaction, preprocess, binning,
forward raster and image download; the cull and the preprocess read the
pose from device memory (lgs_camera.d_pose), so a graph captured once is
replayed for every camera. Requests wait in arrival order and start as soon
as a slot is free, including while other requests are on the GPU; the
slots' streams overlap on the device.

`Scheduler` is the host logic alone (queue, admission, completion) and runs
with any executor; `GpuExecutor` is the device side.
"""
from __future__ import annotations

import collections
import time

import numpy as np
import torch

from . import binding as B
from . import pipeline as PL


# ---------------------------------------------------------------------------
# host scheduling
# ---------------------------------------------------------------------------
class Scheduler:
    """FIFO queue over a fixed set of slots. An executor provides
    start(slot, req), done(slot) -> bool and finish(slot, req)."""

    def __init__(self, n_slots: int, executor):
        if n_slots < 1:
            raise ValueError("at least one slot")
        self.ex = executor
        self.free = list(range(n_slots - 1, -1, -1))
        self.queue = collections.deque()
        self.inflight = {}
        self.completed = []
        self.max_inflight = 0
        self.max_group = 0

    def submit(self, req: dict, now: float):
        req["t_submit"] = now
        self.queue.append(req)

    def step(self, now: float):
        for slot, req in list(self.inflight.items()):
            if self.ex.done(slot):
                req["t_done"] = now
                self.ex.finish(slot, req)
                del self.inflight[slot]
                self.free.append(slot)
                self.completed.append(req)
        group = []
        while self.queue and self.free:
            slot = self.free.pop()
            req = self.queue.popleft()
            req["t_start"] = now
            req["slot"] = slot
            group.append((slot, req))
            self.inflight[slot] = req
        if group:
            if getattr(self.ex, "grouped", False):
                self.ex.start_group(group)   # one launch renders the whole group
            else:
                for slot, req in group:
                    self.ex.start(slot, req)
            self.max_group = max(self.max_group, len(group))
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def idle(self) -> bool:
        return not self.queue and not self.inflight


def replay(scheduler: Scheduler, requests: list, clock=time.perf_counter) -> float:
    """Feeds `requests` (sorted by 'arrival', seconds) to the scheduler in
    real time and runs it until every request is done; returns the wall time."""
    t0 = clock()
    i = 0
    while i < len(requests) or not scheduler.idle():
        now = clock() - t0
        while i < len(requests) and requests[i]["arrival"] <= now:
            scheduler.submit(requests[i], now)
            i += 1
        scheduler.step(clock() - t0)
    return clock() - t0


def latency_stats(requests: list, wall_s: float) -> dict:
    lat = np.array([r["t_done"] - r["arrival"] for r in requests]) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "frames_per_s": round(len(requests) / wall_s, 2), "requests": len(requests)}


# ---------------------------------------------------------------------------
# device side
# ---------------------------------------------------------------------------
class ResidentScene:
    """A scene kept on the device for rendering: Morton-sorted float32
    geometry planes [11][stride] and 16-bit colour planes [3K][stride]."""

    def __init__(self, scene: dict, sh_dtype=torch.bfloat16, device="cuda"):
        self.sh_degree = int(scene["sh_degree"])
        self.n = int(scene["mean"].shape[0])
        self.stride = PL.round_up(max(self.n, 1), 128)
        npl = B.num_planes(self.sh_degree)
        full = torch.zeros((npl, self.stride), dtype=torch.float32, device=device)
        full[:, :self.n].copy_(torch.from_numpy(PL.pack_planes(scene)).to(device))
        dst = torch.empty_like(full)
        codes = torch.empty(self.n, dtype=torch.int64, device=device)
        perm = torch.empty(self.n, dtype=torch.int32, device=device)
        ws = torch.empty(B.lgs_morton_workspace_size(self.n), dtype=torch.uint8, device=device)
        B.lgs_morton_reorder(full, dst, self.n, npl, codes, perm, ws)
        self.geom = dst[:11].contiguous()
        self.sh16 = dst[11:].to(sh_dtype).contiguous()
        del full, dst, codes, perm, ws

    def struct(self) -> B.LgsGaussians:
        return B.gaussians_struct(self.geom, self.n, self.sh_degree, sh16=self.sh16)


def slot_bytes(max_n: int, max_w: int, max_h: int, pair_capacity: int, tile=(16, 16),
               cluster: int = 128) -> int:
    """Device bytes one slot holds (scratch for the largest request)."""
    tw, th = tile
    ntiles = -(-max_w // tw) * -(-max_h // th)
    per_splat = 4 + B.SPLAT_FLOATS * 4 + 4 + 4  # map, record, depth, radius
    image = max_w * max_h * (3 * 4 + 4 + 4)  # image, final T, last
    return int(max_n * per_splat + 4 * pair_capacity + 8 * ntiles + image +
               B.lgs_bin_sort_workspace_size(max_n, pair_capacity, ntiles) +
               B.lgs_ccc_workspace_size(max_n, cluster) + 4 * (-(-max_n // cluster)) + 64)


class _Slot:
    def __init__(self, max_n, max_w, max_h, cap, tile, cluster, dev):
        tw, th = tile
        ntiles = -(-max_w // tw) * -(-max_h // th)
        self.stream = torch.cuda.Stream(device=dev)
        self.event = torch.cuda.Event()
        self.rowmap = torch.empty(max_n, dtype=torch.int32, device=dev)
        self.d_V = torch.zeros(1, dtype=torch.int32, device=dev)
        self.rec = torch.empty((max_n, B.SPLAT_FLOATS), dtype=torch.float32, device=dev)
        self.depth = torch.empty(max_n, dtype=torch.float32, device=dev)
        self.radius = torch.empty(max_n, dtype=torch.int32, device=dev)
        self.vals = torch.empty(cap, dtype=torch.int32, device=dev)
        self.d_P = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ranges = torch.empty((ntiles, 2), dtype=torch.int32, device=dev)
        self.ws_bin = torch.empty(B.lgs_bin_sort_workspace_size(max_n, cap, ntiles),
                                  dtype=torch.uint8, device=dev)
        self.ws_ccc = torch.empty(B.lgs_ccc_workspace_size(max_n, cluster), dtype=torch.uint8,
                                  device=dev)
        self.cluster_visible = torch.empty(-(-max_n // cluster), dtype=torch.int32, device=dev)
        self.image = torch.empty(3 * max_w * max_h, dtype=torch.float32, device=dev)
        self.finalT = torch.empty(max_w * max_h, dtype=torch.float32, device=dev)
        self.last = torch.empty(max_w * max_h, dtype=torch.int32, device=dev)
        self.d_pose = torch.zeros(12, dtype=torch.float32, device=dev)
        self.h_pose = torch.zeros(12, dtype=torch.float32).pin_memory()
        self.h_image = torch.empty(3 * max_w * max_h, dtype=torch.float32).pin_memory()
        self.splats = B.splats_struct(self.rec, self.depth, self.radius)
        self.graphs = {}


class GpuExecutor:
    """Runs requests {'scene': index, 'camera': scenegen camera dict} on slots.
    With use_graphs each request is one replay of a graph captured per
    (slot, scene, resolution); without, the calls are issued one by one.
    With grouped, the requests admitted together run their front ends (pose
    upload, cull + compaction, preprocess, binning: graphs per slot, scene
    and resolution) on their slots' streams and are then rendered by ONE
    persistent batched raster launch over all their tiles
    (lgs_raster_fwd_batch); each image is copied back on its slot's stream."""

    def __init__(self, scenes: list, n_slots: int, resolutions, pair_capacity: int,
                 tile=(16, 16), cluster: int = 128, use_graphs: bool = True,
                 keep_images: bool = False, grouped: bool = False, device="cuda"):
        self.scenes = scenes
        self.tile, self.cluster = tuple(tile), int(cluster)
        self.use_graphs, self.keep_images = use_graphs or grouped, keep_images
        self.grouped = grouped
        self.dev = torch.device(device)
        self.max_n = max(s.n for s in scenes)
        self.max_w = max(w for w, _ in resolutions)
        self.max_h = max(h for _, h in resolutions)
        self.cap = int(pair_capacity)
        self.slots = [_Slot(self.max_n, self.max_w, self.max_h, self.cap, self.tile, self.cluster,
                            self.dev) for _ in range(n_slots)]
        self.structs = [s.struct() for s in scenes]
        if grouped:
            self.gstream = torch.cuda.Stream(device=self.dev)
            self.gevent = torch.cuda.Event()
            self.counter = torch.zeros(1, dtype=torch.int32, device=self.dev)
            self.table_dev = torch.empty(n_slots * ctypes_sizeof_view(), dtype=torch.uint8,
                                         device=self.dev)
            self.table_host = torch.empty(n_slots * ctypes_sizeof_view(),
                                          dtype=torch.uint8).pin_memory()
            self.table_copied = torch.cuda.Event()
            self.table_copied.record(self.gstream)
        if self.use_graphs:
            for k, slot in enumerate(self.slots):
                for si in range(len(scenes)):
                    for (w, h) in resolutions:
                        self._capture(slot, si, w, h, front_only=grouped)
        torch.cuda.synchronize()

    # -- the calls of one request on the slot's current stream ---------------
    def _issue(self, slot: _Slot, si: int, cs: B.LgsCamera, front_only: bool = False):
        tw, th = self.tile
        g = self.structs[si]
        W, H = cs.width, cs.height
        B.lgs_cluster_cull_compact(g, cs, self.cluster, None, slot.cluster_visible, slot.rowmap,
                                   slot.d_V, slot.ws_ccc)
        B.lgs_preprocess(g, slot.rowmap, slot.d_V, cs, tw, th, slot.splats)
        ntiles = -(-W // tw) * -(-H // th)
        B.lgs_bin_sort(slot.splats, slot.d_V, self.scenes[si].n, cs, tw, th, slot.vals,
                       slot.d_P, slot.ranges[:ntiles], slot.ws_bin)
        if not front_only:
            B.lgs_raster_fwd(slot.splats, slot.vals, slot.ranges[:ntiles], cs, tw, th,
                             slot.image[:3 * W * H], slot.finalT[:W * H], slot.last[:W * H])

    def _capture(self, slot: _Slot, si: int, w: int, h: int, front_only: bool = False):
        from . import scenegen
        cam = scenegen.orbit_camera(4.0, 0.0, 0.0, w, h, center=scenegen.BOX_CENTER)
        cs = B.camera_struct(cam, d_pose=slot.d_pose)
        slot.d_pose.copy_(torch.from_numpy(np.concatenate(
            [np.asarray(cam["R"], np.float32).reshape(9), np.asarray(cam["t"], np.float32)])))
        with torch.cuda.stream(slot.stream):   # warm-up run outside the capture
            self._issue(slot, si, cs)
        slot.stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=slot.stream):
            slot.d_pose.copy_(slot.h_pose, non_blocking=True)
            self._issue(slot, si, cs, front_only=front_only)
            if not front_only:
                slot.h_image[:3 * w * h].copy_(slot.image[:3 * w * h], non_blocking=True)
        # one replay now, so that no request pays for the graph's first upload
        slot.h_pose.copy_(slot.d_pose.cpu())
        with torch.cuda.stream(slot.stream):
            graph.replay()
        slot.stream.synchronize()
        slot.graphs[(si, w, h)] = (graph, cs)

    def start_group(self, group: list):
        """Front ends of every request of the group on their slots' streams,
        one batched raster over all their tiles, images back per slot."""
        views = []
        for k, req in group:
            slot = self.slots[k]
            cam = req["camera"]
            w, h = int(cam["width"]), int(cam["height"])
            graph, _ = slot.graphs[(req["scene"], w, h)]
            slot.h_pose.numpy()[:] = np.concatenate([np.asarray(cam["R"], np.float32).reshape(9),
                                                     np.asarray(cam["t"], np.float32).reshape(3)])
            with torch.cuda.stream(slot.stream):
                graph.replay()
                slot.event.record(slot.stream)
            self.gstream.wait_event(slot.event)
            ntiles = -(-w // self.tile[0]) * -(-h // self.tile[1])
            views.append({"camera": cam, "rec": slot.rec, "vals": slot.vals,
                          "ranges": slot.ranges[:ntiles], "image": slot.image[:3 * w * h],
                          "final_T": slot.finalT[:w * h], "last": slot.last[:w * h]})
        raw, total = B.view_table_bytes(views, self.tile)
        self.table_copied.synchronize()   # the previous group's table has left the pinned buffer
        with torch.cuda.stream(self.gstream):
            self.table_host.numpy()[:len(raw)] = np.frombuffer(raw, np.uint8)
            self.table_dev[:len(raw)].copy_(self.table_host[:len(raw)], non_blocking=True)
            self.table_copied.record(self.gstream)
            B.lgs_raster_fwd_batch(self.table_dev, len(views), total, self.counter)
            self.gevent.record(self.gstream)
        for k, req in group:
            slot = self.slots[k]
            cam = req["camera"]
            w, h = int(cam["width"]), int(cam["height"])
            slot.stream.wait_event(self.gevent)
            with torch.cuda.stream(slot.stream):
                slot.h_image[:3 * w * h].copy_(slot.image[:3 * w * h], non_blocking=True)
                slot.event.record(slot.stream)

    # -- executor interface ----------------------------------------------------
    def start(self, k: int, req: dict):
        slot = self.slots[k]
        cam = req["camera"]
        w, h = int(cam["width"]), int(cam["height"])
        pose = np.concatenate([np.asarray(cam["R"], np.float32).reshape(9),
                               np.asarray(cam["t"], np.float32).reshape(3)])
        with torch.cuda.stream(slot.stream):
            if self.use_graphs:
                graph, _ = slot.graphs[(req["scene"], w, h)]
                slot.h_pose.numpy()[:] = pose
                graph.replay()
            else:
                self._issue(slot, req["scene"], B.camera_struct(cam))
                slot.h_image[:3 * w * h].copy_(slot.image[:3 * w * h], non_blocking=True)
            slot.event.record(slot.stream)

    def done(self, k: int) -> bool:
        return self.slots[k].event.query()

    def finish(self, k: int, req: dict):
        if self.keep_images:
            cam = req["camera"]
            w, h = int(cam["width"]), int(cam["height"])
            req["image"] = self.slots[k].h_image[:3 * w * h].numpy().reshape(3, h, w).copy()

    def overflow(self) -> int:
        return B.lgs_get_overflow()


def ctypes_sizeof_view() -> int:
    import ctypes
    return ctypes.sizeof(B.LgsView)


def serve(scenes: list, requests: list, hbm_budget_bytes: int, resolutions,
          pair_capacity: int, use_graphs: bool = True, keep_images: bool = False,
          max_slots: int | None = None, grouped: bool = False) -> dict:
    """Builds the server for the budget, replays the request stream in real
    time and returns latency / throughput statistics."""
    need = slot_bytes(max(s.n for s in scenes), max(w for w, _ in resolutions),
                      max(h for _, h in resolutions), pair_capacity)
    n_slots = max(1, int(hbm_budget_bytes // need))
    if max_slots:
        n_slots = min(n_slots, max_slots)
    ex = GpuExecutor(scenes, n_slots, resolutions, pair_capacity, use_graphs=use_graphs,
                     keep_images=keep_images, grouped=grouped)
    sch = Scheduler(n_slots, ex)
    wall = replay(sch, requests)
    torch.cuda.synchronize()
    stats = latency_stats(sch.completed, wall)
    stats.update({"slots": n_slots, "slot_bytes": need, "max_inflight": sch.max_inflight,
                  "max_group": sch.max_group, "pair_overflow": ex.overflow()})
    return {"stats": stats, "completed": sch.completed, "executor": ex}


def plain_loop(scenes: list, requests: list, resolutions, pair_capacity: int) -> dict:
    """The per-request loop: one request at a time in arrival order, calls
    issued directly, waiting for each image before taking the next."""
    ex = GpuExecutor(scenes, 1, resolutions, pair_capacity, use_graphs=False)
    t0 = time.perf_counter()
    done = []
    for r in requests:
        while time.perf_counter() - t0 < r["arrival"]:
            pass
        ex.start(0, r)
        ex.slots[0].event.synchronize()
        r["t_done"] = time.perf_counter() - t0
        done.append(r)
    wall = time.perf_counter() - t0
    return {"stats": latency_stats(done, wall)}
