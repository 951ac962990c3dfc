"""Continuous-batching render server over resident scenes (forward renders).

Scenes stay resident on the device: the geometric planes 0..10 in float32,
the colour coefficients in BF16 (LGS_SH_BF16), each scene Morton-sorted once
at load (Sec. 3.2.1) so that the cluster cull works on compact clusters.

Admission is by HBM budget. A request needs scratch in proportion to its
resolution (tile lists, binning workspace, image), so the budget buys slots
of several classes: a class is a largest resolution and a (tile, splat)
pair capacity scaled to its tile count, and `plan_slots` splits the budget
over the classes so that small requests, which need several times less
memory, get more slots. Every slot has its own CUDA stream, pinned pose,
image and pair-count buffers, and one CUDA graph per (scene, resolution it
fits) holding a whole request: pose upload, cluster cull + compaction,
preprocess, binning, forward raster, image and pair count download. The
cull and the preprocess read the pose from device memory
(lgs_camera.d_pose), so a graph captured once is replayed for every camera.

Requests wait in arrival order; at each scheduling step the first `window`
queued requests each take the smallest free slot that fits them (a request
behind one that must wait for a large slot may start first), so requests
arriving while others are on the GPU start as slots free up and the slots'
streams overlap on the device. A request whose tile lists overflowed its
slot's pair capacity (the pair count comes back with the image) is run
again in the next larger class, so no truncated render is returned.

`Scheduler` is the host logic alone (queue, admission, completion, retry)
and runs with any executor; `GpuExecutor` is the device side.
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
    """Queue over a fixed set of slots. An executor provides
    start(slot, req), done(slot) -> bool and finish(slot, req) (returning
    False asks for the request to be run again in a larger class), and
    optionally fits(slot, req) -> bool and slot_class(slot) -> int (slots of
    a smaller class are preferred; without them every slot fits every
    request). Each step admits, in queue order, each of the first `window`
    queued requests that a free slot fits."""

    def __init__(self, n_slots: int, executor, window: int = 64):
        if n_slots < 1:
            raise ValueError("at least one slot")
        self.ex = executor
        self.window = int(window)
        self.free = list(range(n_slots))
        self.queue = collections.deque()
        self.inflight = {}
        self.completed = []
        self.max_inflight = 0
        self.max_group = 0
        self.retries = 0
        self._fits = getattr(executor, "fits", None)
        self._cls = getattr(executor, "slot_class", None)

    def submit(self, req: dict, now: float):
        req["t_submit"] = now
        self.queue.append(req)

    def _pick(self, req: dict):
        best, best_cls = None, None
        lo = req.get("min_class", 0)
        for s in self.free:
            c = self._cls(s) if self._cls else 0
            if c < lo or (self._fits and not self._fits(s, req)):
                continue
            if best is None or c < best_cls:
                best, best_cls = s, c
        return best

    def step(self, now: float):
        for slot, req in list(self.inflight.items()):
            if self.ex.done(slot):
                ok = self.ex.finish(slot, req)
                del self.inflight[slot]
                self.free.append(slot)
                if ok is False:   # overflowed its slot: again, in a larger class
                    self.retries += 1
                    req["retries"] = req.get("retries", 0) + 1
                    req["min_class"] = (self._cls(slot) if self._cls else 0) + 1
                    self.queue.appendleft(req)
                else:
                    req["t_done"] = now
                    self.completed.append(req)
        group = []
        if self.queue and self.free:
            kept = collections.deque()
            scanned = 0
            while self.queue and scanned < self.window and self.free:
                req = self.queue.popleft()
                scanned += 1
                slot = self._pick(req)
                if slot is None:
                    kept.append(req)
                    continue
                self.free.remove(slot)
                req["t_start"] = now
                req["slot"] = slot
                group.append((slot, req))
                self.inflight[slot] = req
            kept.extend(self.queue)
            self.queue = kept
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


def plan_slots(budget_bytes: int, class_bytes: list, shares: list) -> list:
    """Slots per class for a device-memory budget: one of every class with a
    share of the requests, then each further slot to the class whose share
    per slot is largest among those that still fit, until none fits.
    class_bytes[c]: bytes of one slot of class c; shares[c]: the fraction of
    requests that class c is the smallest fit for."""
    counts = [1 if s > 0 else 0 for s in shares]
    used = sum(n * b for n, b in zip(counts, class_bytes))
    if used > budget_bytes:
        raise ValueError("the budget does not hold one slot of every class")
    while True:
        best = None
        for c, (b, s) in enumerate(zip(class_bytes, shares)):
            if s <= 0 or used + b > budget_bytes:
                continue
            key = s / (counts[c] + 1)
            if best is None or key > best[0]:
                best = (key, c)
        if best is None:
            return counts
        counts[best[1]] += 1
        used += class_bytes[best[1]]


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
        self.sh16 = torch.zeros((npl - 11, self.stride), dtype=sh_dtype, device=device)
        B.lgs_round_planes(dst[11:], self.sh16, npl - 11, self.n)
        del full, dst, codes, perm, ws

    def struct(self) -> B.LgsGaussians:
        return B.gaussians_struct(self.geom, self.n, self.sh_degree, sh16=self.sh16)


def slot_bytes(max_n: int, max_w: int, max_h: int, pair_capacity: int, tile=(16, 16),
               cluster: int = 128) -> int:
    """Device bytes one slot holds (scratch for its largest request)."""
    tw, th = tile
    ntiles = -(-max_w // tw) * -(-max_h // th)
    per_splat = 4 + B.SPLAT_FLOATS * 4 + 4 + 4  # map, record, depth, radius
    image = max_w * max_h * (3 * 4 + 4 + 4)  # image, final T, last
    return int(max_n * per_splat + 4 * pair_capacity + 8 * ntiles + image +
               B.lgs_bin_sort_workspace_size(max_n, pair_capacity, ntiles) +
               B.lgs_ccc_workspace_size(max_n, cluster) + 4 * (-(-max_n // cluster)) + 64)


def class_capacity(w: int, h: int, max_n: int, ref_w: int, ref_h: int, ref_capacity: int,
                   tile=(16, 16)) -> int:
    """Pair capacity of a class of largest resolution w x h, from a known
    capacity at ref_w x ref_h: scaled with the tile count, plus one pair per
    Gaussian (a small splat is listed in one tile whatever the resolution),
    at least 4M. A request that needs more is run again in a larger class."""
    tiles = -(-w // tile[0]) * -(-h // tile[1])
    ref = -(-ref_w // tile[0]) * -(-ref_h // tile[1])
    return int(min(ref_capacity, max(4_000_000, ref_capacity * tiles // ref + max_n)))


class _Slot:
    def __init__(self, max_n, max_w, max_h, cap, tile, cluster, cls, dev):
        tw, th = tile
        ntiles = -(-max_w // tw) * -(-max_h // th)
        self.max_w, self.max_h, self.cap, self.cls = max_w, max_h, int(cap), cls
        self.stream = torch.cuda.Stream(device=dev)
        self.event = torch.cuda.Event()
        self.rowmap = torch.empty(max_n, dtype=torch.int32, device=dev)
        self.d_V = torch.zeros(1, dtype=torch.int32, device=dev)
        self.rec = torch.empty((max_n, B.SPLAT_FLOATS), dtype=torch.float32, device=dev)
        self.depth = torch.empty(max_n, dtype=torch.float32, device=dev)
        self.radius = torch.empty(max_n, dtype=torch.int32, device=dev)
        self.vals = torch.empty(cap, dtype=torch.int32, device=dev)
        self.d_P = torch.zeros(1, dtype=torch.int64, device=dev)
        self.h_P = torch.zeros(1, dtype=torch.int64).pin_memory()
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

    def fits(self, w: int, h: int) -> bool:
        return w <= self.max_w and h <= self.max_h


class GpuExecutor:
    """Runs requests {'scene': index, 'camera': scenegen camera dict} on slots.

    `slots` is either a count (every slot of one class: the largest of
    `resolutions`, `pair_capacity` pairs) or a list of classes
    (max_w, max_h, pair_capacity, count), smallest first. With use_graphs
    each request is one replay of a graph captured per (slot, scene,
    resolution it fits); without, the calls are issued one by one. With
    grouped, the requests admitted together run their front ends (pose
    upload, cull + compaction, preprocess, binning: graphs per slot, scene
    and resolution) on their slots' streams and are then rendered by ONE
    persistent batched raster launch over all their tiles
    (lgs_raster_fwd_batch); each image is copied back on its slot's stream.
    finish() returns False for a request whose binning overflowed its slot's
    pair capacity (its image is not used)."""

    def __init__(self, scenes: list, slots, resolutions, pair_capacity: int,
                 tile=(16, 16), cluster: int = 128, use_graphs: bool = True,
                 keep_images: bool = False, grouped: bool = False, device="cuda"):
        self.scenes = scenes
        self.tile, self.cluster = tuple(tile), int(cluster)
        self.use_graphs, self.keep_images = use_graphs or grouped, keep_images
        self.grouped = grouped
        self.dev = torch.device(device)
        self.max_n = max(s.n for s in scenes)
        self.resolutions = [tuple(r) for r in resolutions]
        if isinstance(slots, int):
            classes = [(max(w for w, _ in resolutions), max(h for _, h in resolutions),
                        int(pair_capacity), slots)]
        else:
            classes = [tuple(c) for c in slots]
        self.classes = classes
        self.slots = [_Slot(self.max_n, w, h, cap, self.tile, self.cluster, ci, self.dev)
                      for ci, (w, h, cap, count) in enumerate(classes) for _ in range(count)]
        self.overflowed = 0
        self.final_overflow = 0
        self.structs = [s.struct() for s in scenes]
        if grouped:
            self.gstream = torch.cuda.Stream(device=self.dev)
            self.gevent = torch.cuda.Event()
            self.counter = torch.zeros(1, dtype=torch.int32, device=self.dev)
            n = len(self.slots)
            self.table_dev = torch.empty(n * ctypes_sizeof_view(), dtype=torch.uint8,
                                         device=self.dev)
            self.table_host = torch.empty(n * ctypes_sizeof_view(), dtype=torch.uint8).pin_memory()
            self.table_copied = torch.cuda.Event()
            self.table_copied.record(self.gstream)
        if self.use_graphs:
            for slot in self.slots:
                for si in range(len(scenes)):
                    for (w, h) in self.resolutions:
                        if slot.fits(w, h):
                            self._capture(slot, si, w, h, front_only=grouped)
        torch.cuda.synchronize()

    # -- slot classes ----------------------------------------------------------
    def fits(self, k: int, req: dict) -> bool:
        cam = req["camera"]
        return self.slots[k].fits(int(cam["width"]), int(cam["height"]))

    def slot_class(self, k: int) -> int:
        return self.slots[k].cls

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
        slot.h_P.copy_(slot.d_P, non_blocking=True)
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

    @staticmethod
    def _pose(cam) -> np.ndarray:
        return np.concatenate([np.asarray(cam["R"], np.float32).reshape(9),
                               np.asarray(cam["t"], np.float32).reshape(3)])

    def start_group(self, group: list):
        """Front ends of every request of the group on their slots' streams,
        one batched raster over all their tiles, images back per slot."""
        views = []
        for k, req in group:
            slot = self.slots[k]
            cam = req["camera"]
            w, h = int(cam["width"]), int(cam["height"])
            graph, _ = slot.graphs[(req["scene"], w, h)]
            slot.h_pose.numpy()[:] = self._pose(cam)
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
        with torch.cuda.stream(slot.stream):
            if self.use_graphs:
                graph, _ = slot.graphs[(req["scene"], w, h)]
                slot.h_pose.numpy()[:] = self._pose(cam)
                graph.replay()
            else:
                self._issue(slot, req["scene"], B.camera_struct(cam))
                slot.h_image[:3 * w * h].copy_(slot.image[:3 * w * h], non_blocking=True)
            slot.event.record(slot.stream)

    def done(self, k: int) -> bool:
        return self.slots[k].event.query()

    def finish(self, k: int, req: dict) -> bool:
        slot = self.slots[k]
        req["pairs"] = int(slot.h_P[0])
        if req["pairs"] > slot.cap:
            self.overflowed += 1
            if slot.cls + 1 < len(self.classes):
                return False
            req["overflow"] = True    # no larger class: done, but its lists were cut
            self.final_overflow += 1
        if self.keep_images:
            cam = req["camera"]
            w, h = int(cam["width"]), int(cam["height"])
            req["image"] = slot.h_image[:3 * w * h].numpy().reshape(3, h, w).copy()
        return True

    def overflow(self) -> int:
        """Completed requests whose tile lists were cut (an overflow is run
        again in a larger class, so only the largest class can leave one)."""
        B.lgs_get_overflow()   # clear the library's flag, set by the retried ones too
        return self.final_overflow


def ctypes_sizeof_view() -> int:
    import ctypes
    return ctypes.sizeof(B.LgsView)


def serve(scenes: list, requests: list, hbm_budget_bytes: int, resolutions,
          pair_capacity: int, use_graphs: bool = True, keep_images: bool = False,
          max_slots: int | None = None, grouped: bool = False, classes=None) -> dict:
    """Builds the server for the budget, replays the request stream in real
    time and returns latency / throughput statistics.

    classes: None for one class of slots (the largest resolution with
    pair_capacity pairs, as many as the budget pays for, at most max_slots),
    or a list of (max_w, max_h, pair_capacity) smallest first, whose slot
    counts plan_slots takes from the budget, each class weighted by the
    share of requests it is the smallest fit for."""
    max_n = max(s.n for s in scenes)
    if classes is None:
        need = slot_bytes(max_n, max(w for w, _ in resolutions), max(h for _, h in resolutions),
                          pair_capacity)
        n_slots = max(1, int(hbm_budget_bytes // need))
        if max_slots:
            n_slots = min(n_slots, max_slots)
        slots = n_slots
        plan = [{"max_w": max(w for w, _ in resolutions), "max_h": max(h for _, h in resolutions),
                 "pair_capacity": int(pair_capacity), "slots": n_slots, "slot_bytes": need}]
    else:
        res = [tuple(r) for r in resolutions]
        cbytes = [slot_bytes(max_n, w, h, cap) for w, h, cap in classes]
        first = []
        for w, h in res:
            first.append(next(c for c, (cw, ch, _) in enumerate(classes) if w <= cw and h <= ch))
        shares = [first.count(c) / len(first) for c in range(len(classes))]
        counts = plan_slots(hbm_budget_bytes, cbytes, shares)
        slots = [(w, h, cap, n) for (w, h, cap), n in zip(classes, counts) if n]
        n_slots = sum(counts)
        plan = [{"max_w": w, "max_h": h, "pair_capacity": int(cap), "slots": n, "slot_bytes": b}
                for (w, h, cap), n, b in zip(classes, counts, cbytes) if n]
    ex = GpuExecutor(scenes, slots, resolutions, pair_capacity, use_graphs=use_graphs,
                     keep_images=keep_images, grouped=grouped)
    sch = Scheduler(len(ex.slots), ex)
    wall = replay(sch, requests)
    torch.cuda.synchronize()
    stats = latency_stats(sch.completed, wall)
    stats.update({"slots": n_slots, "slot_classes": plan, "max_inflight": sch.max_inflight,
                  "max_group": sch.max_group, "retries": sch.retries,
                  "pair_overflow": ex.overflow()})
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
        ex.finish(0, r)
        r["t_done"] = time.perf_counter() - t0
        done.append(r)
    wall = time.perf_counter() - t0
    stats = latency_stats(done, wall)
    stats["pair_overflow"] = ex.overflow()
    return {"stats": stats}
