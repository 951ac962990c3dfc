"""One training step of the LiteGS rasterizer hot path on one GPU, as a
sequence of liblgs calls (Sec. 3 pipeline):

  a1 Morton re-sort of parameters and Adam moments        lgs_morton_reorder
  a2 cluster AABB frustum cull + compaction map           lgs_cluster_cull_compact
  a3 preprocess (EWA projection, SH colour, opacity)      lgs_preprocess
  a4 tile binning + depth/tile sort                       lgs_bin_sort
  a5 forward rasterisation                                lgs_raster_fwd
  a6 L1 loss gradient                                     lgs_loss_l1
  a7 backward rasterisation + opacity-gradient moments    lgs_raster_bwd
  a8 densification metric C Var = S - M^2/C               lgs_opacity_variance
                                                          (in the fused a9 + a10 call of a step)
  a9 preprocess backward + a10 sparse Adam                lgs_preprocess_bwd_adam
                                                          (or lgs_preprocess_bwd + lgs_adam_step)

torch provides the device buffers and the stream; every step runs in the
library's kernels. All calls are asynchronous and no count is read back, so
the a2-a8 sequence (and a step's work) can be captured in a CUDA graph; the
Adam step count is a host argument, so a captured optimizer call would
replay one fixed step count.

Parameters and the two Adam moments live in one buffer of planes
[3][P][stride] (params, m, v) so that the Morton re-sort permutes all of
them in one gather; a second buffer of the same shape receives it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B

# Learning rates per parameter group: the common 3DGS set (the paper only
# says "same learning rates as TamingGS", Sec. 4, without printing them).
DEFAULT_LR = {"mean": 1.6e-4, "log_scale": 5e-3, "quat": 1e-3, "logit": 5e-2,
              "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20.0}


def lr_per_plane(sh_degree: int, lr: dict | None = None) -> list[float]:
    lr = dict(DEFAULT_LR, **(lr or {}))
    k = (sh_degree + 1) ** 2
    return ([lr["mean"]] * 3 + [lr["log_scale"]] * 3 + [lr["quat"]] * 4 + [lr["logit"]] +
            [lr["sh_dc"]] * 3 + [lr["sh_rest"]] * 3 * (k - 1))


def pack_planes(scene: dict) -> np.ndarray:
    """Scene dict (scenegen layout) -> float32 planes [P, N] in lgs.h order."""
    n = scene["mean"].shape[0]
    return np.ascontiguousarray(np.concatenate([
        np.asarray(scene["mean"], np.float32).T, np.asarray(scene["log_scale"], np.float32).T,
        np.asarray(scene["quat"], np.float32).T, np.asarray(scene["logit"], np.float32)[None],
        np.asarray(scene["sh"], np.float32).reshape(n, -1).T]))


def unpack_planes(planes: np.ndarray, sh_degree: int) -> dict:
    n = planes.shape[1]
    return {"mean": planes[0:3].T.copy(), "log_scale": planes[3:6].T.copy(),
            "quat": planes[6:10].T.copy(), "logit": planes[10].copy(),
            "sh": planes[11:].T.reshape(n, -1, 3).copy(), "sh_degree": sh_degree}


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


@dataclass
class StepConfig:
    tile: tuple = (16, 16)
    cluster: int = 128
    pair_capacity: int | None = None   # default: 64 pairs per Gaussian, at least 1M
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    lr: dict = field(default_factory=dict)
    # Cluster-Cull-Compact (Sec. 3.2.2); off: every row is processed each
    # step (culled Gaussians get zero gradients, Adam touches every row)
    ccc: bool = True
    # raster blend precision: B.LGS_FP32, LGS_MIXED_FP16 or LGS_MIXED_BF16
    precision: int = 0
    # colour coefficients read by the forward: "fp32", or "bf16" / "fp16" (a
    # rounded 16-bit copy of the FP32 planes, which stay the Adam masters;
    # the fused optimizer keeps the copy up to date, so fused=True only)
    sh_precision: str = "fp32"
    # every this many steps, step() reads the binning's overflow flag (a
    # host synchronisation; skipped while a CUDA graph is being captured)
    # and raises if any binning since the last read needed more pairs than
    # pair_capacity: the tile lists were then truncated (0: never)
    overflow_check_every: int = 64


class Trainer:
    """Device-resident scene + all step buffers for one camera size."""

    def __init__(self, scene: dict, width: int, height: int, cfg: StepConfig | None = None,
                 device: str = "cuda", capacity: int | None = None):
        self.cfg = cfg or StepConfig()
        self.dev = torch.device(device)
        self.sh_degree = int(scene["sh_degree"])
        self.n = int(scene["mean"].shape[0])
        self.np_ = B.num_planes(self.sh_degree)
        # rows available for densification; every per-Gaussian buffer is sized for it
        self.capacity = max(int(capacity or self.n), self.n)
        self.stride = round_up(max(self.capacity, 1), 128)
        self.W, self.H = int(width), int(height)
        tw, th = self.cfg.tile
        self.gx, self.gy = -(-self.W // tw), -(-self.H // th)
        self.ntiles = self.gx * self.gy
        n, dev = self.capacity, self.dev
        # [buffer][params, m, v][plane][row]
        self.state = torch.zeros((2, 3, self.np_, self.stride), dtype=torch.float32, device=dev)
        self.cur = 0
        planes = torch.from_numpy(pack_planes(scene))
        self.state[0, 0, :, :self.n].copy_(planes.to(dev))
        self.codes = torch.zeros(n, dtype=torch.int64, device=dev)
        self.perm = torch.zeros(n, dtype=torch.int32, device=dev)
        self.ws_morton = torch.empty(B.lgs_morton_workspace_size(n), dtype=torch.uint8, device=dev)
        ncl = -(-n // self.cfg.cluster)
        self.ws_ccc = torch.empty(B.lgs_ccc_workspace_size(n, self.cfg.cluster), dtype=torch.uint8,
                                  device=dev)
        self.cluster_visible = torch.zeros(ncl, dtype=torch.int32, device=dev)
        self.rowmap = torch.zeros(n, dtype=torch.int32, device=dev)
        self.d_V = torch.zeros(1, dtype=torch.int32, device=dev)
        self.rec = torch.zeros((n, B.SPLAT_FLOATS), dtype=torch.float32, device=dev)
        self.depth = torch.zeros(n, dtype=torch.float32, device=dev)
        self.radius = torch.zeros(n, dtype=torch.int32, device=dev)
        cap = self.cfg.pair_capacity or max(64 * n, 1 << 20)
        self.cap = int(cap)
        self.vals = torch.zeros(self.cap, dtype=torch.int32, device=dev)
        self.d_P = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ranges = torch.zeros((self.ntiles, 2), dtype=torch.int32, device=dev)
        self.ws_bin = torch.empty(B.lgs_bin_sort_workspace_size(n, self.cap, self.ntiles),
                                  dtype=torch.uint8, device=dev)
        self.image = torch.zeros((3, self.H, self.W), dtype=torch.float32, device=dev)
        self.finalT = torch.zeros((self.H, self.W), dtype=torch.float32, device=dev)
        self.last = torch.zeros((self.H, self.W), dtype=torch.int32, device=dev)
        self.dLdI = torch.zeros_like(self.image)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.gacc = torch.zeros((n, B.GRAD_FLOATS), dtype=torch.float32, device=dev)
        self.metric = torch.zeros(n, dtype=torch.float32, device=dev)
        # opacity-gradient moments summed over the views of a densification interval
        self.S_acc = torch.zeros(n, dtype=torch.float32, device=dev)
        self.M_acc = torch.zeros(n, dtype=torch.float32, device=dev)
        self.C_acc = torch.zeros(n, dtype=torch.int32, device=dev)
        self.track_moments = False
        self.grad_planes = None
        self.lr = lr_per_plane(self.sh_degree, self.cfg.lr)
        self.step_count = 0
        self.splats = B.splats_struct(self.rec, self.depth, self.radius)
        sh_types = {"fp32": None, "bf16": torch.bfloat16, "fp16": torch.float16}
        if self.cfg.sh_precision not in sh_types:
            raise ValueError(f"sh_precision must be one of {sorted(sh_types)}")
        self.sh16 = None
        if sh_types[self.cfg.sh_precision] is not None:
            self.sh16 = torch.zeros((self.np_ - 11, self.stride),
                                    dtype=sh_types[self.cfg.sh_precision], device=dev)
            self._round_sh16()

    # -- views ------------------------------------------------------------
    def _map(self):
        return self.rowmap if self.cfg.ccc else None

    def _dV(self):
        return self.d_V if self.cfg.ccc else None

    @property
    def params(self) -> torch.Tensor:
        return self.state[self.cur, 0]

    @property
    def m(self) -> torch.Tensor:
        return self.state[self.cur, 1]

    @property
    def v(self) -> torch.Tensor:
        return self.state[self.cur, 2]

    def gaussians(self) -> B.LgsGaussians:
        return B.gaussians_struct(self.params, self.n, self.sh_degree, sh16=self.sh16)

    def _g32(self) -> B.LgsGaussians:
        """The parameters with their FP32 colour planes (the calls that
        change parameters other than through Adam take these)."""
        return B.gaussians_struct(self.params, self.n, self.sh_degree)

    def _round_sh16(self):
        """The 16-bit colour copy of the FP32 colour planes (all live rows)."""
        if self.sh16 is not None:
            B.lgs_round_planes(self.params[11:], self.sh16, self.np_ - 11, self.n)

    # -- steps ------------------------------------------------------------
    def morton_reorder(self):
        """a1: permute params, m and v (3 x P planes) into Morton order."""
        src = self.state[self.cur].view(3 * self.np_, self.stride)
        dst = self.state[self.cur ^ 1].view(3 * self.np_, self.stride)
        B.lgs_morton_reorder(src, dst, self.n, 3 * self.np_, self.codes, self.perm, self.ws_morton)
        self.cur ^= 1
        self._round_sh16()

    def render(self, cam: dict, camst: B.LgsCamera | None = None):
        """a2..a5 for one camera: cull, preprocess, bin, forward."""
        cs = camst or B.camera_struct(cam)
        tw, th = self.cfg.tile
        g = self.gaussians()
        if self.cfg.ccc:
            B.lgs_cluster_cull_compact(g, cs, self.cfg.cluster, None, self.cluster_visible,
                                       self.rowmap, self.d_V, self.ws_ccc)
        B.lgs_preprocess(g, self._map(), self._dV(), cs, tw, th, self.splats)
        B.lgs_bin_sort(self.splats, self._dV(), self.n, cs, tw, th, self.vals, self.d_P,
                       self.ranges, self.ws_bin)
        B.lgs_raster_fwd(self.splats, self.vals, self.ranges, cs, tw, th, self.image, self.finalT,
                         self.last, precision=self.cfg.precision)
        return cs

    def backward(self, cs: B.LgsCamera, target: torch.Tensor, accumulate=False, metric=True):
        """a6..a8: loss gradient, backward rasterisation, variance metric
        (metric=False leaves a8 to the fused optimizer, which writes the
        same values from the gradient rows it reads)."""
        tw, th = self.cfg.tile
        B.lgs_loss_l1(self.image, target, self.dLdI, self.loss)
        B.lgs_raster_bwd(self.splats, self.vals, self.ranges, cs, tw, th, self.finalT, self.last,
                         self.dLdI, self.gacc, accumulate=accumulate,
                         precision=self.cfg.precision)
        if metric:
            B.lgs_opacity_variance(self.gacc, self._map(), self._dV(), self.n, self.metric)
        if self.track_moments:
            B.lgs_moments_accumulate(self.gacc, self._map(), self._dV(), self.n, self.S_acc,
                                     self.M_acc, self.C_acc)

    # -- densification (Sec. 3.3) --------------------------------------------
    def densify(self, max_new: int, split_scale: float, seed: int = 0) -> int:
        """Clone / split the Gaussians with the largest opacity-gradient
        variance summed over the views since the last call, then Morton
        re-sort (Sec. 3.2.1). Returns the number of Gaussians added."""
        max_new = min(int(max_new), self.capacity - self.n)
        g = self._g32()
        B.lgs_moments_metric(self.S_acc, self.M_acc, self.C_acc, self.n, self.metric)
        gen = torch.Generator(device=self.dev).manual_seed(seed)
        normals = torch.randn((max(max_new, 1), 2, 3), generator=gen, device=self.dev)
        d_n = torch.zeros(1, dtype=torch.int64, device=self.dev)
        ws = torch.empty(B.lgs_densify_workspace_size(self.n), dtype=torch.uint8, device=self.dev)
        B.lgs_densify(g, self.m, self.v, self.metric, max_new, split_scale, normals, d_n, None, ws)
        new_n = int(d_n.item())
        added = new_n - self.n
        self.n = new_n
        for t in (self.S_acc, self.M_acc, self.C_acc):
            t.zero_()
        self.morton_reorder()
        return added

    def opacity_decay(self):
        """Halves every activated opacity (Sec. 3.3)."""
        B.lgs_opacity_decay(self._g32())

    def optimize(self, cs: B.LgsCamera, fused=True, metric=False):
        """a9 + a10: preprocess backward and Adam on the visible rows
        (fused, metric=True: also the a8 metric, in the same launch)."""
        self.step_count += 1
        c = self.cfg
        g = self.gaussians()
        if fused:
            B.lgs_preprocess_bwd_adam(g, self.m, self.v, self._map(), self._dV(), cs, self.gacc,
                                      self.lr, c.beta1, c.beta2, c.eps, self.step_count,
                                      splats=self.splats, metric=self.metric if metric else None)
        else:
            if self.sh16 is not None:
                raise ValueError("a 16-bit colour copy is kept up to date by the fused optimizer only")
            if self.grad_planes is None:
                self.grad_planes = torch.zeros((self.np_, self.stride), dtype=torch.float32,
                                               device=self.dev)
            B.lgs_preprocess_bwd(g, self._map(), self._dV(), cs, self.gacc, self.grad_planes)
            B.lgs_adam_step(self.params, self.grad_planes, self.m, self.v, self.np_, self.lr,
                            c.beta1, c.beta2, c.eps, self.step_count, self._map(), self._dV(),
                            self.n)

    # -- checkpoint / resume -------------------------------------------------
    def save(self, path) -> None:
        """Write the scene state as raw arrays (numpy .npz): the parameter
        planes and both Adam moments of the live rows (current storage order),
        the SH degree and the step count, so that a resumed run continues the
        same Adam schedule."""
        n = self.n
        np.savez(path, params=self.params[:, :n].cpu().numpy(), m=self.m[:, :n].cpu().numpy(),
                 v=self.v[:, :n].cpu().numpy(), sh_degree=np.int64(self.sh_degree),
                 step_count=np.int64(self.step_count))

    def load(self, path) -> None:
        """Read a checkpoint written by save() into this trainer (its
        capacity must hold the saved rows; the camera size and buffers are
        this trainer's own)."""
        with np.load(path) as z:
            if int(z["sh_degree"]) != self.sh_degree:
                raise ValueError("checkpoint has another SH degree")
            n = int(z["params"].shape[1])
            if n > self.capacity:
                raise ValueError("checkpoint has more rows than this trainer's capacity")
            st = self.state[self.cur]
            st.zero_()
            for k, name in enumerate(("params", "m", "v")):
                st[k, :, :n].copy_(torch.from_numpy(np.ascontiguousarray(z[name])).to(self.dev))
            self.n = n
            self.step_count = int(z["step_count"])
        self._round_sh16()

    def check_overflow(self) -> None:
        """Raises LgsError if a binning since the last check needed more
        (tile, splat) pairs than the pair capacity: its tile lists were cut
        at the capacity, so images and gradients of those steps were wrong.
        Reads the library's overflow flag, which synchronises the device and
        clears the flag (it is shared by every caller in the process)."""
        needed = B.lgs_get_overflow()
        if needed:
            raise B.LgsError(f"tile binning needed {needed} pairs but pair_capacity is {self.cap}; "
                             "raise StepConfig.pair_capacity")

    def step(self, cam: dict | B.LgsCamera, target: torch.Tensor, reorder: bool = True,
             fused: bool = True):
        """One full training step a1..a10 (and, every
        cfg.overflow_check_every steps outside graph capture, the overflow
        check of check_overflow())."""
        if reorder:
            self.morton_reorder()
        cs = cam if isinstance(cam, B.LgsCamera) else B.camera_struct(cam)
        self.render(None, cs)
        self.backward(cs, target, metric=not fused)
        self.optimize(cs, fused=fused, metric=fused)
        every = self.cfg.overflow_check_every
        if every and self.step_count % every == 0 and not torch.cuda.is_current_stream_capturing():
            self.check_overflow()
        return self.loss


class MultiView:
    """Forward + backward of one scene for several cameras at once.

    Per view: cluster cull + compaction, preprocess and binning (each view
    keeps its own map, splats and tile lists); then ONE batched raster
    forward over the tiles of all views, the L1 loss gradient of each view,
    ONE batched raster backward, and per view the preprocess backward adding
    into one gradient buffer (the parameters' gradient summed over views).
    `capture()` records the whole sequence as one CUDA graph; `run_sequential`
    is the same work with one plain launch sequence per view.

    The views' front ends are independent of one another, so run_batched
    spreads them over `streams` side streams (view k on slot k % streams,
    each slot with its own cull and binning workspaces), forked from and
    joined back into the calling stream; the small views' latency-bound
    launches then overlap. Each look-back kernel waits only on CTAs of its
    own launch, so launches running side by side never wait on each other.
    """

    def __init__(self, planes: torch.Tensor, n: int, sh_degree: int, cams: list, targets: list,
                 pair_capacity: int, tile=(16, 16), cluster: int = 128, device="cuda",
                 streams: int = 4):
        self.planes, self.n, self.deg = planes, int(n), int(sh_degree)
        self.cams = cams
        self.tile, self.cluster = tuple(tile), int(cluster)
        self.cap = int(pair_capacity)
        dev = self.dev = torch.device(device)
        tw, th = self.tile
        self.g = B.gaussians_struct(planes, n, sh_degree)
        self.cs = [B.camera_struct(c) for c in cams]
        nt = [-(-c["width"] // tw) * -(-c["height"] // th) for c in cams]
        self.n_slots = max(1, min(int(streams), len(cams)))
        self.slots = [{"ws_ccc": torch.empty(B.lgs_ccc_workspace_size(n, cluster),
                                             dtype=torch.uint8, device=dev),
                       "ws_bin": torch.empty(B.lgs_bin_sort_workspace_size(n, self.cap, max(nt)),
                                             dtype=torch.uint8, device=dev),
                       "cluster_visible": torch.empty(-(-n // cluster), dtype=torch.int32,
                                                      device=dev),
                       "stream": torch.cuda.Stream(device=dev)}
                      for _ in range(self.n_slots)]
        self.gacc = torch.zeros((len(cams), n, B.GRAD_FLOATS), dtype=torch.float32, device=dev)
        self.grad = torch.zeros_like(planes)
        self.counter = torch.zeros(1, dtype=torch.int32, device=dev)
        self.views = []
        for k, (c, tgt) in enumerate(zip(cams, targets)):
            W, H = int(c["width"]), int(c["height"])
            v = {"camera": c,
                 "rowmap": torch.empty(n, dtype=torch.int32, device=dev),
                 "d_V": torch.zeros(1, dtype=torch.int32, device=dev),
                 "rec": torch.empty((n, B.SPLAT_FLOATS), dtype=torch.float32, device=dev),
                 "depth": torch.empty(n, dtype=torch.float32, device=dev),
                 "radius": torch.empty(n, dtype=torch.int32, device=dev),
                 "vals": torch.empty(self.cap, dtype=torch.int32, device=dev),
                 "d_P": torch.zeros(1, dtype=torch.int64, device=dev),
                 "ranges": torch.empty((nt[k], 2), dtype=torch.int32, device=dev),
                 "image": torch.empty((3, H, W), dtype=torch.float32, device=dev),
                 "final_T": torch.empty((H, W), dtype=torch.float32, device=dev),
                 "last": torch.empty((H, W), dtype=torch.int32, device=dev),
                 "dL_dimage": torch.empty((3, H, W), dtype=torch.float32, device=dev),
                 "loss": torch.zeros(1, dtype=torch.float32, device=dev),
                 "target": tgt, "grad_acc": self.gacc[k]}
            v["splats"] = B.splats_struct(v["rec"], v["depth"], v["radius"])
            self.views.append(v)
        self.table, self.total_tiles = B.view_table(self.views, self.tile, device=dev)
        self.graph = None

    def _front(self, k: int, slot: int = 0):
        v, cs, sl = self.views[k], self.cs[k], self.slots[slot]
        tw, th = self.tile
        B.lgs_cluster_cull_compact(self.g, cs, self.cluster, None, sl["cluster_visible"],
                                   v["rowmap"], v["d_V"], sl["ws_ccc"])
        B.lgs_preprocess(self.g, v["rowmap"], v["d_V"], cs, tw, th, v["splats"])
        B.lgs_bin_sort(v["splats"], v["d_V"], self.n, cs, tw, th, v["vals"], v["d_P"],
                       v["ranges"], sl["ws_bin"])

    def _fronts_concurrent(self):
        main = torch.cuda.current_stream(self.dev)
        fork = torch.cuda.Event()
        fork.record(main)
        for sl in self.slots:
            sl["stream"].wait_event(fork)
        for k in range(len(self.views)):
            slot = k % self.n_slots
            with torch.cuda.stream(self.slots[slot]["stream"]):
                self._front(k, slot)
        for sl in self.slots:
            done = torch.cuda.Event()
            done.record(sl["stream"])
            main.wait_event(done)

    def run_batched(self, precision=B.LGS_FP32):
        self._fronts_concurrent()
        B.lgs_raster_fwd_batch(self.table, len(self.views), self.total_tiles, self.counter,
                               precision=precision)
        for v in self.views:
            B.lgs_loss_l1(v["image"], v["target"], v["dL_dimage"], v["loss"])
        self.gacc.zero_()
        B.lgs_raster_bwd_batch(self.table, len(self.views), self.total_tiles, self.counter,
                               precision=precision)
        for k, v in enumerate(self.views):
            B.lgs_preprocess_bwd(self.g, v["rowmap"], v["d_V"], self.cs[k], v["grad_acc"],
                                 self.grad, accumulate=k > 0)

    def run_sequential(self, precision=B.LGS_FP32):
        tw, th = self.tile
        for k, v in enumerate(self.views):
            cs = self.cs[k]
            self._front(k)
            B.lgs_raster_fwd(v["splats"], v["vals"], v["ranges"], cs, tw, th, v["image"],
                             v["final_T"], v["last"], precision=precision)
            B.lgs_loss_l1(v["image"], v["target"], v["dL_dimage"], v["loss"])
            B.lgs_raster_bwd(v["splats"], v["vals"], v["ranges"], cs, tw, th, v["final_T"],
                             v["last"], v["dL_dimage"], v["grad_acc"], precision=precision)
            B.lgs_preprocess_bwd(self.g, v["rowmap"], v["d_V"], cs, v["grad_acc"], self.grad,
                                 accumulate=k > 0)

    def capture(self, precision=B.LGS_FP32):
        """Records run_batched as one CUDA graph (after one eager run)."""
        side = torch.cuda.Stream(device=self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            self.run_batched(precision)
        side.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            self.run_batched(precision)
        torch.cuda.current_stream(self.dev).wait_stream(side)
        return self.graph

    def replay(self):
        self.graph.replay()
