"""The rasterizer as a torch.autograd.Function (Eq. 1-3, App. A.1).

    image = rasterize(planes, camera, rasterizer)

`planes` is the float32 parameter tensor [num_planes(deg)][stride] in the
library's plane order (centre xyz, log-scales, quaternion wxyz, opacity
logit, SH coefficient-major with RGB innermost); its gradient comes back in
the same layout. The forward runs a2..a5 (cluster cull + compaction,
preprocess, binning, forward raster); the hand-written backward runs a7 and
a9 (backward raster + preprocess backward). Per pixel, the forward keeps only
the final transmittance and the index of the last included splat: the
backward walks each tile's list from that splat to the front and recovers
every earlier transmittance by dividing out (1 - alpha), so nothing per
fragment is stored between the two passes.

Every call returns fresh output and saved buffers from torch's caching
allocator, so several forwards may be pending before their backwards run.
The backward reads the forward's pair count (one host synchronisation) and
raises LgsError if the binning needed more pairs than `pair_capacity`.
The optional `metric` tensor [n] receives the densification statistic
C Var = S - M^2/C (Sec. 3.3) of the visible Gaussians when backward runs;
rows of culled clusters are left as they are.

Everything on the path runs in liblgs kernels; torch supplies memory, the
stream and the autograd graph.
"""
from __future__ import annotations

import torch

from . import binding as B

PRECISIONS = {"fp32": B.LGS_FP32, "fp16": B.LGS_MIXED_FP16, "bf16": B.LGS_MIXED_BF16}


class GaussianRasterizer:
    """Settings and reusable scratch for rendering scenes of up to `n`
    Gaussians on cameras of up to `max_width` x `max_height`.

    precision: "fp32" (plain), or "fp16" / "bf16" for the mixed-precision
    raster (per-pixel blend intermediates in 16 bits; transmittance, colour
    accumulators, gradient sums and the conic in FP32).
    """

    def __init__(self, n: int, sh_degree: int, max_width: int, max_height: int,
                 tile=(16, 16), cluster: int = 128, pair_capacity: int | None = None,
                 precision: str = "fp32", device="cuda"):
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.tile = tuple(tile)
        self.cluster = int(cluster)
        self.precision = precision
        self.dev = torch.device(device)
        tw, th = self.tile
        self.max_tiles = -(-int(max_width) // tw) * -(-int(max_height) // th)
        self.cap = int(pair_capacity or max(64 * self.n, 1 << 20))
        self.ws_ccc = torch.empty(B.lgs_ccc_workspace_size(self.n, self.cluster), dtype=torch.uint8,
                                  device=self.dev)
        self.ws_bin = torch.empty(B.lgs_bin_sort_workspace_size(self.n, self.cap, self.max_tiles),
                                  dtype=torch.uint8, device=self.dev)
        self.cluster_visible = torch.empty(-(-self.n // self.cluster), dtype=torch.int32,
                                           device=self.dev)

    def __call__(self, planes: torch.Tensor, camera, metric: torch.Tensor | None = None):
        return rasterize(planes, camera, self, metric)


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, planes, r: GaussianRasterizer, cs: B.LgsCamera, metric):
        n, dev = r.n, r.dev
        tw, th = r.tile
        W, H = cs.width, cs.height
        if -(-W // tw) * -(-H // th) > r.max_tiles:
            raise B.LgsError("camera larger than the rasterizer was sized for")
        g = B.gaussians_struct(planes, n, r.sh_degree)
        rowmap = torch.empty(n, dtype=torch.int32, device=dev)
        d_V = torch.empty(1, dtype=torch.int32, device=dev)
        rec = torch.empty((n, B.SPLAT_FLOATS), dtype=torch.float32, device=dev)
        depth = torch.empty(n, dtype=torch.float32, device=dev)
        radius = torch.empty(n, dtype=torch.int32, device=dev)
        vals = torch.empty(r.cap, dtype=torch.int32, device=dev)
        d_P = torch.empty(1, dtype=torch.int64, device=dev)
        ranges = torch.empty((-(-W // tw) * -(-H // th), 2), dtype=torch.int32, device=dev)
        image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        final_T = torch.empty((H, W), dtype=torch.float32, device=dev)
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
        sp = B.splats_struct(rec, depth, radius)
        B.lgs_cluster_cull_compact(g, cs, r.cluster, None, r.cluster_visible, rowmap, d_V, r.ws_ccc)
        B.lgs_preprocess(g, rowmap, d_V, cs, tw, th, sp)
        B.lgs_bin_sort(sp, d_V, n, cs, tw, th, vals, d_P, ranges, r.ws_bin)
        B.lgs_raster_fwd(sp, vals, ranges, cs, tw, th, image, final_T, last,
                         precision=PRECISIONS[r.precision])
        ctx.r, ctx.cs, ctx.metric = r, cs, metric
        ctx.save_for_backward(planes, rowmap, d_V, rec, depth, radius, vals, ranges, final_T, last,
                              d_P)
        ctx.mark_non_differentiable(final_T)
        return image

    @staticmethod
    def backward(ctx, dL_dimage):
        planes, rowmap, d_V, rec, depth, radius, vals, ranges, final_T, last, d_P = ctx.saved_tensors
        r, cs = ctx.r, ctx.cs
        # the binning writes at most r.cap pairs; more means the forward's
        # tile lists were cut and neither its image nor these gradients hold
        # (one host read of the pair count per backward)
        P = int(d_P.item())
        if P > r.cap:
            raise B.LgsError(f"tile binning needed {P} pairs but pair_capacity is {r.cap}; "
                             "construct GaussianRasterizer with a larger pair_capacity")
        tw, th = r.tile
        sp = B.splats_struct(rec, depth, radius)
        gacc = torch.empty((r.n, B.GRAD_FLOATS), dtype=torch.float32, device=r.dev)
        B.lgs_raster_bwd(sp, vals, ranges, cs, tw, th, final_T, last,
                         dL_dimage.to(torch.float32).contiguous(), gacc, accumulate=False,
                         precision=PRECISIONS[r.precision])
        grad = torch.zeros_like(planes)
        g = B.gaussians_struct(planes, r.n, r.sh_degree)
        B.lgs_preprocess_bwd(g, rowmap, d_V, cs, gacc, grad)
        if ctx.metric is not None:
            B.lgs_opacity_variance(gacc, rowmap, d_V, r.n, ctx.metric)
        return grad, None, None, None


def rasterize(planes: torch.Tensor, camera, r: GaussianRasterizer,
              metric: torch.Tensor | None = None) -> torch.Tensor:
    """Render `planes` (float32 [num_planes][stride], CUDA, contiguous) from
    `camera` (a scenegen camera dict or an LgsCamera); returns the image
    [3][H][W]. Differentiable with respect to `planes`."""
    if planes.dtype != torch.float32 or not planes.is_cuda or not planes.is_contiguous():
        raise B.LgsError("planes must be a contiguous float32 CUDA tensor")
    if planes.shape[0] < B.num_planes(r.sh_degree) or planes.shape[1] < r.n:
        raise B.LgsError("planes tensor smaller than [num_planes(deg)][n]")
    cs = camera if isinstance(camera, B.LgsCamera) else B.camera_struct(camera)
    return _Rasterize.apply(planes, r, cs, metric)
