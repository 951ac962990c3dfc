"""Thin Python binding of liblgs (include/lgs.h): the same entry points,
taking torch CUDA tensors and marshalling them to pointers, sizes and the
current CUDA stream. Every step runs in the library's kernels; nothing here
computes. There is no fallback: if the library cannot be loaded or CUDA is
not available, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np
import torch

from . import build as _build

LGS_OK, LGS_ERR_INVALID_ARG, LGS_ERR_CAPACITY, LGS_ERR_CUDA, LGS_ERR_TIMEOUT = 0, 1, 2, 3, 4
LGS_ERR_TOO_LARGE = 5
LGS_ERR_BOUNDS = 6
LGS_FP32, LGS_MIXED_FP16, LGS_MIXED_BF16 = 0, 1, 2
LGS_WARP_REDUCE_INT = 16
LGS_SH_F32, LGS_SH_BF16, LGS_SH_F16 = 0, 1, 2
NOALLOC_MAX_CLUSTERS = 65536
SPLAT_FLOATS = 12
GRAD_FLOATS = 16
MAX_PLANES = 59

ENTRY_POINTS = (
    "lgs_version", "lgs_last_cuda_error", "lgs_kernel_launches", "lgs_morton_workspace_size", "lgs_morton_reorder",
    "lgs_ccc_workspace_size", "lgs_cluster_cull_compact", "lgs_cluster_cull_compact_noalloc",
    "lgs_compact_gather", "lgs_preprocess",
    "lgs_bin_sort_workspace_size", "lgs_bin_sort", "lgs_bin_keys", "lgs_get_overflow", "lgs_get_wait_timeouts", "lgs_set_wait_limit",
    "lgs_debug_build", "lgs_get_debug_error",
    "lgs_raster_fwd",
    "lgs_raster_fwd_batch", "lgs_raster_bwd_batch", "lgs_loss_l1", "lgs_raster_bwd",
    "lgs_raster_bwd_det_workspace_size", "lgs_raster_bwd_deterministic", "lgs_get_det_overflow",
    "lgs_opacity_variance", "lgs_preprocess_bwd",
    "lgs_adam_step", "lgs_preprocess_bwd_adam", "lgs_round_planes", "lgs_moments_accumulate", "lgs_moments_metric",
    "lgs_densify_workspace_size", "lgs_densify", "lgs_opacity_decay",
    "lgs_peak_ex2", "lgs_peak_ffma", "lgs_peak_red",
)


def num_planes(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


class LgsCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("znear", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("d_pose", ctypes.c_void_p)]


class LgsGaussians(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("sh_degree", ctypes.c_int32), ("sh_dtype", ctypes.c_int32),
                ("sh16", ctypes.c_void_p)]


class LgsSplats(ctypes.Structure):
    _fields_ = [("rec", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("capacity", ctypes.c_int64)]


class LgsView(ctypes.Structure):
    _fields_ = [("rec", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("tile_ranges", ctypes.c_void_p), ("image", ctypes.c_void_p),
                ("final_T", ctypes.c_void_p), ("last_contrib", ctypes.c_void_p),
                ("dL_dimage", ctypes.c_void_p), ("grad_acc", ctypes.c_void_p),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_offset", ctypes.c_uint32), ("bg", ctypes.c_float * 3)]


class LgsError(RuntimeError):
    pass


_lib = None


def library_path() -> Path:
    """The release library, or the bounds-checked debug build when the
    environment sets LGS_DEBUG=1 (read when the library is first loaded)."""
    return _build.DEBUG_LIB if os.environ.get("LGS_DEBUG") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Load liblgs.so (building it if needed). Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = library_path()
    if not path.exists():
        raise LgsError(f"liblgs.so not found at {path}; run paper_2503_01199_gb300/build.py")
    L = ctypes.CDLL(str(path))
    P, i32, i64, f32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    u32 = ctypes.c_uint32
    sig = {
        "lgs_version": (ctypes.c_char_p, []),
        "lgs_last_cuda_error": (i32, []),
        "lgs_kernel_launches": (ctypes.c_uint64, []),
        "lgs_morton_workspace_size": (sz, [i64]),
        "lgs_morton_reorder": (i32, [P, P, i64, i64, i32, P, P, P, sz, P]),
        "lgs_ccc_workspace_size": (sz, [i64, i32]),
        "lgs_cluster_cull_compact": (i32, [P, P, i32, P, P, P, P, P, sz, P]),
        "lgs_cluster_cull_compact_noalloc": (i32, [P, P, i32, P, P, P, P, P]),
        "lgs_compact_gather": (i32, [P, i64, P, i64, i32, P, P, i64, P]),
        "lgs_preprocess": (i32, [P, P, P, P, i32, i32, P, P]),
        "lgs_bin_sort_workspace_size": (sz, [i64, i64, i32]),
        "lgs_bin_sort": (i32, [P, P, i64, P, i32, i32, i32, P, i64, P, P, P, sz, P]),
        "lgs_get_overflow": (i32, [P]),
        "lgs_get_wait_timeouts": (i32, [P]),
        "lgs_set_wait_limit": (i32, [u32]),
        "lgs_debug_build": (i32, []),
        "lgs_get_debug_error": (i32, [P]),
        "lgs_raster_fwd": (i32, [P, P, P, P, i32, i32, i32, P, P, P, P]),
        "lgs_loss_l1": (i32, [P, P, i64, P, P, P]),
        "lgs_raster_bwd": (i32, [P, P, P, P, i32, i32, i32, P, P, P, P, i64, i32, P]),
        "lgs_raster_bwd_det_workspace_size": (sz, [i64]),
        "lgs_raster_bwd_deterministic": (i32, [P, P, P, P, i32, i32, i32, P, P, P, P, i64, P, sz,
                                                P]),
        "lgs_get_det_overflow": (i32, [P]),
        "lgs_opacity_variance": (i32, [P, P, P, i64, P, P]),
        "lgs_preprocess_bwd": (i32, [P, P, P, P, P, P, i32, P]),
        "lgs_raster_fwd_batch": (i32, [P, i32, u32, i32, P, P]),
        "lgs_raster_bwd_batch": (i32, [P, i32, u32, i32, P, P]),
        "lgs_adam_step": (i32, [P, P, P, P, i64, i32, P, f32, f32, f32, i32, P, P, i64, P]),
        "lgs_preprocess_bwd_adam": (i32, [P, P, P, P, P, P, P, P, P, f32, f32, f32, i32, P, P]),
        "lgs_moments_accumulate": (i32, [P, P, P, i64, P, P, P, P]),
        "lgs_round_planes": (i32, [P, i64, P, i64, i32, i64, i32, P]),
        "lgs_moments_metric": (i32, [P, P, P, i64, P, P]),
        "lgs_densify_workspace_size": (sz, [i64]),
        "lgs_densify": (i32, [P, P, P, P, i64, f32, P, P, P, P, sz, P]),
        "lgs_opacity_decay": (i32, [P, P]),
        "lgs_bin_keys": (i32, [P, P, P, i32, P, P]),
        "lgs_peak_ex2": (i32, [P, i32, i32, P]),
        "lgs_peak_ffma": (i32, [P, i32, i32, i32, P]),
        "lgs_peak_red": (i32, [P, i64, i32, i32, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, what: str):
    if status != LGS_OK:
        err = _lib.lgs_last_cuda_error() if _lib is not None else 0
        names = {1: "LGS_ERR_INVALID_ARG", 2: "LGS_ERR_CAPACITY", 3: "LGS_ERR_CUDA", 4: "LGS_ERR_TIMEOUT",
                 5: "LGS_ERR_TOO_LARGE"}
        raise LgsError(f"{what} failed: {names.get(status, status)} (cuda error {err})")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.numel() and not t.is_cuda:
        raise LgsError("liblgs takes CUDA tensors only")
    if not t.is_contiguous():
        raise LgsError("liblgs takes contiguous tensors only")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# --------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------
def camera_struct(cam: dict, d_pose=None) -> LgsCamera:
    """Host camera descriptor; d_pose (optional float32 CUDA tensor of 12:
    R row-major, t) makes the cull and preprocess read the pose from device
    memory when they run."""
    c = LgsCamera()
    R = [float(x) for x in np.asarray(cam["R"]).reshape(9)]
    t = [float(x) for x in np.asarray(cam["t"]).reshape(3)]
    bg = [float(x) for x in np.asarray(cam["bg"]).reshape(3)]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.znear = float(cam["znear"])
    c.bg[:] = bg
    c.d_pose = _ptr(d_pose)
    return c


def gaussians_struct(planes: torch.Tensor, n: int, sh_degree: int,
                     sh16: torch.Tensor | None = None) -> LgsGaussians:
    """planes: float32 CUDA tensor [>= num_planes, stride] (or [>= 11, stride]
    with sh16 given); sh16: optional bfloat16 / float16 CUDA tensor
    [3 (deg+1)^2, stride] holding the colour coefficients instead."""
    g = LgsGaussians()
    g.data = _ptr(planes)
    g.n = int(n)
    g.stride = int(planes.shape[-1])
    g.sh_degree = int(sh_degree)
    g.sh_dtype = LGS_SH_F32
    if sh16 is not None:
        if sh16.shape[-1] != planes.shape[-1]:
            raise LgsError("sh16 must have the planes' stride")
        g.sh_dtype = {torch.bfloat16: LGS_SH_BF16, torch.float16: LGS_SH_F16}[sh16.dtype]
        g.sh16 = _ptr(sh16)
    return g


def splats_struct(rec: torch.Tensor, depth: torch.Tensor, radius: torch.Tensor) -> LgsSplats:
    s = LgsSplats()
    s.rec, s.depth, s.radius = _ptr(rec), _ptr(depth), _ptr(radius)
    s.capacity = int(depth.shape[0])
    return s


# --------------------------------------------------------------------------
# entry points
# --------------------------------------------------------------------------
def lgs_version() -> str:
    return load().lgs_version().decode()


def lgs_kernel_launches() -> int:
    return int(load().lgs_kernel_launches())


def lgs_morton_workspace_size(n: int) -> int:
    return int(load().lgs_morton_workspace_size(n))


def lgs_morton_reorder(src, dst, n, n_planes, codes_out, perm_out, workspace, stream=None):
    L = load()
    _check(L.lgs_morton_reorder(_ptr(src), _ptr(dst), n, src.shape[-1], n_planes, _ptr(codes_out),
                                _ptr(perm_out), _ptr(workspace), workspace.numel(),
                                _stream(stream)), "lgs_morton_reorder")


def lgs_ccc_workspace_size(n: int, cluster_size: int) -> int:
    return int(load().lgs_ccc_workspace_size(n, cluster_size))


def lgs_cluster_cull_compact(g: LgsGaussians, cam: LgsCamera, cluster_size, aabb_out,
                             cluster_visible_out, map_out, d_num_visible, workspace, stream=None):
    L = load()
    _check(L.lgs_cluster_cull_compact(ctypes.byref(g), ctypes.byref(cam), cluster_size,
                                      _ptr(aabb_out), _ptr(cluster_visible_out), _ptr(map_out),
                                      _ptr(d_num_visible), _ptr(workspace), workspace.numel(),
                                      _stream(stream)), "lgs_cluster_cull_compact")


def lgs_cluster_cull_compact_noalloc(g: LgsGaussians, cam: LgsCamera, cluster_size, aabb_out,
                                     cluster_visible_out, map_out, d_num_visible, stream=None):
    """Same as lgs_cluster_cull_compact, with no workspace: for callers that
    cannot allocate device memory. Uses a fixed scratch array inside the
    library (see include/lgs.h for its limit and sharing rules)."""
    L = load()
    _check(L.lgs_cluster_cull_compact_noalloc(ctypes.byref(g), ctypes.byref(cam), cluster_size,
                                              _ptr(aabb_out), _ptr(cluster_visible_out),
                                              _ptr(map_out), _ptr(d_num_visible),
                                              _stream(stream)),
           "lgs_cluster_cull_compact_noalloc")


def lgs_compact_gather(src, dst, n_planes, map_, d_num_visible, max_rows, stream=None):
    L = load()
    _check(L.lgs_compact_gather(_ptr(src), src.shape[-1], _ptr(dst), dst.shape[-1], n_planes,
                                _ptr(map_), _ptr(d_num_visible), max_rows, _stream(stream)),
           "lgs_compact_gather")


def lgs_preprocess(g: LgsGaussians, map_, d_num_visible, cam: LgsCamera, tile_w, tile_h,
                   out: LgsSplats, stream=None):
    L = load()
    _check(L.lgs_preprocess(ctypes.byref(g), _ptr(map_), _ptr(d_num_visible), ctypes.byref(cam),
                            tile_w, tile_h, ctypes.byref(out), _stream(stream)), "lgs_preprocess")


def lgs_bin_sort_workspace_size(max_splats: int, pair_capacity: int, n_tiles: int) -> int:
    return int(load().lgs_bin_sort_workspace_size(max_splats, pair_capacity, n_tiles))


def lgs_bin_sort(sp: LgsSplats, d_num_visible, max_splats, cam: LgsCamera, tile_w, tile_h, vals,
                 d_num_pairs, tile_ranges, workspace, stream=None, tile_cull=1):
    L = load()
    _check(L.lgs_bin_sort(ctypes.byref(sp), _ptr(d_num_visible), max_splats, ctypes.byref(cam),
                          tile_w, tile_h, int(tile_cull), _ptr(vals), vals.numel(), _ptr(d_num_pairs),
                          _ptr(tile_ranges), _ptr(workspace), workspace.numel(), _stream(stream)),
           "lgs_bin_sort")


def lgs_get_overflow() -> int:
    """Returns the pair count needed by an overflowed lgs_bin_sort (0 if none)."""
    L = load()
    needed = ctypes.c_int64(0)
    st = L.lgs_get_overflow(ctypes.byref(needed))
    if st not in (LGS_OK, LGS_ERR_CAPACITY):
        _check(st, "lgs_get_overflow")
    return int(needed.value)


def lgs_get_wait_timeouts() -> int:
    """Bounded device waits that gave up since the last query (0 if none)."""
    L = load()
    count = ctypes.c_uint32(0)
    st = L.lgs_get_wait_timeouts(ctypes.byref(count))
    if st not in (LGS_OK, LGS_ERR_TIMEOUT):
        _check(st, "lgs_get_wait_timeouts")
    return int(count.value)


def lgs_get_debug_error() -> int:
    """(site << 32) | line of the first failed bounds check of the debug
    build since the last query (0: none; always 0 in the release build)."""
    L = load()
    code = ctypes.c_uint64(0)
    st = L.lgs_get_debug_error(ctypes.byref(code))
    if st not in (LGS_OK, LGS_ERR_BOUNDS):
        _check(st, "lgs_get_debug_error")
    return int(code.value)


LGS_DEFAULT_WAIT_LIMIT = 4194304


def lgs_set_wait_limit(spins: int) -> None:
    """Polls after which a bounded device wait gives up (testing the give-up path)."""
    _check(load().lgs_set_wait_limit(int(spins)), "lgs_set_wait_limit")


def lgs_raster_fwd(sp: LgsSplats, vals, tile_ranges, cam: LgsCamera, tile_w, tile_h, image,
                   final_T, last_contrib, stream=None, precision=LGS_FP32):
    L = load()
    _check(L.lgs_raster_fwd(ctypes.byref(sp), _ptr(vals), _ptr(tile_ranges), ctypes.byref(cam),
                            tile_w, tile_h, int(precision), _ptr(image), _ptr(final_T),
                            _ptr(last_contrib), _stream(stream)), "lgs_raster_fwd")


def view_table(views: list, tile=(16, 16), device="cuda") -> tuple[torch.Tensor, int]:
    """Device table of lgs_view for the batched raster calls.
    views: dicts with rec, vals, ranges, image, final_T, last (tensors), and
    optionally dL_dimage, grad_acc, plus the camera dict 'camera' (width,
    height, bg). Returns (uint8 CUDA tensor holding the table, total tiles)."""
    raw, off = view_table_bytes(views, tile)
    table = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
    return table, off


def view_table_bytes(views: list, tile=(16, 16)) -> tuple[bytes, int]:
    """The bytes of an lgs_view table (see view_table) and the total tiles."""
    arr = (LgsView * len(views))()
    off = 0
    for i, v in enumerate(views):
        cam = v["camera"]
        w, h = int(cam["width"]), int(cam["height"])
        e = arr[i]
        e.rec, e.vals, e.tile_ranges = _ptr(v["rec"]), _ptr(v["vals"]), _ptr(v["ranges"])
        e.image, e.final_T, e.last_contrib = _ptr(v["image"]), _ptr(v["final_T"]), _ptr(v["last"])
        e.dL_dimage, e.grad_acc = _ptr(v.get("dL_dimage")), _ptr(v.get("grad_acc"))
        e.width, e.height, e.tile_offset = w, h, off
        e.bg[:] = [float(x) for x in np.asarray(cam["bg"]).reshape(3)]
        off += -(-w // tile[0]) * -(-h // tile[1])
    return bytes(arr), off


def lgs_raster_fwd_batch(table, n_views, total_tiles, counter, precision=LGS_FP32, stream=None):
    L = load()
    _check(L.lgs_raster_fwd_batch(_ptr(table), int(n_views), int(total_tiles), int(precision),
                                  _ptr(counter), _stream(stream)), "lgs_raster_fwd_batch")


def lgs_raster_bwd_batch(table, n_views, total_tiles, counter, precision=LGS_FP32, stream=None):
    L = load()
    _check(L.lgs_raster_bwd_batch(_ptr(table), int(n_views), int(total_tiles), int(precision),
                                  _ptr(counter), _stream(stream)), "lgs_raster_bwd_batch")


def lgs_loss_l1(image, target, dL_dimage, d_loss, stream=None):
    L = load()
    _check(L.lgs_loss_l1(_ptr(image), _ptr(target), image.numel(), _ptr(dL_dimage), _ptr(d_loss),
                         _stream(stream)), "lgs_loss_l1")


def lgs_raster_bwd(sp: LgsSplats, vals, tile_ranges, cam: LgsCamera, tile_w, tile_h, final_T,
                   last_contrib, dL_dimage, grad_acc, accumulate=False, stream=None,
                   precision=LGS_FP32):
    L = load()
    _check(L.lgs_raster_bwd(ctypes.byref(sp), _ptr(vals), _ptr(tile_ranges), ctypes.byref(cam),
                            tile_w, tile_h, int(precision), _ptr(final_T), _ptr(last_contrib),
                            _ptr(dL_dimage), _ptr(grad_acc), grad_acc.shape[0],
                            int(bool(accumulate)), _stream(stream)), "lgs_raster_bwd")


def lgs_raster_bwd_det_workspace_size(max_splats: int) -> int:
    return int(load().lgs_raster_bwd_det_workspace_size(int(max_splats)))


def lgs_raster_bwd_deterministic(sp: LgsSplats, vals, tile_ranges, cam: LgsCamera, tile_w, tile_h,
                                 final_T, last_contrib, dL_dimage, grad_acc, workspace,
                                 stream=None, precision=LGS_FP32):
    L = load()
    _check(L.lgs_raster_bwd_deterministic(
        ctypes.byref(sp), _ptr(vals), _ptr(tile_ranges), ctypes.byref(cam), tile_w, tile_h,
        int(precision), _ptr(final_T), _ptr(last_contrib), _ptr(dL_dimage), _ptr(grad_acc),
        grad_acc.shape[0], _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream)), "lgs_raster_bwd_deterministic")


def lgs_round_planes(src, dst, n_planes: int, n: int, stream=None):
    """dst (bfloat16 / float16 planes) = src (float32 planes) rounded, rows < n."""
    L = load()
    dtype = {torch.bfloat16: LGS_SH_BF16, torch.float16: LGS_SH_F16}[dst.dtype]
    _check(L.lgs_round_planes(_ptr(src), src.shape[-1], _ptr(dst), dst.shape[-1], int(n_planes),
                              int(n), dtype, _stream(stream)), "lgs_round_planes")


def lgs_get_det_overflow() -> int:
    """Contributions the deterministic backward left out as out of range."""
    L = load()
    count = ctypes.c_uint32(0)
    st = L.lgs_get_det_overflow(ctypes.byref(count))
    if st not in (LGS_OK, LGS_ERR_CAPACITY):
        _check(st, "lgs_get_det_overflow")
    return int(count.value)


def lgs_opacity_variance(grad_acc, map_, d_num_visible, max_rows, metric, stream=None):
    L = load()
    _check(L.lgs_opacity_variance(_ptr(grad_acc), _ptr(map_), _ptr(d_num_visible), max_rows,
                                  _ptr(metric), _stream(stream)), "lgs_opacity_variance")


def lgs_preprocess_bwd(g: LgsGaussians, map_, d_num_visible, cam: LgsCamera, grad_acc,
                       grad_planes, stream=None, accumulate=False):
    L = load()
    _check(L.lgs_preprocess_bwd(ctypes.byref(g), _ptr(map_), _ptr(d_num_visible),
                                ctypes.byref(cam), _ptr(grad_acc), _ptr(grad_planes),
                                int(bool(accumulate)), _stream(stream)), "lgs_preprocess_bwd")


def _lr_array(lr) -> ctypes.Array:
    vals = [float(x) for x in lr]
    arr = (ctypes.c_float * len(vals))(*vals)
    return arr


def lgs_adam_step(params, grads, m, v, n_planes, lr, beta1, beta2, eps, step, map_,
                  d_num_visible, max_rows, stream=None):
    L = load()
    arr = _lr_array(lr)
    _check(L.lgs_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.shape[-1],
                           n_planes, arr, beta1, beta2, eps, step, _ptr(map_),
                           _ptr(d_num_visible), max_rows, _stream(stream)), "lgs_adam_step")


def lgs_preprocess_bwd_adam(g: LgsGaussians, m, v, map_, d_num_visible, cam: LgsCamera, grad_acc,
                            lr, beta1, beta2, eps, step, stream=None, splats=None, metric=None):
    """splats: the LgsSplats of the forward (optional; the colour clamp then
    comes from their stored colours and the SH planes are read once).
    metric: a float32 tensor of n rows (optional) that receives the a8
    densification metric as lgs_opacity_variance would write it."""
    L = load()
    arr = _lr_array(lr)
    _check(L.lgs_preprocess_bwd_adam(ctypes.byref(g), _ptr(m), _ptr(v), _ptr(map_),
                                     _ptr(d_num_visible), ctypes.byref(cam),
                                     ctypes.byref(splats) if splats is not None else None,
                                     _ptr(grad_acc), arr, beta1, beta2, eps, step,
                                     _ptr(metric), _stream(stream)),
           "lgs_preprocess_bwd_adam")


def lgs_moments_accumulate(grad_acc, map_, d_num_visible, max_rows, S, M, C, stream=None):
    L = load()
    _check(L.lgs_moments_accumulate(_ptr(grad_acc), _ptr(map_), _ptr(d_num_visible), max_rows,
                                    _ptr(S), _ptr(M), _ptr(C), _stream(stream)),
           "lgs_moments_accumulate")


def lgs_moments_metric(S, M, C, n, metric, stream=None):
    L = load()
    _check(L.lgs_moments_metric(_ptr(S), _ptr(M), _ptr(C), n, _ptr(metric), _stream(stream)),
           "lgs_moments_metric")


def lgs_densify_workspace_size(n: int) -> int:
    return int(load().lgs_densify_workspace_size(n))


def lgs_densify(g: LgsGaussians, m, v, metric, max_new, split_scale, normals, d_n_out,
                selected_out, workspace, stream=None):
    L = load()
    _check(L.lgs_densify(ctypes.byref(g), _ptr(m), _ptr(v), _ptr(metric), int(max_new),
                         float(split_scale), _ptr(normals), _ptr(d_n_out), _ptr(selected_out),
                         _ptr(workspace), workspace.numel(), _stream(stream)), "lgs_densify")


def lgs_opacity_decay(g: LgsGaussians, stream=None):
    L = load()
    _check(L.lgs_opacity_decay(ctypes.byref(g), _stream(stream)), "lgs_opacity_decay")


# ---- unit-rate microbenchmarks (measurement helpers; counts per call)
PEAK_THREADS = 256
PEAK_UNROLL = 32


def lgs_peak_ex2(out, blocks: int, iters: int, stream=None) -> int:
    """Enqueues the ex2 chain; returns the number of exponentials."""
    L = load()
    _check(L.lgs_peak_ex2(_ptr(out), int(blocks), int(iters), _stream(stream)), "lgs_peak_ex2")
    return blocks * PEAK_THREADS * PEAK_UNROLL * iters


def lgs_peak_ffma(out, blocks: int, iters: int, packed: bool, stream=None) -> int:
    """Enqueues the FMA chain (scalar or packed); returns the number of FMAs."""
    L = load()
    _check(L.lgs_peak_ffma(_ptr(out), int(blocks), int(iters), int(bool(packed)), _stream(stream)),
           "lgs_peak_ffma")
    return blocks * PEAK_THREADS * PEAK_UNROLL * iters * (2 if packed else 1)


def lgs_peak_red(rows, n_rows: int, blocks: int, iters: int, stream=None) -> int:
    """Enqueues the float reductions into rows; returns their number."""
    L = load()
    _check(L.lgs_peak_red(_ptr(rows), int(n_rows), int(blocks), int(iters), _stream(stream)),
           "lgs_peak_red")
    return blocks * (PEAK_THREADS // 32) * 12 * iters


def lgs_bin_keys(splats, vals, tile_ranges, keys, stream=None):
    """keys (int64 tensor, one per pair) = tile << 32 | depth bits of each
    pair of a finished binning (tile_ranges: [n_tiles, 2])."""
    L = load()
    _check(L.lgs_bin_keys(ctypes.byref(splats), _ptr(vals), _ptr(tile_ranges),
                          int(tile_ranges.shape[0]), _ptr(keys), _stream(stream)), "lgs_bin_keys")
