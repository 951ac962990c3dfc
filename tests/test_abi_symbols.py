"""The C-ABI library builds, loads and exports every entry point that
include/lgs.h declares, and the Python binding wraps exactly those. No
compute call is made (no GPU needed)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared() -> set[str]:
    text = (ROOT / "include" / "lgs.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(lgs_[a-z0-9_]+)\s*\(", text))


def test_header_declares_the_hot_path():
    names = declared()
    for step in ("lgs_morton_reorder", "lgs_cluster_cull_compact", "lgs_preprocess",
                 "lgs_bin_sort", "lgs_raster_fwd", "lgs_raster_bwd", "lgs_opacity_variance",
                 "lgs_preprocess_bwd", "lgs_adam_step"):
        assert step in names


def test_library_exports_every_declared_symbol():
    from paper_2503_01199_gb300 import binding as B
    B.load()
    lib = ctypes.CDLL(str(B.library_path()))
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(B.ENTRY_POINTS) == declared()
    assert B.lgs_version().startswith("lgs")
    assert lib.lgs_debug_build() == 0


def test_debug_build_exports_the_same_symbols():
    """The bounds-checked build is the same ABI with checks compiled in."""
    from paper_2503_01199_gb300 import build as LB
    LB.build()
    lib = ctypes.CDLL(str(LB.DEBUG_LIB))
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.lgs_debug_build() == 1


def test_invalid_arguments_are_rejected_without_a_gpu():
    from paper_2503_01199_gb300 import binding as B
    L = B.load()
    # null pointers / sizes are refused before anything is enqueued
    assert L.lgs_loss_l1(None, None, 0, None, None, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_morton_reorder(None, None, 0, 0, 0, None, None, None, 0, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_adam_step(None, None, None, None, 0, 0, None, 0.9, 0.999, 1e-15, 1, None, None, 0,
                           None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_bin_sort_workspace_size(1000, 100000, 64) > 100000 * 6
    assert L.lgs_bin_keys(None, None, None, 0, None, None) == B.LGS_ERR_INVALID_ARG
    # unit-rate microbenchmarks: null buffers, sizes and counts out of range
    assert L.lgs_peak_ex2(None, 8, 1, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_ffma(None, 8, 1, 1, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_red(None, 16, 8, 1, None) == B.LGS_ERR_INVALID_ARG
    # (a host buffer: every call below is refused before any launch)
    raw, addr = _aligned(16 * 16 * 4)
    ptr = ctypes.c_void_p(addr)
    assert L.lgs_peak_ex2(ptr, 0, 1, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_ffma(ptr, 8, 0, 0, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_red(ptr, 0, 8, 1, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_red(ptr, 1 << 31, 8, 1, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_peak_red(ctypes.c_void_p(addr + 4), 16, 8, 1, None) == B.LGS_ERR_INVALID_ARG


def _aligned(nbytes: int):
    import numpy as np
    raw = np.zeros(nbytes + 64, np.uint8)
    off = (-raw.ctypes.data) % 64
    return raw, raw.ctypes.data + off


def test_capacity_and_grid_rules_are_checked_on_the_host():
    """The argument rules the header states for the binning and the fused
    optimizer are checked before anything is enqueued: every case below is
    refused without touching a device."""
    from paper_2503_01199_gb300 import binding as B
    L = B.load()
    keep = []

    def buf(nbytes):
        raw, p = _aligned(nbytes)
        keep.append(raw)
        return ctypes.c_void_p(p)

    cam = B.LgsCamera()
    cam.R[:] = [1, 0, 0, 0, 1, 0, 0, 0, 1]
    cam.fx = cam.fy = 500.0
    cam.cx, cam.cy, cam.width, cam.height, cam.znear = 64.0, 64.0, 128, 128, 0.01
    n = 256
    sp = B.LgsSplats(buf(48 * n).value, buf(4 * n).value, buf(4 * n).value, n)
    ws = buf(1 << 20)
    vals, npairs, ranges, nvis = buf(4 * 4096), buf(8), buf(8 * 65536), buf(4)

    def bin_sort(sp_, max_splats, cam_, tw, th, cull, cap, wsb=1 << 20):
        return L.lgs_bin_sort(ctypes.byref(sp_), nvis, max_splats, ctypes.byref(cam_), tw, th, cull,
                              vals, cap, npairs, ranges, ws, wsb, None)

    bad = B.LGS_ERR_INVALID_ARG
    assert bin_sort(sp, n + 1, cam, 16, 16, 1, 4096) == bad          # capacity < max_splats
    assert bin_sort(sp, n, cam, 16, 16, 2, 4096) == bad              # tile_cull not 0 / 1
    assert bin_sort(sp, n, cam, 0, 16, 1, 4096) == bad               # empty tile
    assert bin_sort(sp, n, cam, 16, 16, 1, 1 << 32) == bad           # pairs beyond u32 indices
    assert bin_sort(sp, n, cam, 16, 16, 1, 4096, wsb=16) == bad      # workspace too small
    big = B.LgsCamera.from_buffer_copy(cam)
    big.width, big.height = 257 * 16, 256 * 16                       # 65,792 tiles > 65,536
    assert bin_sort(sp, n, big, 16, 16, 1, 4096) == bad
    unaligned = B.LgsSplats(sp.rec + 4, sp.depth, sp.radius, n)
    assert bin_sort(unaligned, n, cam, 16, 16, 1, 4096) == bad

    deg = 3
    stride = 256
    planes = buf(4 * B.num_planes(deg) * stride)
    g = B.LgsGaussians(planes.value, n, stride, deg, B.LGS_SH_F32, None)
    m, v = buf(4 * B.num_planes(deg) * stride), buf(4 * B.num_planes(deg) * stride)
    gacc, lr, rowmap = buf(64 * n), buf(4 * B.num_planes(deg)), buf(4 * n)

    def fused(g_, sp_, gacc_=gacc, step=1, cam_=cam):
        return L.lgs_preprocess_bwd_adam(ctypes.byref(g_), m, v, rowmap, nvis, ctypes.byref(cam_),
                                         None if sp_ is None else ctypes.byref(sp_), gacc_, lr,
                                         0.9, 0.999, 1e-15, step, None, None)

    small = B.LgsSplats(sp.rec, sp.depth, sp.radius, n - 1)
    assert fused(g, small) == bad                                    # records fewer than rows
    assert fused(g, sp, step=0) == bad                               # Adam step counts from 1
    assert fused(g, sp, gacc_=ctypes.c_void_p(gacc.value + 4)) == bad
    posed = B.LgsCamera.from_buffer_copy(cam)
    posed.d_pose = buf(48).value                                     # training takes a host pose
    assert fused(g, sp, cam_=posed) == bad
    g16 = B.LgsGaussians(planes.value, n, stride, deg, B.LGS_SH_BF16, buf(2 * 48 * stride).value)
    assert fused(g16, None) == bad                                   # 16-bit copy needs the records
    assert L.lgs_preprocess_bwd(ctypes.byref(g16), rowmap, nvis, ctypes.byref(cam), gacc,
                                buf(4 * 59 * stride), 0, None) == bad  # separate backward: FP32 only
    h16 = buf(2 * 48 * stride)
    assert L.lgs_round_planes(planes, stride, h16, stride, 48, n, 7, None) == bad   # bad dtype
    assert L.lgs_round_planes(planes, stride, h16, n - 1, 48, n, B.LGS_SH_BF16, None) == bad
    skew = B.LgsGaussians(planes.value, n, stride + 2, deg, B.LGS_SH_F32, None)
    assert fused(skew, sp) == bad                                    # stride a multiple of 4

    # the deterministic backward: its workspace size and the raster rules
    assert L.lgs_raster_bwd_det_workspace_size(n) == 160 * n
    img = buf(4 * 128 * 128 * 3)
    fT, lastc = buf(4 * 128 * 128), buf(4 * 128 * 128)
    dws = buf(160 * n)

    def det(tw=16, ws_=dws, wsb=160 * n, prec=B.LGS_FP32, gacc_=gacc, rows=n):
        return L.lgs_raster_bwd_deterministic(ctypes.byref(sp), vals, ranges, ctypes.byref(cam), tw,
                                              16, prec, fT, lastc, img, gacc_, rows, ws_, wsb, None)

    assert det(wsb=160 * n - 1) == bad                               # workspace too small
    assert det(ws_=ctypes.c_void_p(dws.value + 8)) == bad            # workspace not 16-byte aligned
    assert det(tw=8) == bad                                          # 16 x 16 tiles only
    assert det(prec=3) == bad                                        # unknown precision
    assert det(gacc_=ctypes.c_void_p(gacc.value + 4)) == bad         # gradient rows unaligned
