"""CPU oracle for the LiteGS rasterizer training step (arXiv 2503.01199).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package. The product path (``paper_2503_01199_gb300``) never imports it and
shares no code with it; the only thing both sides take is the seeded input
of ``paper_2503_01199_gb300.scenegen``, which is passed in as arrays.

The arithmetic lives in ``lgs_oracle.c`` (plain C, double precision, one
function per step, each citing the paper). This module compiles it with gcc
on first use and converts numpy arrays in and out.

Thresholds that a single-precision kernel may decide differently from this
double-precision code are reported rather than hidden:
  * preprocess ``flags`` bit0: the radius within rounding of a step; bit1:
    the near-plane test within rounding; bit2: the tile rectangle's edges
    within rounding of a tile boundary;
  * render ``pixflags`` bit0: an alpha (1/255) or transmittance (1e-4) test
    within a relative margin of its threshold (set_margins(): 2e-4 by
    default); bit1: two included splats whose depths differ by less than a
    relative 2e-6 (their order may flip);
  * render-backward ``sflags`` bit0: a fragment in a flagged pixel; bit1: a
    fragment with o*G within the alpha margin of the 0.99 clamp;
  * tile culling (``tile_reachable``, ``tile_near_pairs``): (splat, tile)
    pairs whose box minimum of the exponent's quadratic form lies within
    rounding of tau. tau is widened beyond alpha = 1/255, so such a pair
    holds no fragment that passes the alpha test, and listing it or not
    changes no pixel, only list positions.
Parity tests compare exactly where no flag is set and count the flagged.

Every function here is pinned by the CPU tests in ``tests/test_oracle_*.py``
against closed forms, brute force, finite differences or library routines.
"""
from __future__ import annotations

import ctypes
import os
import platform
import shutil
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lgs_oracle.c"
_OUT = _HERE / "_build" / "liblgs_oracle.so"
_lib = None
OMP = False

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def build(force: bool = False) -> Path:
    """Compile lgs_oracle.c into oracle/_build/liblgs_oracle.so (gcc, -O2)."""
    global OMP
    _OUT.parent.mkdir(exist_ok=True)
    machine = _OUT.parent / "machine.txt"
    if (not force and _OUT.exists() and _OUT.stat().st_mtime >= _SRC.stat().st_mtime
            and machine.exists() and machine.read_text().strip() == platform.machine()):
        OMP = (_OUT.parent / "omp").exists()
        return _OUT
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", str(_SRC)]
    tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
    r = subprocess.run(base + ["-fopenmp", "-o", str(tmp), "-lm"], capture_output=True, text=True)
    omp = r.returncode == 0
    if not omp:
        r = subprocess.run(base + ["-o", str(tmp), "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _OUT)
    machine.write_text(platform.machine())
    flag = _OUT.parent / "omp"
    if omp:
        flag.write_text("1")
    elif flag.exists():
        flag.unlink()
    OMP = omp
    return _OUT


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(str(path))
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "or_version": (i32, []),
            "or_set_margins": (None, [f64] * 5),
            "or_sh_basis_spherical": (None, [i32, P, P]),
            "or_sh_basis_cartesian": (None, [i32, P, P, P]),
            "or_preprocess": (None, [i64, i32, P, P, P, P, P, P, i32, i32, P, P, P, P, P, P, P, P, P]),
            "or_morton_interleave": (ctypes.c_uint64, [ctypes.c_uint32] * 3),
            "or_morton_codes": (None, [i64, P, P]),
            "or_sort_u64_stable": (None, [i64, P, P]),
            "or_cluster_cull": (i64, [i64, i32, P, P, P, P, P, P, P]),
            "or_bin": (i64, [i64, P, P, P, P, P, P, i32, i32, i32, i32, i32, i64, P, P]),
            "or_render_fwd": (ctypes.c_uint64, [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P]),
            "or_render_bwd": (None, [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, i64, P, P, P, P, P]),
            "or_l1_loss": (f64, [i64, P, P, P]),
            "or_opacity_variance": (None, [i64, P, P, P, P]),
            "or_preprocess_bwd": (None, [i64, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]),
            "or_adam": (None, [i64, i32, P, P, P, P, P, f64, f64, f64, i32, P, i64]),
            "or_densify": (i64, [i64, i32, i64, P, P, P, P, i64, f64, P, P]),
            "or_tile_reachable": (None, [i64, P, P, P, P, P, P, i32, i32, P]),
            "or_tile_near_pairs": (i64, [i64, P, P, P, P, P, i32, i32, i32, i32, i64, P]),
            "or_set_tau_margin": (None, [f64]),
            "or_set_threads": (i32, [i32]),
            "or_opacity_decay": (None, [i64, P]),
            "or_moments_accumulate": (None, [i64, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


MARGINS_END_TO_END = (2e-4, 2e-4, 2e-3, 1e-5, 5e-7)
TAU_MARGIN = 4e-6   # the tile decisions' near-tau flag (or_set_tau_margin)
MARGINS_SHARED_SPLATS = (2e-5, 2e-4, 2e-3, 1e-5, 0.0)


def set_margins(alpha: float, T: float, px: float, radius: float, depth: float) -> None:
    """Flag margins (relative for alpha, T, radius, depth; pixels for px).

    A single-precision kernel computes alpha = o exp(power) with a relative
    error of a few 1e-6 when it reads the same float32 splats
    (MARGINS_SHARED_SPLATS), and of a few 1e-5 when it also projected them
    itself (MARGINS_END_TO_END, the default: the screen centre carries a
    1e-5 px rounding that the exponent's slope of ~3 / sigma amplifies).
    Depths: with shared float32 depths both sides order equal keys by the
    same stable rule (margin 0 disables the flag); a kernel that computes
    the depth itself is within a few ulps (5e-7 relative).
    """
    lib().or_set_margins(alpha, T, px, radius, depth)


def threads() -> int:
    """Threads the oracle uses (OpenMP's current setting, else 1)."""
    lib()
    if not OMP:
        return 1
    return int(_lib.or_set_threads(-1))


def set_threads(n: int | None) -> int:
    """Use n threads in the oracle's parallel loops (None: all processors);
    returns the number in use."""
    lib()
    return int(_lib.or_set_threads(int(n) if n else 0))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def camera_array(cam: dict) -> np.ndarray:
    return np.concatenate([
        np.asarray(cam["R"], np.float64).reshape(9), np.asarray(cam["t"], np.float64).reshape(3),
        [cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"], cam["znear"]],
        np.asarray(cam["bg"], np.float64).reshape(3)]).astype(np.float64)


def grid(cam: dict, tile) -> tuple[int, int]:
    tw, th = tile
    return (cam["width"] + tw - 1) // tw, (cam["height"] + th - 1) // th


# --------------------------------------------------------------------------
# spherical harmonics
# --------------------------------------------------------------------------
def sh_spherical(deg: int, d) -> np.ndarray:
    d = _c(d, np.float64)
    Y = np.zeros(16)
    lib().or_sh_basis_spherical(deg, _p(d), _p(Y))
    return Y[: (deg + 1) ** 2]


def sh_cartesian(deg: int, d):
    d = _c(d, np.float64)
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().or_sh_basis_cartesian(deg, _p(d), _p(Y), _p(dY))
    k = (deg + 1) ** 2
    return Y[:k], dY[:k]


# --------------------------------------------------------------------------
# steps
# --------------------------------------------------------------------------
def _scene64(scene: dict):
    return (_c(scene["mean"], np.float64), _c(scene["log_scale"], np.float64),
            _c(scene["quat"], np.float64), _c(scene["logit"], np.float64),
            _c(scene["sh"], np.float64))


def preprocess(scene: dict, cam: dict, tile=(16, 16)) -> dict:
    """EWA projection, SH colour and opacity per Gaussian (double precision)."""
    mean, ls, q, logit, sh = _scene64(scene)
    n = mean.shape[0]
    out = {"uv": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "depth": np.zeros(n),
           "opacity": np.zeros(n), "rgb": np.zeros((n, 3)), "radius": np.zeros(n, np.int32),
           "rect": np.zeros((n, 4), np.int32), "flags": np.zeros(n, np.uint8),
           "tau": np.zeros(n)}
    camv = camera_array(cam)
    lib().or_preprocess(n, int(scene["sh_degree"]), _p(mean), _p(ls), _p(q), _p(logit), _p(sh),
                        _p(camv), tile[0], tile[1], _p(out["uv"]), _p(out["conic"]),
                        _p(out["depth"]), _p(out["opacity"]), _p(out["rgb"]), _p(out["radius"]),
                        _p(out["rect"]), _p(out["flags"]), _p(out["tau"]))
    return out


def morton_codes(mean) -> np.ndarray:
    mean = _c(mean, np.float32)
    codes = np.zeros(mean.shape[0], np.uint64)
    lib().or_morton_codes(mean.shape[0], _p(mean), _p(codes))
    return codes


def morton_interleave(x: int, y: int, z: int) -> int:
    return int(lib().or_morton_interleave(x, y, z))


def sort_u64_stable(keys) -> np.ndarray:
    keys = _c(keys, np.uint64)
    perm = np.zeros(keys.shape[0], np.uint32)
    lib().or_sort_u64_stable(keys.shape[0], _p(keys), _p(perm))
    return perm


def morton_reorder(scene: dict) -> tuple[np.ndarray, np.ndarray]:
    """Morton codes of the centres and the stable sort permutation (Sec. 3.2.1)."""
    codes = morton_codes(scene["mean"])
    perm = sort_u64_stable(codes)
    return codes[perm], perm


def cluster_cull(scene: dict, cam: dict, cluster: int = 128) -> dict:
    mean, ls = _c(scene["mean"], np.float64), _c(scene["log_scale"], np.float64)
    n = mean.shape[0]
    ncl = (n + cluster - 1) // cluster
    aabb = np.zeros((ncl, 6))
    vis = np.zeros(ncl, np.uint8)
    flags = np.zeros(ncl, np.uint8)
    rowmap = np.zeros(n, np.uint32)
    camv = camera_array(cam)
    V = lib().or_cluster_cull(n, cluster, _p(mean), _p(ls), _p(camv), _p(aabb), _p(vis),
                              _p(flags), _p(rowmap))
    return {"aabb": aabb, "visible": vis, "flags": flags, "map": rowmap[:V], "V": int(V)}


def bin_splats(u, v, radius, depth, width: int, height: int, tile=(16, 16), conic=None,
               tau=None, cull=None):
    """Per-tile depth-ordered lists: (vals, ranges[ntiles, 2], P). With conic
    and tau given (float32 [n,3], [n]) the tile-level culling test applies
    (cull defaults to whether they are given)."""
    u, v = _c(u, np.float32), _c(v, np.float32)
    radius, depth = _c(radius, np.int32), _c(depth, np.float32)
    n = u.shape[0]
    if cull is None:
        cull = conic is not None and tau is not None
    if cull:
        conic, tau = _c(conic, np.float32), _c(tau, np.float32)
    gx, gy = (width + tile[0] - 1) // tile[0], (height + tile[1] - 1) // tile[1]
    ranges = np.zeros((gx * gy, 2), np.uint32)
    cp = _p(conic) if cull else None
    tp = _p(tau) if cull else None
    # count first, then fill
    P = lib().or_bin(n, _p(u), _p(v), _p(radius), _p(depth), cp, tp, int(bool(cull)), width,
                     height, tile[0], tile[1], 0, None, _p(ranges))
    vals = np.zeros(max(P, 1), np.uint32)
    P2 = lib().or_bin(n, _p(u), _p(v), _p(radius), _p(depth), cp, tp, int(bool(cull)), width,
                      height, tile[0], tile[1], P, _p(vals), _p(ranges))
    assert P2 == P
    return vals[:P], ranges, int(P)


def _splat64(sp: dict):
    return (_c(sp["uv"], np.float64), _c(sp["conic"], np.float64), _c(sp["opacity"], np.float64),
            _c(sp["rgb"], np.float64), _c(sp["depth"], np.float64))


def render_fwd(sp: dict, vals, ranges, cam: dict, tile=(16, 16)) -> dict:
    """Eq. 1-2 / Alg. 1 per pixel. sp holds uv, conic, opacity, rgb, depth."""
    uv, conic, op, rgb, depth = _splat64(sp)
    W, H = cam["width"], cam["height"]
    vals, ranges = _c(vals, np.uint32), _c(ranges, np.uint32)
    bg = _c(cam["bg"], np.float64)
    image = np.zeros((3, H, W))
    T = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    pf = np.zeros((H, W), np.uint8)
    h = lib().or_render_fwd(W, H, tile[0], tile[1], _p(bg), _p(uv), _p(conic), _p(op), _p(rgb),
                            _p(depth), _p(vals if vals.size else np.zeros(1, np.uint32)),
                            _p(ranges), _p(image), _p(T), _p(last), _p(pf))
    return {"image": image, "T": T, "last": last, "pixflags": pf, "hash": int(h)}


def render_bwd(sp: dict, vals, ranges, cam: dict, dL_dimage, tile=(16, 16)) -> dict:
    """Per-splat gradients (du, dv, dA, dB, dC, do, dr, dg, db) and S, M, C."""
    uv, conic, op, rgb, depth = _splat64(sp)
    n = uv.shape[0]
    W, H = cam["width"], cam["height"]
    vals, ranges = _c(vals, np.uint32), _c(ranges, np.uint32)
    bg = _c(cam["bg"], np.float64)
    g = _c(dL_dimage, np.float64)
    grad9 = np.zeros((n, 9))
    S, M = np.zeros(n), np.zeros(n)
    C = np.zeros(n, np.int64)
    sf = np.zeros(n, np.uint8)
    lib().or_render_bwd(W, H, tile[0], tile[1], _p(bg), _p(uv), _p(conic), _p(op), _p(rgb),
                        _p(depth), _p(vals if vals.size else np.zeros(1, np.uint32)), _p(ranges),
                        _p(g), n, _p(grad9), _p(S), _p(M), _p(C), _p(sf))
    return {"grad9": grad9, "S": S, "M": M, "C": C, "sflags": sf}


def l1_loss(image, target):
    image, target = _c(image, np.float64), _c(target, np.float64)
    grad = np.zeros_like(image)
    L = lib().or_l1_loss(image.size, _p(image), _p(target), _p(grad))
    return float(L), grad


def opacity_variance(S, M, C) -> np.ndarray:
    S, M, C = _c(S, np.float64), _c(M, np.float64), _c(C, np.int64)
    out = np.zeros_like(S)
    lib().or_opacity_variance(S.size, _p(S), _p(M), _p(C), _p(out))
    return out


def preprocess_bwd(scene: dict, cam: dict, grad9) -> dict:
    """Chain the nine splat gradients back to the Gaussian parameters."""
    mean, ls, q, logit, sh = _scene64(scene)
    n = mean.shape[0]
    g9 = _c(grad9, np.float64)
    g_uv, g_conic = _c(g9[:, 0:2], np.float64), _c(g9[:, 2:5], np.float64)
    g_o, g_rgb = _c(g9[:, 5], np.float64), _c(g9[:, 6:9], np.float64)
    out = {"mean": np.zeros((n, 3)), "log_scale": np.zeros((n, 3)), "quat": np.zeros((n, 4)),
           "logit": np.zeros(n), "sh": np.zeros_like(sh)}
    camv = camera_array(cam)
    lib().or_preprocess_bwd(n, int(scene["sh_degree"]), _p(mean), _p(ls), _p(q), _p(logit),
                            _p(sh), _p(camv), _p(g_uv), _p(g_conic), _p(g_o), _p(g_rgb),
                            _p(out["mean"]), _p(out["log_scale"]), _p(out["quat"]),
                            _p(out["logit"]), _p(out["sh"]))
    return out


def adam(param, grad, m, v, lr, step: int, rows, beta1=0.9, beta2=0.999, eps=1e-15):
    """Sparse Adam on planes [nplanes, nrows]; updates param, m, v in place."""
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _c(grad, np.float64)
    lr = _c(lr, np.float64)
    rows = _c(rows, np.uint32)
    nplanes, nrows = param.shape
    lib().or_adam(nrows, nplanes, _p(param), _p(grad), _p(m), _p(v), _p(lr), beta1, beta2, eps,
                  step, _p(rows), rows.size)


# --------------------------------------------------------------------------
# parameter planes (the order the step uses for Adam and the reorder)
# --------------------------------------------------------------------------
def densify(planes, m, v, metric, K: int, split_scale: float, normals) -> dict:
    """Variance-driven clone / split (Sec. 3.3, readings in lgs_oracle.c).
    planes, m, v: float64 [nplanes, stride] with stride >= n + K (copied);
    metric: C Var per Gaussian [n]; normals: standard normal samples
    [K, 2, 3]. Returns the new planes, m, v, the new count and the selected
    rows in selection order."""
    planes = np.array(planes, np.float64, order="C", copy=True)
    m = np.array(m, np.float64, order="C", copy=True)
    v = np.array(v, np.float64, order="C", copy=True)
    metric = _c(metric, np.float64)
    normals = _c(normals, np.float64)
    n = metric.shape[0]
    assert planes.shape[1] >= n + K and normals.size >= 6 * K
    sel = np.zeros(max(K, 1), np.int64)
    n_new = lib().or_densify(n, planes.shape[0], planes.shape[1], _p(planes), _p(m), _p(v),
                             _p(metric), K, float(split_scale), _p(normals), _p(sel))
    return {"planes": planes, "m": m, "v": v, "n": int(n_new), "selected": sel[:n_new - n]}


def tile_reachable(u, v, conic, tau, tx, ty, tile=(16, 16)):
    """The tile-culling decision for each (splat, tile) query: (listed,
    near), near marking a box minimum within rounding of tau."""
    u, v, tau = _c(u, np.float32), _c(v, np.float32), _c(tau, np.float32)
    conic = _c(conic, np.float32)
    tx, ty = _c(tx, np.int32), _c(ty, np.int32)
    out = np.zeros(u.size, np.uint8)
    lib().or_tile_reachable(u.size, _p(u), _p(v), _p(conic), _p(tau), _p(tx), _p(ty), tile[0],
                            tile[1], _p(out))
    return (out & 1).astype(bool), (out & 2).astype(bool)


def tile_near_pairs(u, v, radius, conic, tau, width: int, height: int, tile=(16, 16)) -> np.ndarray:
    """(tile << 32) | splat of every rectangle pair whose tile-culling
    decision is within rounding of tau (listed or not), uint64."""
    u, v, tau = _c(u, np.float32), _c(v, np.float32), _c(tau, np.float32)
    radius, conic = _c(radius, np.int32), _c(conic, np.float32)
    args = (u.size, _p(u), _p(v), _p(radius), _p(conic), _p(tau), width, height, tile[0], tile[1])
    k = lib().or_tile_near_pairs(*args, 0, None)
    keys = np.zeros(max(k, 1), np.uint64)
    k2 = lib().or_tile_near_pairs(*args, k, _p(keys))
    assert k2 == k
    return keys[:k]


def set_tau_margin(rel: float) -> None:
    """Relative input perturbation behind the tile decisions' near-tau flag."""
    lib().or_set_tau_margin(float(rel))


def opacity_decay(logit) -> np.ndarray:
    out = np.array(logit, np.float64, copy=True)
    lib().or_opacity_decay(out.size, _p(out))
    return out


def moments_accumulate(rows, S, M, C, S_acc, M_acc, C_acc):
    """Adds one view's moments of its visible rows into per-Gaussian sums (in place)."""
    rows, S, M, C = _c(rows, np.uint32), _c(S, np.float64), _c(M, np.float64), _c(C, np.int64)
    for a, t in ((S_acc, np.float64), (M_acc, np.float64), (C_acc, np.int64)):
        assert a.dtype == t and a.flags.c_contiguous
    lib().or_moments_accumulate(rows.size, _p(rows), _p(S), _p(M), _p(C), _p(S_acc), _p(M_acc),
                                _p(C_acc))


def scene_planes(scene: dict) -> np.ndarray:
    """Stack a scene into planes [11 + 3K, N]: mean(3), log-scale(3),
    quat(4), logit, then SH coefficient k channel c at 11 + 3k + c."""
    n = scene["mean"].shape[0]
    return np.ascontiguousarray(np.concatenate([
        np.asarray(scene["mean"], np.float64).T, np.asarray(scene["log_scale"], np.float64).T,
        np.asarray(scene["quat"], np.float64).T, np.asarray(scene["logit"], np.float64)[None],
        np.asarray(scene["sh"], np.float64).reshape(n, -1).T]))


def planes_scene(planes: np.ndarray, sh_degree: int) -> dict:
    n = planes.shape[1]
    return {"mean": planes[0:3].T.copy(), "log_scale": planes[3:6].T.copy(),
            "quat": planes[6:10].T.copy(), "logit": planes[10].copy(),
            "sh": planes[11:].T.reshape(n, -1, 3).copy(), "sh_degree": sh_degree}


def grad_planes(g: dict) -> np.ndarray:
    n = g["mean"].shape[0]
    return np.ascontiguousarray(np.concatenate([g["mean"].T, g["log_scale"].T, g["quat"].T,
                                                g["logit"][None], g["sh"].reshape(n, -1).T]))


# --------------------------------------------------------------------------
# composites
# --------------------------------------------------------------------------
def render_scene(scene: dict, cam: dict, tile=(16, 16), cull: bool = True) -> dict:
    """preprocess -> bin (with tile-level culling unless cull=False) ->
    forward; returns everything (double precision)."""
    sp = preprocess(scene, cam, tile)
    vals, ranges, P = bin_splats(sp["uv"][:, 0], sp["uv"][:, 1], sp["radius"], sp["depth"],
                                 cam["width"], cam["height"], tile, conic=sp["conic"],
                                 tau=sp["tau"], cull=cull)
    fw = render_fwd(sp, vals, ranges, cam, tile)
    return {"splats": sp, "vals": vals, "ranges": ranges, "P": P, **fw}


def loss_and_grad(scene: dict, cam: dict, target, tile=(16, 16)) -> dict:
    """L1 loss of the render and its gradient w.r.t. every parameter, plus a
    hash of every discrete decision taken (for finite-difference tests)."""
    r = render_scene(scene, cam, tile)
    L, dL = l1_loss(r["image"], target)
    bw = render_bwd(r["splats"], r["vals"], r["ranges"], cam, dL, tile)
    g = preprocess_bwd(scene, cam, bw["grad9"])
    sp = r["splats"]
    dec = r["hash"]
    h = np.concatenate([sp["radius"].astype(np.int64), sp["rect"].ravel().astype(np.int64),
                        (sp["rgb"] > 0).ravel().astype(np.int64),
                        np.sign(r["image"] - np.asarray(target, np.float64)).ravel().astype(np.int64)])
    return {"loss": L, "grad": g, "render": r, "bwd": bw,
            "decisions": (dec, hash(h.tobytes()), _clamp_signature(scene, cam))}


def _clamp_signature(scene: dict, cam: dict) -> int:
    """Which Gaussians have the 1.3 x FOV Jacobian clamp active (a kink)."""
    R = np.asarray(cam["R"], np.float64)
    pc = np.asarray(scene["mean"], np.float64) @ R.T + np.asarray(cam["t"], np.float64)
    limx = 1.3 * cam["width"] / (2.0 * cam["fx"])
    limy = 1.3 * cam["height"] / (2.0 * cam["fy"])
    with np.errstate(divide="ignore", invalid="ignore"):
        cx = np.sign(np.clip(np.abs(pc[:, 0] / pc[:, 2]) - limx, 0, None))
        cy = np.sign(np.clip(np.abs(pc[:, 1] / pc[:, 2]) - limy, 0, None))
    return hash(np.stack([cx, cy]).tobytes())
