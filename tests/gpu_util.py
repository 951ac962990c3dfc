"""Helpers for the GPU parity tests: run single liblgs steps on numpy inputs
through the C ABI (via the binding) and return numpy outputs, plus the
comparison measures the tests use."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import pipeline as PL

DEV = "cuda"


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    B.load()


def t(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype))).to(DEV)


def rel_l2(a, b) -> float:
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def planes_tensor(scene: dict, stride: int | None = None) -> tuple[torch.Tensor, int]:
    p = PL.pack_planes(scene)
    n = p.shape[1]
    stride = stride or PL.round_up(max(n, 1), 128)
    out = np.zeros((p.shape[0], stride), np.float32)
    out[:, :n] = p
    return t(out), n


def gpu_preprocess(scene: dict, cam: dict, tile=(16, 16), rowmap=None, V=None):
    planes, n = planes_tensor(scene)
    g = B.gaussians_struct(planes, n, scene["sh_degree"])
    cs = B.camera_struct(cam)
    rows = n if V is None else V
    rec = torch.zeros((max(n, 1), 12), dtype=torch.float32, device=DEV)
    depth = torch.zeros(max(n, 1), dtype=torch.float32, device=DEV)
    radius = torch.zeros(max(n, 1), dtype=torch.int32, device=DEV)
    sp = B.splats_struct(rec, depth, radius)
    mp = None if rowmap is None else t(np.asarray(rowmap, np.uint32).view(np.int32))
    dV = None if V is None else t(np.array([V], np.int32))
    B.lgs_preprocess(g, mp, dV, cs, tile[0], tile[1], sp)
    torch.cuda.synchronize()
    r = rec.cpu().numpy()[:rows]
    return {"uv": r[:, 0:2], "conic": r[:, 2:5], "opacity": r[:, 5], "rgb": r[:, 6:9],
            "depth": depth.cpu().numpy()[:rows], "radius": radius.cpu().numpy()[:rows]}


def tau_of(opacity) -> np.ndarray:
    """The splat record's tau for the given opacities (input data here: the
    kernels read it from the record as given)."""
    t = 2.0 * np.log(255.0 * np.asarray(opacity, np.float64))
    return np.where(t > -1e30, t + 1e-3 * (1.0 + np.abs(t)), -np.inf).astype(np.float32)


def pack_splats(u, v, conic, opacity, rgb, depth, radius, tau=None):
    n = len(u)
    rec = np.zeros((max(n, 1), 12), np.float32)
    rec[:n, 0], rec[:n, 1] = u, v
    rec[:n, 2:5] = conic
    rec[:n, 5] = opacity
    rec[:n, 6:9] = rgb
    rec[:n, 9] = tau_of(opacity) if tau is None else tau
    d = np.zeros(max(n, 1), np.float32)
    d[:n] = depth
    r = np.zeros(max(n, 1), np.int32)
    r[:n] = radius
    return t(rec), t(d), t(r)


def gpu_bin(u, v, radius, depth, W, H, tile=(16, 16), cap=None, V=None, conic=None, tau=None,
            cull=0):
    n = len(u)
    zeros3 = np.zeros((n, 3), np.float32)
    rec, d, r = pack_splats(u, v, zeros3 if conic is None else conic, np.zeros(n), zeros3, depth,
                            radius, tau=np.zeros(n, np.float32) if tau is None else tau)
    sp = B.splats_struct(rec, d, r)
    cam = {"R": np.eye(3), "t": np.zeros(3), "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0,
           "width": W, "height": H, "znear": 0.2, "bg": np.zeros(3)}
    cs = B.camera_struct(cam)
    gx, gy = -(-W // tile[0]), -(-H // tile[1])
    cap = cap or max(64, 200 * n)
    vals = torch.zeros(cap, dtype=torch.int32, device=DEV)
    dP = torch.zeros(1, dtype=torch.int64, device=DEV)
    ranges = torch.zeros((gx * gy, 2), dtype=torch.int32, device=DEV)
    ws = torch.empty(B.lgs_bin_sort_workspace_size(max(n, 1), cap, gx * gy), dtype=torch.uint8,
                     device=DEV)
    dV = None if V is None else t(np.array([V], np.int32))
    B.lgs_bin_sort(sp, dV, max(n, 1), cs, tile[0], tile[1], vals, dP, ranges, ws, tile_cull=cull)
    torch.cuda.synchronize()
    P = int(dP.item())
    return (vals.cpu().numpy().view(np.uint32)[:min(P, cap)], ranges.cpu().numpy().view(np.uint32),
            P)


def gpu_raster(sp: dict, cam: dict, tile=(16, 16), dLdI=None, cull=1, precision=B.LGS_FP32):
    """Bin + forward (+ backward if dLdI is given) of float32 splats.
    sp: uv, conic, opacity, rgb, depth, radius, tau (float32 / int32)."""
    n = sp["uv"].shape[0]
    rec, d, r = pack_splats(sp["uv"][:, 0], sp["uv"][:, 1], sp["conic"], sp["opacity"], sp["rgb"],
                            sp["depth"], sp["radius"], tau=sp["tau"])
    spl = B.splats_struct(rec, d, r)
    cs = B.camera_struct(cam)
    W, H = cam["width"], cam["height"]
    gx, gy = -(-W // tile[0]), -(-H // tile[1])
    cap = max(1024, 400 * n)
    vals = torch.zeros(cap, dtype=torch.int32, device=DEV)
    dP = torch.zeros(1, dtype=torch.int64, device=DEV)
    ranges = torch.zeros((gx * gy, 2), dtype=torch.int32, device=DEV)
    ws = torch.empty(B.lgs_bin_sort_workspace_size(max(n, 1), cap, gx * gy), dtype=torch.uint8,
                     device=DEV)
    B.lgs_bin_sort(spl, None, max(n, 1), cs, tile[0], tile[1], vals, dP, ranges, ws, tile_cull=cull)
    image = torch.zeros((3, H, W), dtype=torch.float32, device=DEV)
    T = torch.zeros((H, W), dtype=torch.float32, device=DEV)
    last = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    B.lgs_raster_fwd(spl, vals, ranges, cs, tile[0], tile[1], image, T, last, precision=precision)
    out = {}
    if dLdI is not None:
        gacc = torch.zeros((max(n, 1), 16), dtype=torch.float32, device=DEV)
        B.lgs_raster_bwd(spl, vals, ranges, cs, tile[0], tile[1], T, last,
                         t(np.asarray(dLdI, np.float32)), gacc, precision=precision)
        torch.cuda.synchronize()
        ga = gacc.cpu().numpy()[:n]
        out.update(grad9=ga[:, :9], S=ga[:, 9], M=ga[:, 10], C=ga[:, 11].view(np.uint32),
                   pad=ga[:, 12:])
    torch.cuda.synchronize()
    P = int(dP.item())
    out.update(image=image.cpu().numpy(), T=T.cpu().numpy(), last=last.cpu().numpy(),
               vals=vals.cpu().numpy().view(np.uint32)[:P], ranges=ranges.cpu().numpy().view(np.uint32),
               P=P)
    # the device buffers, for further calls on the same binning and forward
    out["dev"] = {"splats": spl, "keep": (rec, d, r), "vals": vals, "ranges": ranges, "T": T,
                  "last": last, "cam": cs, "n": n}
    return out


def f32_splats(sp64: dict) -> dict:
    """Round the oracle's double-precision splats to the float32 the kernels read."""
    return {"uv": sp64["uv"].astype(np.float32), "conic": sp64["conic"].astype(np.float32),
            "opacity": sp64["opacity"].astype(np.float32), "rgb": sp64["rgb"].astype(np.float32),
            "depth": sp64["depth"].astype(np.float32), "radius": sp64["radius"].astype(np.int32),
            "tau": sp64["tau"].astype(np.float32)}


def random_splat_dict(n, seed, W, H, max_radius=40):
    from paper_2503_01199_gb300 import scenegen
    s = scenegen.random_splats(n, seed, W, H, max_radius=max_radius)
    return {"uv": np.stack([s["u"], s["v"]], 1), "conic": s["conic"], "opacity": s["opacity"],
            "rgb": s["rgb"], "depth": s["depth"], "radius": s["radius"], "tau": tau_of(s["opacity"])}


def assert_same_tile_lists(vals_a, ranges_a, vals_b, ranges_b, near=None, max_near_diff=None):
    """Every tile's list is the same sequence (the tiles' groups may be laid
    out in different orders in the two vals arrays). `near` (uint64 keys
    (tile << 32) | splat from the oracle's tile_near_pairs) names the pairs
    whose tile-culling decision lies within rounding of tau: either side may
    list those, so they are removed from both lists before the comparison,
    and only they may make the lists' lengths differ. Returns the keys of
    the near pairs listed by one side only."""
    ra, rb = np.asarray(ranges_a, np.int64), np.asarray(ranges_b, np.int64)
    assert ra.shape == rb.shape
    va, vb = np.asarray(vals_a), np.asarray(vals_b)
    near_by_tile = {}
    if near is not None and len(near):
        keys = np.asarray(near, np.uint64)
        tiles, splats = (keys >> np.uint64(32)).astype(np.int64), (keys & np.uint64(0xffffffff)).astype(np.int64)
        for t_, j in zip(tiles.tolist(), splats.tolist()):
            near_by_tile.setdefault(t_, set()).add(j)
    diff = []
    la, lb = ra[:, 1] - ra[:, 0], rb[:, 1] - rb[:, 0]
    for t_ in np.flatnonzero((la > 0) | (lb > 0)):
        a, b = va[ra[t_, 0]:ra[t_, 1]], vb[rb[t_, 0]:rb[t_, 1]]
        if np.array_equal(a, b):
            continue
        nb = near_by_tile.get(int(t_))
        if nb is None:
            raise AssertionError(f"tile {t_}: lists differ")
        fa = np.array([j for j in a.tolist() if j not in nb], np.int64)
        fb = np.array([j for j in b.tolist() if j not in nb], np.int64)
        if not np.array_equal(fa, fb):
            raise AssertionError(f"tile {t_}: lists differ outside the near-tau pairs")
        diff += [(int(t_) << 32) | j for j in sorted(set(a.tolist()) ^ set(b.tolist()))]
    if max_near_diff is not None:
        assert len(diff) <= max_near_diff, len(diff)
    return np.array(diff, np.uint64)


def assert_near_pairs_hold_no_fragment(near, sp, W, H, tile=(16, 16)):
    """The given (tile << 32) | splat pairs hold no fragment that passes the
    alpha >= 1/255 test, so listing them or not changes no pixel (tau is
    widened by 1e-3 (1 + |tau|) beyond that threshold, far more than the
    rounding of a single-precision decision). Brute force over every pixel
    centre of each pair's tile, in double precision."""
    gx = -(-W // tile[0])
    keys = np.asarray(near, np.uint64)
    for key in keys.tolist():
        t_, j = key >> 32, key & 0xffffffff
        tx, ty = t_ % gx, t_ // gx
        px, py = np.meshgrid(tx * tile[0] + np.arange(tile[0]) + 0.5, ty * tile[1] + np.arange(tile[1]) + 0.5)
        A, B_, C = (float(c) for c in sp["conic"][j])
        dx, dy = float(sp["uv"][j, 0]) - px, float(sp["uv"][j, 1]) - py
        a = float(sp["opacity"][j]) * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B_ * dx * dy)
        assert (a < 1.0 / 255.0).all(), (t_, j, a.max())


def last_ids(last, vals, ranges, W, tile=(16, 16)):
    """Each pixel's last composited splat as a splat index (-1 for none):
    `last` is a position in the pixel's tile list, so two binnings that
    differ only in near-tau pairs (which hold no fragment) give different
    positions for the same splat."""
    last = np.asarray(last, np.int64)
    H = last.shape[0]
    gx = -(-W // tile[0])
    ys, xs = np.mgrid[0:H, 0:last.shape[1]]
    t_ = (ys // tile[1]) * gx + xs // tile[0]
    start = np.asarray(ranges, np.int64)[t_, 0]
    v = np.asarray(vals, np.int64)
    out = np.full(last.shape, -1, np.int64)
    m = last > 0
    out[m] = v[start[m] + last[m] - 1]
    return out


def check_bins(orc, vals, ranges, P, sp, W, H, tile=(16, 16), cull=True, max_near_frac=1e-3):
    """Compares a GPU binning of float32 splats `sp` (uv, conic, depth,
    radius, tau, opacity) with the oracle's: bit-exact tile lists apart from
    near-tau pairs (at most max_near_frac of P differ), which must hold no
    contributing fragment when the conic is positive definite. Returns the
    oracle's (vals, ranges, P)."""
    u, v = sp["uv"][:, 0], sp["uv"][:, 1]
    rv, rr, rP = orc.bin_splats(u, v, sp["radius"], sp["depth"], W, H, tile,
                                conic=sp["conic"] if cull else None, tau=sp["tau"] if cull else None,
                                cull=bool(cull))
    near = orc.tile_near_pairs(u, v, sp["radius"], sp["conic"], sp["tau"], W, H, tile) if cull else None
    diff = assert_same_tile_lists(vals, ranges, rv, rr, near=near,
                                  max_near_diff=int(max_near_frac * max(rP, 1)))
    assert abs(P - rP) <= len(diff), (P, rP, len(diff))
    if len(diff) and "opacity" in sp:
        # the pairs the two binnings decide differently hold no contributing
        # fragment (definite conics only: the others have no such meaning)
        c = np.asarray(sp["conic"], np.float64)
        pd = (c[:, 0] > 0) & (c[:, 0] * c[:, 2] - c[:, 1] ** 2 > 0)
        j = (diff & np.uint64(0xffffffff)).astype(np.int64)
        assert_near_pairs_hold_no_fragment(diff[pd[j]], sp, W, H, tile)
    return rv, rr, rP
