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


def assert_same_tile_lists(vals_a, ranges_a, vals_b, ranges_b):
    """Every tile's list is the same sequence (the tiles' groups may be laid
    out in different orders in the two vals arrays)."""
    ra, rb = np.asarray(ranges_a, np.int64), np.asarray(ranges_b, np.int64)
    assert ra.shape == rb.shape
    np.testing.assert_array_equal(ra[:, 1] - ra[:, 0], rb[:, 1] - rb[:, 0])
    va, vb = np.asarray(vals_a), np.asarray(vals_b)
    for t in np.flatnonzero(ra[:, 1] > ra[:, 0]):
        if not np.array_equal(va[ra[t, 0]:ra[t, 1]], vb[rb[t, 0]:rb[t, 1]]):
            raise AssertionError(f"tile {t}: lists differ")
