"""Closed-form cases for the cluster frustum cull (Sec. 3.2.2).

A cluster's box bounds its centres widened by 3 x the largest scale of each
member; it is culled when the box lies entirely outside one of the near plane
z = znear or the four side planes x = +-lx z, y = +-ly z (camera space,
lx = 1.3 W / (2 fx), ly = 1.3 H / (2 fy)). The camera here is turned by a
signed permutation, so a world-space cube of half-size e around c is, in
camera space, the cube of half-size e around C = R c + t, and whether it
meets the half-space inside a side plane is decided by its corner nearest to
that half-space:
    right   x <=  lx z :  C_x - e <=  lx (C_z + e)
    left    x >= -lx z :  C_x + e >= -lx (C_z + e)
    bottom  y <=  ly z :  C_y - e <=  ly (C_z + e)
    top     y >= -ly z :  C_y + e >= -ly (C_z + e)
    near    z >= znear :  C_z + e >= znear
Each case puts one cluster's nearest corner a relative 1e-3 of its distance
inside or outside exactly one plane, every other plane far inside.
"""
from __future__ import annotations

import numpy as np

W, H, FX, FY, ZNEAR = 96, 64, 80.0, 100.0, 0.2
LX, LY = 1.3 * W / (2 * FX), 1.3 * H / (2 * FY)
# world -> camera: camera z (forward) = world +x, camera y = world +y,
# camera x = world -z; a signed permutation whose transpose is another turn
R = np.array([[0.0, 0.0, -1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])
T = np.array([0.25, -0.5, 1.5])
CLUSTER = 128


def camera() -> dict:
    return {"R": R.astype(np.float32), "t": T.astype(np.float32), "fx": FX, "fy": FY,
            "cx": W / 2.0, "cy": H / 2.0, "width": W, "height": H, "znear": ZNEAR,
            "bg": np.zeros(3, np.float32)}


def _centre(plane: str, e: float, z: float, inside: bool, rel=1e-3) -> np.ndarray:
    """Camera-space centre of a cube of half-size e whose nearest corner lies
    a relative `rel` inside or outside `plane` at depth z."""
    if plane == "near":
        return np.array([0.0, 0.0, ZNEAR * ((1.0 + rel) if inside else (1.0 - rel)) - e])
    s = (1.0 - rel) if inside else (1.0 + rel)
    lim = LX if plane in ("right", "left") else LY
    edge = lim * (z + e) * s + e           # |coordinate| of the centre
    sign = 1.0 if plane in ("right", "bottom") else -1.0
    c = np.array([0.0, 0.0, z])
    c[0 if plane in ("right", "left") else 1] = sign * edge
    return c


def _world(C: np.ndarray) -> np.ndarray:
    return (C - T) @ R          # R^T (C - T) for each row


def side_plane_scene(scale: float = 0.01):
    """Ten clusters (128 identical Gaussians each, isotropic scale `scale`):
    for each of the five planes, one just inside (kept) and one just outside
    (culled). Returns (scene, expected visible flags)."""
    e = 3.0 * scale
    means, vis = [], []
    for plane in ("right", "left", "bottom", "top", "near"):
        for inside in (True, False):
            means.append(_world(_centre(plane, e, 3.0, inside)))
            vis.append(1 if inside else 0)
    mean = np.repeat(np.array(means), CLUSTER, axis=0)
    ls = np.full(mean.shape, np.log(scale))
    return {"mean": mean, "log_scale": ls}, np.array(vis, np.uint8)


def widening_scene():
    """Clusters whose centres all lie outside one side plane; one member has a
    largest scale s (on a different axis for each case) with 3 s a relative
    2e-3 above or below the reach e* the box needs to touch the plane
    (e* = distance of the nearest corner, from the closed form above solved
    for e). The others are tiny. Kept when 3 s >= e*, culled otherwise; with
    the widening factor or the largest-scale rule changed, cases flip.
    Returns (scene, expected visible flags)."""
    means, ls, vis = [], [], []
    tiny = np.log(1e-6)
    z = 2.0
    for plane, axis in (("right", 2), ("left", 0), ("bottom", 1), ("top", 2)):
        lim = LX if plane in ("right", "left") else LY
        ci = 0 if plane in ("right", "left") else 1
        sign = 1.0 if plane in ("right", "bottom") else -1.0
        # centres a fixed 0.3 beyond the plane at depth z
        C = np.array([0.0, 0.0, z])
        C[ci] = sign * (lim * z + 0.3)
        # reach needed: |C_i| - e <= lim (z + e)  <=>  e >= (|C_i| - lim z) / (1 + lim)
        e_star = (abs(C[ci]) - lim * z) / (1.0 + lim)
        for reaches in (True, False):
            s = e_star / 3.0 * ((1.0 + 2e-3) if reaches else (1.0 - 2e-3))
            block = np.repeat(_world(C)[None], CLUSTER, axis=0)
            lsb = np.full((CLUSTER, 3), tiny)
            lsb[17, axis] = np.log(s)     # one member, its largest scale on `axis`
            means.append(block)
            ls.append(lsb)
            vis.append(1 if reaches else 0)
    return ({"mean": np.concatenate(means), "log_scale": np.concatenate(ls)},
            np.array(vis, np.uint8))
