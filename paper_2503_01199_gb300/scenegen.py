"""Seeded synthetic inputs: Gaussian scenes, cameras and target images.

This module only draws random numbers and lays them out. It holds none of
the rendering, projection or optimisation arithmetic, so both the CUDA path
and the CPU oracle can take their inputs from it without sharing any of the
method's code.

The scenes stand in for the paper's captures (Mip-NeRF 360, Tanks & Temples,
Deep Blending, Sec. 4), which are not available here. Their primitive counts
follow the scales of Table 3 (500k .. 5.7M) and their resolutions follow the
pre-downsampled captures (Sec. 4, "Datasets").

A scene is a dict of float32 arrays:
    mean       (N, 3)   world-space centre p_i                (Sec. 3, g_i)
    log_scale  (N, 3)   log of the per-axis standard deviation
    quat       (N, 4)   rotation quaternion, (w, x, y, z)
    logit      (N,)     opacity before the sigmoid
    sh         (N, K, 3) colour coefficients c_i, K = (deg+1)^2, l-major
plus 'sh_degree'. A camera is a dict with R (3x3 world->camera rotation,
row-major), t (3,), fx, fy, cx, cy, width, height, znear and bg (3,).

Draw order is fixed (means, log-scales, quaternions, logits, SH, then the
target or the camera angles), so a seed names one scene exactly.
"""
from __future__ import annotations

import numpy as np

ZNEAR = 0.2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sh(rng: np.random.Generator, n: int, sh_degree: int, dc_sigma: float,
        rest_sigma: float) -> np.ndarray:
    k = (sh_degree + 1) ** 2
    sh = np.empty((n, k, 3), np.float32)
    sh[:, 0, :] = rng.normal(0.0, dc_sigma, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_sigma, (n, k - 1, 3))
    return sh


def pinhole_camera(width: int, height: int, focal: float, R=None, t=None,
                   bg=(0.0, 0.0, 0.0)) -> dict:
    """A pinhole camera with the principal point at the image centre."""
    return {
        "R": np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
        "t": np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32),
        "fx": float(focal), "fy": float(focal),
        "cx": width / 2.0, "cy": height / 2.0,
        "width": int(width), "height": int(height),
        "znear": ZNEAR, "bg": np.asarray(bg, np.float32),
    }


def orbit_camera(radius: float, azimuth: float, elevation: float, width: int,
                 height: int, focal_scale: float = 0.78, center=(0.0, 0.0, 0.0)) -> dict:
    """Camera on a sphere of the given radius around `center`, looking at it,
    up = +y.

    Rows of R are the camera's x, y, z axes in world coordinates; the camera
    looks along +z (camera space), so a point in front has z > 0.
    """
    off = radius * np.array([np.cos(elevation) * np.sin(azimuth),
                             np.sin(elevation),
                             np.cos(elevation) * np.cos(azimuth)])
    c = np.asarray(center, np.float64) + off
    fwd = -off / np.linalg.norm(off)
    up = np.array([0.0, 1.0, 0.0])
    right = np.cross(up, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float64)
    t = -R @ c
    return pinhole_camera(width, height, focal_scale * width, R=R, t=t)


def uniform_box_scene(n: int, sh_degree: int, seed: int, width: int, height: int,
                      focal: float | None = None, with_target: bool = True) -> dict:
    """Means uniform in [-1,1]^3 shifted 4 units in front of an identity camera.

    log-scales N(-3.5, 0.5) per axis, uniform random rotations, opacity logits
    N(0, 1), SH DC N(0, 0.5) and higher orders N(0, 0.1); the target image is
    uniform in [0, 1]. This is the generator of the 4,096-Gaussian 128x128
    case and of the 3M-Gaussian scenes.
    """
    rng = _rng(seed)
    mean = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    mean[:, 2] += 4.0
    log_scale = rng.normal(-3.5, 0.5, (n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.0, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree, 0.5, 0.1)
    scene = {"mean": mean, "log_scale": log_scale, "quat": quat, "logit": logit,
             "sh": sh, "sh_degree": sh_degree}
    cam = pinhole_camera(width, height, float(width) if focal is None else focal)
    target = rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32) if with_target else None
    return {"scene": scene, "camera": cam, "target": target}


def interior_scene(n: int, sh_degree: int, seed: int, width: int, height: int,
                   half: float = 6.0) -> dict:
    """Means uniform in the cube [-half, half]^3 around an identity camera at
    the origin (a view from inside a large scene: about a tenth of it lies
    in the frustum). Log-scales N(-3.5 + ln(half), 0.5), so the ratio of
    Gaussian size to spacing matches the unit box of uniform_box_scene;
    rotations, opacities and SH as there; fx = fy = W."""
    rng = _rng(seed)
    mean = rng.uniform(-half, half, (n, 3)).astype(np.float32)
    log_scale = rng.normal(-3.5 + np.log(half), 0.5, (n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.0, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree, 0.5, 0.1)
    scene = {"mean": mean, "log_scale": log_scale, "quat": quat, "logit": logit,
             "sh": sh, "sh_degree": sh_degree}
    cam = pinhole_camera(width, height, float(width))
    target = rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)
    return {"scene": scene, "camera": cam, "target": target}


def surface_scene(n: int, sh_degree: int, seed: int, width: int, height: int,
                  n_planes: int = 32, n_spheres: int = 32, shell_fraction: float = 0.1,
                  shell_radius: float = 20.0, jitter: float = 0.01) -> dict:
    """Means on random planes and spheres plus a distant background shell.

    90% of the means lie on 32 square planes (centre U[-2,2]^3, random normal,
    side U(0.5, 2)) and 32 spheres (centre U[-2,2]^3, radius U(0.1, 0.8)),
    each surface picked with probability proportional to its area and points
    area-uniform on it, with N(0, jitter^2) isotropic jitter; 10% lie on a
    shell of radius 20. log-scales N(-4, 0.7), logits N(0, 1.5). The camera
    sits on a radius-4 orbit at 0.3 rad elevation looking at the origin,
    fx = fy = 0.78 W, with the azimuth drawn from the seed.
    """
    rng = _rng(seed)
    n_shell = int(round(n * shell_fraction))
    n_surf = n - n_shell
    # surfaces
    pc = rng.uniform(-2.0, 2.0, (n_planes, 3))
    pn = rng.standard_normal((n_planes, 3))
    pn /= np.linalg.norm(pn, axis=1, keepdims=True)
    side = rng.uniform(0.5, 2.0, n_planes)
    sc = rng.uniform(-2.0, 2.0, (n_spheres, 3))
    sr = rng.uniform(0.1, 0.8, n_spheres)
    area = np.concatenate([side ** 2, 4.0 * np.pi * sr ** 2])
    which = rng.choice(n_planes + n_spheres, size=n_surf, p=area / area.sum())
    pts = np.empty((n_surf, 3))
    is_plane = which < n_planes
    ip = which[is_plane]
    # in-plane basis from the normal
    a = np.where(np.abs(pn[:, 0:1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(pn, a)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(pn, e1)
    st = rng.uniform(-0.5, 0.5, (ip.size, 2)) * side[ip, None]
    pts[is_plane] = pc[ip] + st[:, :1] * e1[ip] + st[:, 1:] * e2[ip]
    isph = which[~is_plane] - n_planes
    d = rng.standard_normal((isph.size, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[~is_plane] = sc[isph] + sr[isph, None] * d
    pts += rng.normal(0.0, jitter, pts.shape)
    ds = rng.standard_normal((n_shell, 3))
    ds /= np.linalg.norm(ds, axis=1, keepdims=True)
    mean = np.concatenate([pts, shell_radius * ds]).astype(np.float32)
    log_scale = rng.normal(-4.0, 0.7, (n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.5, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree, 0.5, 0.1)
    scene = {"mean": mean, "log_scale": log_scale, "quat": quat, "logit": logit,
             "sh": sh, "sh_degree": sh_degree}
    azimuth = rng.uniform(0.0, 2.0 * np.pi)
    cam = orbit_camera(4.0, azimuth, 0.3, width, height)
    target = rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)
    return {"scene": scene, "camera": cam, "target": target}


def orbit_cameras(seed: int, resolutions, radius: float = 4.0,
                  elevation: float = 0.3, center=(0.0, 0.0, 0.0)) -> list:
    """Cameras on a seeded orbit, one per (width, height)."""
    rng = _rng(seed)
    az = rng.uniform(0.0, 2.0 * np.pi, len(resolutions))
    return [orbit_camera(radius, float(a), elevation, w, h, center=center)
            for a, (w, h) in zip(az, resolutions)]


BOX_CENTER = (0.0, 0.0, 4.0)  # centre of the uniform-box scenes


def render_requests(seed: int, duration_s: float, rate_hz: float, n_scenes: int,
                    resolutions, radius: float = 4.0, center=BOX_CENTER) -> list:
    """A seeded stream of render requests: Poisson arrivals at rate_hz over
    duration_s seconds, each with a uniform scene index, a uniform
    resolution from `resolutions` and an orbit camera (uniform azimuth,
    elevation uniform in [-0.4, 0.4] rad) around `center`."""
    rng = _rng(seed)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        sc = int(rng.integers(n_scenes))
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        az, el = rng.uniform(0.0, 2.0 * np.pi), rng.uniform(-0.4, 0.4)
        out.append({"arrival": t, "scene": sc, "camera": orbit_camera(radius, az, el, w, h,
                                                                       center=center)})


def random_splats(n: int, seed: int, width: int, height: int, max_radius: int = 40,
                  depth_ties: bool = True) -> dict:
    """Projected splats drawn directly, for testing binning and rasterisation alone.

    Returns float32 u, v, conic (A, B, C) of a positive-definite inverse
    covariance, depth, opacity, rgb and an int32 radius. With depth_ties a
    tenth of the depths repeat an earlier value exactly, so the tie rule of
    the sort is exercised.
    """
    rng = _rng(seed)
    u = rng.uniform(-0.1 * width, 1.1 * width, n).astype(np.float32)
    v = rng.uniform(-0.1 * height, 1.1 * height, n).astype(np.float32)
    sig = np.exp(rng.uniform(np.log(0.6), np.log(max_radius / 3.0), (n, 2)))
    th = rng.uniform(0.0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    # covariance = Rot diag(sig^2) Rot^T, inverse via the same rotation
    ia, ib = 1.0 / sig[:, 0] ** 2, 1.0 / sig[:, 1] ** 2
    A = c * c * ia + s * s * ib
    B = c * s * (ia - ib)
    C = s * s * ia + c * c * ib
    depth = rng.uniform(0.5, 10.0, n).astype(np.float32)
    if depth_ties and n > 10:
        k = n // 10
        src = rng.integers(0, n, k)
        dst = rng.integers(0, n, k)
        depth[dst] = depth[src]
    opacity = (1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, n)))).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    radius = np.ceil(3.0 * sig.max(axis=1)).astype(np.int32)
    return {"u": u, "v": v, "conic": np.stack([A, B, C], 1).astype(np.float32),
            "depth": depth, "opacity": opacity, "rgb": rgb, "radius": radius}


def random_image(seed: int, channels: int, height: int, width: int) -> np.ndarray:
    return _rng(seed).uniform(0.0, 1.0, (channels, height, width)).astype(np.float32)
