"""Pins of the oracle's preprocess, binning and forward rendering.

Closed forms (Eq. 1-2 for one and two splats, the EWA covariance of an
isotropic / axis-aligned / off-axis / rotated Gaussian), invariants of Eq. 1 (zero
opacity gives the background, weights plus final transmittance sum to one,
alpha never exceeds 0.99, T never drops below 1e-4) and a brute-force
per-tile enumeration of the binning.
"""
import numpy as np
import pytest

from paper_2503_01199_gb300 import scenegen

Y00 = 0.5 / np.sqrt(np.pi)  # textbook real SH of degree 0


def _one(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, rgb=(0.8, 0.5, 0.2)):
    sh = np.array([[(np.array(rgb) - 0.5) / Y00]])
    return {"mean": np.array([mean], np.float64), "log_scale": np.array([log_scale], np.float64),
            "quat": np.array([quat], np.float64), "logit": np.array([logit], np.float64),
            "sh": sh, "sh_degree": 0}


def _cat(*scenes):
    out = {k: np.concatenate([s[k] for s in scenes]) for k in ("mean", "log_scale", "quat", "logit", "sh")}
    out["sh_degree"] = 0
    return out


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def test_single_isotropic_gaussian_closed_form(orc):
    W = H = 64
    f = 64.0
    cam = scenegen.pinhole_camera(W, H, f, bg=(0.1, 0.2, 0.3))
    z, s = 3.0, 0.05
    q = np.random.default_rng(0).standard_normal(4)
    sc = _one([0.0, 0.0, z], [np.log(s)] * 3, quat=q, logit=0.7)
    r = orc.render_scene(sc, cam, (16, 16))
    sp = r["splats"]
    sig2 = (f * s / z) ** 2 + 0.3  # EWA: J = f/z I on the axis, plus the 0.3 low-pass
    np.testing.assert_allclose(sp["conic"][0], [1 / sig2, 0.0, 1 / sig2], rtol=1e-13, atol=1e-15)
    assert sp["radius"][0] == int(np.ceil(3 * np.sqrt(sig2)))
    np.testing.assert_allclose(sp["uv"][0], [W / 2, H / 2])
    np.testing.assert_allclose(sp["depth"][0], z)
    # Eq. 1 with one splat: I = c a + (1 - a) bg, a = min(0.99, o G)
    o = _sigmoid(0.7)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    G = np.exp(-((px - W / 2) ** 2 + (py - H / 2) ** 2) / (2 * sig2))
    a = np.minimum(0.99, o * G)
    rad = sp["radius"][0]
    x0, x1 = int(np.floor((W / 2 - rad) / 16)), int(np.floor((W / 2 + rad) / 16)) + 1
    inrect = (px // 16 >= x0) & (px // 16 < x1) & (py // 16 >= x0) & (py // 16 < x1)
    keep = (a >= 1 / 255) & inrect
    a = np.where(keep, a, 0.0)
    rgb = np.array([0.8, 0.5, 0.2])
    bg = np.array([0.1, 0.2, 0.3])
    expect = rgb[:, None, None] * a + (1 - a) * bg[:, None, None]
    np.testing.assert_allclose(r["image"], expect, atol=1e-14)
    np.testing.assert_allclose(r["T"], 1 - a, atol=1e-14)
    np.testing.assert_array_equal(r["last"], keep.astype(np.int32))


def test_axis_aligned_and_off_axis_covariance(orc):
    W, H, f = 128, 96, 100.0
    cam = scenegen.pinhole_camera(W, H, f)
    sx, sy, sz = 0.02, 0.05, 0.3
    # on the axis, identity rotation: diag((f sx/z)^2, (f sy/z)^2) + 0.3
    z = 4.0
    sp = orc.preprocess(_one([0, 0, z], np.log([sx, sy, sz])), cam)
    a, c = (f * sx / z) ** 2 + 0.3, (f * sy / z) ** 2 + 0.3
    np.testing.assert_allclose(sp["conic"][0], [1 / a, 0, 1 / c], rtol=1e-13, atol=1e-16)
    # off axis at (x, 0, z): row 0 of J is (f/z, 0, -f x / z^2), so the
    # depth extent leaks into the screen x variance
    x = 0.5
    sp = orc.preprocess(_one([x, 0, z], np.log([sx, sy, sz])), cam)
    a = (f / z) ** 2 * sx ** 2 + (f * x / z ** 2) ** 2 * sz ** 2 + 0.3
    c = (f / z) ** 2 * sy ** 2 + 0.3
    np.testing.assert_allclose(sp["conic"][0], [1 / a, 0, 1 / c], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(sp["uv"][0], [f * x / z + W / 2, H / 2], rtol=1e-14)
    # a 90-degree rotation about z swaps the screen axes
    q = [np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)]
    sp = orc.preprocess(_one([0, 0, z], np.log([sx, sy, sz]), quat=q), cam)
    a, c = (f * sy / z) ** 2 + 0.3, (f * sx / z) ** 2 + 0.3
    np.testing.assert_allclose(sp["conic"][0], [1 / a, 0, 1 / c], rtol=1e-12, atol=1e-12)


def test_near_plane_and_offscreen_cull(orc):
    cam = scenegen.pinhole_camera(64, 64, 64.0)
    sc = _cat(_one([0, 0, 0.1], [-3] * 3), _one([0, 0, -2], [-3] * 3), _one([50, 0, 3], [-3] * 3),
              _one([0, 0, 3], [-3] * 3))
    sp = orc.preprocess(sc, cam)
    np.testing.assert_array_equal(sp["radius"] > 0, [False, False, False, True])


def test_two_splats_over_operator_and_order_invariance(orc):
    W = H = 32
    cam = scenegen.pinhole_camera(W, H, 32.0, bg=(0.0, 0.0, 0.0))
    front = _one([0, 0, 2.0], [np.log(0.1)] * 3, logit=0.3, rgb=(1.0, 0.0, 0.0))
    back = _one([0, 0, 3.0], [np.log(0.15)] * 3, logit=-0.2, rgb=(0.0, 0.0, 1.0))
    r1 = orc.render_scene(_cat(front, back), cam)
    r2 = orc.render_scene(_cat(back, front), cam)
    np.testing.assert_array_equal(r1["image"], r2["image"])
    sp = r1["splats"]
    px = py = W / 2 + 0.5  # pixel (16, 16)
    al = []
    for j in range(2):
        dx, dy = sp["uv"][j, 0] - px, sp["uv"][j, 1] - py
        A, B, C = sp["conic"][j]
        al.append(min(0.99, sp["opacity"][j] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)))
    expect = np.array([1, 0, 0]) * al[0] + np.array([0, 0, 1]) * al[1] * (1 - al[0])
    np.testing.assert_allclose(r1["image"][:, 16, 16], expect, atol=1e-15)
    np.testing.assert_allclose(r1["T"][16, 16], (1 - al[0]) * (1 - al[1]), atol=1e-15)


def test_zero_opacity_gives_background(orc):
    d = scenegen.uniform_box_scene(512, 1, 5, 64, 64, focal=64.0)
    sc, cam = d["scene"], dict(d["camera"], bg=np.array([0.1, 0.2, 0.3], np.float32))
    sc = dict(sc, logit=np.full_like(sc["logit"], -30.0))
    r = orc.render_scene(sc, cam)
    bg = np.array([0.1, 0.2, 0.3], np.float32).astype(np.float64)
    np.testing.assert_array_equal(r["image"], np.broadcast_to(bg[:, None, None], r["image"].shape))
    assert (r["last"] == 0).all()


def test_weights_sum_with_final_transmittance(orc):
    d = scenegen.uniform_box_scene(2048, 0, 6, 64, 64, focal=64.0)
    sc = dict(d["scene"])
    sc["sh"] = np.full_like(sc["sh"], 0.5 / Y00)  # every colour = 1
    sc["log_scale"] = sc["log_scale"] + 1.0
    r = orc.render_scene(sc, d["camera"])
    # bg = 0 and c = 1:  I = sum_k a_k T_k = 1 - T_final
    np.testing.assert_allclose(r["image"][0] + r["T"], 1.0, atol=1e-13)
    assert r["T"].min() >= 1e-4
    assert (r["last"] > 0).mean() > 0.5


def test_opaque_splat_is_clamped(orc):
    cam = scenegen.pinhole_camera(32, 32, 32.0, bg=(0.5, 0.5, 0.5))
    # sigma^2 = (32 * 0.5 / 2)^2 + 0.3; the pixel centre 0.5 px off the mean on
    # both axes has G = exp(-0.5 / (2 sigma^2)) > 0.996, so o G > 0.99 clamps
    sc = _one([0, 0, 2.0], [np.log(0.5)] * 3, logit=40.0, rgb=(0.9, 0.1, 0.3))
    r = orc.render_scene(sc, cam)
    expect = 0.99 * np.array([0.9, 0.1, 0.3]) + 0.01 * 0.5
    np.testing.assert_allclose(r["image"][:, 16, 16], expect, rtol=1e-6)
    assert r["image"].max() <= 0.99 * 0.9 + 0.01 * 0.5 + 1e-15


def test_stop_rule_excludes_the_crossing_splat(orc):
    # 3 identical opaque splats stacked: after two, T = 1e-4 exactly would be
    # crossed by the third, which must then not be composited.
    cam = scenegen.pinhole_camera(16, 16, 16.0)
    # scale 1 at z ~ 2 with f = 16: sigma^2 ~ 64, so o G > 0.99 at pixel (8, 8)
    sc = _cat(*[_one([0, 0, 2.0 + 0.1 * k], [0.0] * 3, logit=40.0, rgb=(1, 1, 1)) for k in range(3)])
    r = orc.render_scene(sc, cam, (16, 16))
    # centre pixel: a = 0.99, T after two = 1e-4 (not < 1e-4): composited;
    # the third would give 1e-6 < 1e-4: stop without it.
    c = r["image"][0, 8, 8]
    assert r["last"][8, 8] == 2
    np.testing.assert_allclose(c, 0.99 + 0.99 * 0.01, rtol=1e-6)
    assert r["T"][8, 8] >= 1e-4


def _rect_f32(u, v, r, tw, th, gx, gy):
    u, v, r = np.float32(u), np.float32(v), np.float32(r)
    x0 = np.floor((u - r) / np.float32(tw)); x1 = np.floor((u + r) / np.float32(tw)) + np.float32(1)
    y0 = np.floor((v - r) / np.float32(th)); y1 = np.floor((v + r) / np.float32(th)) + np.float32(1)
    cl = lambda a, g: int(min(max(a, 0), g))
    return cl(x0, gx), cl(y0, gy), cl(x1, gx), cl(y1, gy)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_binning_matches_brute_force(orc, tile):
    W, H = 100, 70
    s = scenegen.random_splats(400, 3, W, H, max_radius=25)
    s["radius"][::17] = 0  # culled splats
    vals, ranges, P = orc.bin_splats(s["u"], s["v"], s["radius"], s["depth"], W, H, tile)
    gx, gy = (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]
    rects = [_rect_f32(s["u"][i], s["v"][i], s["radius"][i], tile[0], tile[1], gx, gy)
             for i in range(400)]
    total = 0
    for t in range(gx * gy):
        tx, ty = t % gx, t // gx
        members = [i for i in range(400) if s["radius"][i] > 0 and rects[i][0] <= tx < rects[i][2]
                   and rects[i][1] <= ty < rects[i][3]]
        members.sort(key=lambda i: (float(s["depth"][i]), i))  # depth, then index (stable)
        a, b = ranges[t]
        assert list(vals[a:b]) == members
        total += len(members)
    assert total == P


def _tau(opacity):
    t = 2.0 * np.log(255.0 * np.asarray(opacity, np.float64))
    return np.where(t > -1e30, t + 1e-3 * (1.0 + np.abs(t)), -np.inf).astype(np.float32)


def test_tile_culling_keeps_every_contributing_pair(orc):
    # App. A.1 tile-level culling: a tile is dropped only if no pixel centre
    # in it can reach alpha >= 1/255. Brute force over every pixel centre of
    # every tile of every rectangle, in double precision.
    W, H, tw = 96, 80, 16
    s = scenegen.random_splats(300, 9, W, H, max_radius=30)
    tau = _tau(s["opacity"])
    full = orc.bin_splats(s["u"], s["v"], s["radius"], s["depth"], W, H)
    cull = orc.bin_splats(s["u"], s["v"], s["radius"], s["depth"], W, H, conic=s["conic"], tau=tau)
    gx, gy = W // tw, H // tw
    listed = set()
    for t in range(gx * gy):
        for j in cull[0][cull[1][t, 0]:cull[1][t, 1]]:
            listed.add((int(j), t))
    pairs_full = {(int(j), t) for t in range(gx * gy) for j in full[0][full[1][t, 0]:full[1][t, 1]]}
    assert listed <= pairs_full
    A, B, C = (s["conic"][:, k].astype(np.float64) for k in range(3))
    for (j, t) in pairs_full:
        tx, ty = t % gx, t // gx
        px, py = np.meshgrid(tx * tw + np.arange(tw) + 0.5, ty * tw + np.arange(tw) + 0.5)
        dx, dy = float(s["u"][j]) - px, float(s["v"][j]) - py
        a = float(s["opacity"][j]) * np.exp(-0.5 * (A[j] * dx * dx + C[j] * dy * dy) - B[j] * dx * dy)
        if (a >= 1.0 / 255.0).any():
            assert (j, t) in listed, (j, t)
    assert len(listed) < 0.9 * len(pairs_full)   # the rectangles over-cover


def test_tile_culling_leaves_the_image_unchanged(orc):
    d = scenegen.uniform_box_scene(3000, 1, 13, 96, 96, focal=96.0)
    a = orc.render_scene(d["scene"], d["camera"], cull=False)
    b = orc.render_scene(d["scene"], d["camera"], cull=True)
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["T"], b["T"])
    assert b["P"] < a["P"]


def _tile_queries(n, seed, W=400, H=300, max_radius=60, reach=3):
    rng = np.random.default_rng(seed)
    sp = scenegen.random_splats(n, seed + 1, W, H, max_radius=max_radius)
    tau = _tau(sp["opacity"]).astype(np.float32)
    tx = (np.floor(sp["u"] / 16) + rng.integers(-reach, reach + 1, n)).astype(np.int32)
    ty = (np.floor(sp["v"] / 16) + rng.integers(-reach, reach + 1, n)).astype(np.int32)
    return sp, tau, tx, ty


def test_tile_culling_axis_aligned_closed_form(orc):
    """App. A.1's tile test for an axis-aligned conic (B = 0): the minimum of
    A dx^2 + C dy^2 over the box of pixel centres is A ex^2 + C ey^2, ex and
    ey the distances from the splat centre to the box's x and y ranges (0
    inside). Swapping A and C, or measuring to the far edge, fails it."""
    n = 100000
    sp, tau, tx, ty = _tile_queries(n, 60)
    conic = sp["conic"].copy()
    conic[:, 1] = 0.0
    u, v = sp["u"].astype(np.float64), sp["v"].astype(np.float64)
    A, C = conic[:, 0].astype(np.float64), conic[:, 2].astype(np.float64)
    xl, xh = tx * 16 + 0.5, tx * 16 + 15.5
    yl, yh = ty * 16 + 0.5, ty * 16 + 15.5
    ex = np.maximum(np.maximum(xl - u, u - xh), 0.0)
    ey = np.maximum(np.maximum(yl - v, v - yh), 0.0)
    qmin = A * ex * ex + C * ey * ey
    got, near = orc.tile_reachable(sp["u"], sp["v"], conic, tau, tx, ty)
    t = tau.astype(np.float64)
    np.testing.assert_array_equal(got[~near], (qmin <= t)[~near])
    assert near.mean() < 1e-3 and 0.05 < got.mean() < 0.95
    swapped = C * ex * ex + A * ey * ey
    assert ((swapped <= t) != got).sum() > 100


def test_tile_culling_rotated_conic_against_a_numerical_minimum(orc):
    """For rotated conics the box minimum is found independently: zero when a
    positive-definite form's box holds the centre, else the least of a
    bounded scalar minimisation (scipy) along each of the four edges."""
    from scipy.optimize import minimize_scalar
    n = 1500
    sp, tau, tx, ty = _tile_queries(n, 61, reach=2)
    got, near = orc.tile_reachable(sp["u"], sp["v"], sp["conic"], tau, tx, ty)
    agree = 0
    for i in range(n):
        A, B, C = (float(c) for c in sp["conic"][i])
        u, v = float(sp["u"][i]), float(sp["v"][i])
        xl, xh = tx[i] * 16 + 0.5, tx[i] * 16 + 15.5
        yl, yh = ty[i] * 16 + 0.5, ty[i] * 16 + 15.5
        q = lambda x, y: A * (u - x) ** 2 + 2 * B * (u - x) * (v - y) + C * (v - y) ** 2
        if xl <= u <= xh and yl <= v <= yh:
            best = 0.0
        else:
            best = np.inf
            for f, lo, hi in ((lambda y: q(xl, y), yl, yh), (lambda y: q(xh, y), yl, yh),
                              (lambda x: q(x, yl), xl, xh), (lambda x: q(x, yh), xl, xh)):
                r = minimize_scalar(f, bounds=(lo, hi), method="bounded",
                                    options={"xatol": 1e-10})
                best = min(best, r.fun, f(lo), f(hi))
        t = float(tau[i])
        if abs(best - t) > 1e-6 * (1 + abs(t)):
            assert got[i] == (best <= t), (i, best, t)
            agree += 1
    assert agree > 0.99 * n and 0.1 < got.mean() < 0.9


def _row_form_f32(u, v, A, B, C, tau, tx, ty, tw=16, th=16):
    """A single-precision evaluation of the same test in its row form (per
    tile row the x interval [L, U] of the ellipse q <= tau, then the tile's
    offsets against it; a conic whose determinant rounds to <= 0 takes the
    edge minima), each operation rounded once, as a kernel evaluates it."""
    f32 = np.float32
    u, v, A, B, C, tau = (np.asarray(a, f32) for a in (u, v, A, B, C, tau))
    with np.errstate(all="ignore"):
        det = A * C - B * B
        ex, ey = np.sqrt((tau * C) / det), np.sqrt((tau * A) / det)
        dyU = -((B * ex) / C)
        yl, yh = (ty * th).astype(f32) + f32(0.5), (ty * th + th).astype(f32) + f32(-0.5)
        xl, xh = (tx * tw).astype(f32) + f32(0.5), (tx * tw + tw).astype(f32) + f32(-0.5)
        ay, by = v - yh, v - yl
        At = A * tau
        d = np.minimum(np.maximum(dyU, ay), by)
        Uu = (np.sqrt(np.maximum(At - det * (d * d), f32(0))) - B * d) / A
        d = np.minimum(np.maximum(-dyU, ay), by)
        L = (-(np.sqrt(np.maximum(At - det * (d * d), f32(0))) + B * d)) / A
        row = (tau >= 0) & (ay <= ey) & (by >= -ey) & ((u - xh) <= Uu) & ((u - xl) >= L)
        ax, bx = u - xh, u - xl
        inside = (ax <= 0) & (bx >= 0) & (ay <= 0) & (by >= 0)
        rA, rC = f32(1) / A, f32(1) / C
        qf = lambda dx, dy: ((A * dx) * dx + ((B * dx) * dy) * f32(2)) + (C * dy) * dy
        q = qf(ax, np.minimum(np.maximum(-((B * ax) * rC), ay), by))
        q = np.minimum(q, qf(bx, np.minimum(np.maximum(-((B * bx) * rC), ay), by)))
        q = np.minimum(q, qf(np.minimum(np.maximum(-((B * ay) * rA), ax), bx), ay))
        q = np.minimum(q, qf(np.minimum(np.maximum(-((B * by) * rA), ax), bx), by))
        box = (inside & (tau >= 0)) | (q <= tau)
    return np.where(det > 0, row, box)


@pytest.mark.parametrize("case", ["plain", "large", "degenerate"])
def test_tile_culling_single_precision_agrees_off_the_flags(orc, case):
    """The oracle's near-tau flag covers single-precision evaluation: a row
    form evaluated with one rounding per operation takes the oracle's
    decision on every unflagged pair, including thin ellipses (axis ratio up
    to ~1000) and conics whose determinant is 0 or negative."""
    n = 300000
    sp, tau, tx, ty = _tile_queries(n, 70 + len(case), W=1297, H=840,
                                    max_radius=600 if case != "plain" else 40, reach=4)
    conic = sp["conic"].astype(np.float64)
    if case == "degenerate":
        A, C = conic[:, 0], conic[:, 2]
        conic[::7, 1] = np.sqrt(A[::7] * C[::7])
        conic[3::11, 1] = 1.5 * np.sqrt(A[3::11] * C[3::11])
        conic[5::13, 0] *= 1e3
    conic = conic.astype(np.float32)
    got, near = orc.tile_reachable(sp["u"], sp["v"], conic, tau, tx, ty)
    emu = _row_form_f32(sp["u"], sp["v"], conic[:, 0], conic[:, 1], conic[:, 2], tau, tx, ty)
    np.testing.assert_array_equal(emu[~near], got[~near])
    assert near.mean() < 1e-3 and 0.02 < got.mean() < 0.98


def _edge_min(u, v, A, B, C, tx, ty):
    """Box minimum by the clamped stationary point of each edge (convex
    edges: A, C > 0), 0 when the box holds the centre; numpy, double."""
    xl, xh, yl, yh = tx * 16 + 0.5, tx * 16 + 15.5, ty * 16 + 0.5, ty * 16 + 15.5
    ax, bx, ay, by = u - xh, u - xl, v - yh, v - yl
    q = lambda dx, dy: A * dx * dx + 2 * B * dx * dy + C * dy * dy
    best = np.full(u.shape, np.inf)
    for dx in (ax, bx):
        best = np.minimum(best, q(dx, np.clip(-B * dx / C, ay, by)))
    for dy in (ay, by):
        best = np.minimum(best, q(np.clip(-B * dy / A, ax, bx), dy))
    return np.where((ax <= 0) & (bx >= 0) & (ay <= 0) & (by >= 0), 0.0, best)


@pytest.mark.parametrize("seed,max_radius", [(1, 40), (2, 200), (3, 600)])
def test_tile_culling_flag_covers_the_boundary(orc, seed, max_radius):
    """Stress of the near-tau flag where it matters: tau placed within a
    relative 3e-6 of each pair's exact box minimum, so that a few percent of
    single-precision decisions differ from the exact ones. Every such
    difference is flagged, and it still is with the margin cut 64-fold."""
    n = 300000
    rng = np.random.default_rng(seed)
    sp = scenegen.random_splats(n, seed, 1297, 840, max_radius=max_radius)
    tx = (np.floor(sp["u"] / 16) + rng.integers(-4, 5, n)).astype(np.int32)
    ty = (np.floor(sp["v"] / 16) + rng.integers(-4, 5, n)).astype(np.int32)
    A, B, C = (sp["conic"][:, k].astype(np.float64) for k in range(3))
    qm = _edge_min(sp["u"].astype(np.float64), sp["v"].astype(np.float64), A, B, C, tx, ty)
    border = (qm > 0.5) & (qm < 30)
    tau = (qm * (1 + rng.uniform(-3e-6, 3e-6, n))).astype(np.float32)
    emu = _row_form_f32(sp["u"], sp["v"], sp["conic"][:, 0], sp["conic"][:, 1], sp["conic"][:, 2],
                        tau, tx, ty)
    for m in (orc.TAU_MARGIN, orc.TAU_MARGIN / 64):
        orc.set_tau_margin(m)
        try:
            got, near = orc.tile_reachable(sp["u"], sp["v"], sp["conic"], tau, tx, ty)
        finally:
            orc.set_tau_margin(orc.TAU_MARGIN)
        differ = (emu != got) & border
        assert differ.sum() > 0.01 * border.sum()
        assert near[differ].all()


def test_tile_culling_near_pairs_enumerated(orc):
    """tile_near_pairs lists exactly the rectangle pairs that tile_reachable
    flags (with the flag widened so that many exist)."""
    W, H = 300, 200
    s = scenegen.random_splats(3000, 90, W, H, max_radius=40)
    tau = _tau(s["opacity"]).astype(np.float32)
    orc.set_tau_margin(1e-3)
    try:
        keys = orc.tile_near_pairs(s["u"], s["v"], s["radius"], s["conic"], tau, W, H)
        full, ranges, P = orc.bin_splats(s["u"], s["v"], s["radius"], s["depth"], W, H)
        gx = -(-W // 16)
        tiles = np.repeat(np.arange(ranges.shape[0]), (ranges[:, 1] - ranges[:, 0]).astype(np.int64))
        j = full[np.concatenate([np.arange(a, b) for a, b in ranges.astype(np.int64)])]
        _, near = orc.tile_reachable(s["u"][j], s["v"][j], s["conic"][j], tau[j], tiles % gx, tiles // gx)
    finally:
        orc.set_tau_margin(orc.TAU_MARGIN)
    want = np.sort((tiles[near].astype(np.uint64) << np.uint64(32)) | j[near].astype(np.uint64))
    np.testing.assert_array_equal(np.sort(keys), want)
    assert 10 < keys.size < 0.1 * P


def test_tile_culling_near_pairs_hold_no_fragment(orc):
    """At the default margin and for splats up to 60 px, no near-tau pair
    holds a pixel centre with alpha >= 1/255 (tau is widened by
    1e-3 (1 + |tau|) beyond that threshold, more than the flag's margin on
    such offsets), so whichever way a kernel decides them, no pixel changes.
    Brute force over each pair's tile. (For much larger splats the margin,
    64 roundings of the offsets, can exceed the widening; the GPU tests then
    check the pairs that the two binnings actually decide differently.)"""
    W, H = 1297, 840
    s = scenegen.random_splats(200000, 91, W, H, max_radius=60)
    tau = _tau(s["opacity"]).astype(np.float32)
    keys = orc.tile_near_pairs(s["u"], s["v"], s["radius"], s["conic"], tau, W, H)
    assert keys.size > 5
    gx = -(-W // 16)
    for key in keys.tolist():
        t, i = key >> 32, key & 0xffffffff
        px, py = np.meshgrid((t % gx) * 16 + np.arange(16) + 0.5, (t // gx) * 16 + np.arange(16) + 0.5)
        A, B, C = (float(c) for c in s["conic"][i])
        dx, dy = float(s["u"][i]) - px, float(s["v"][i]) - py
        a = float(s["opacity"][i]) * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
        assert (a < 1 / 255).all()


def test_rotated_splat_off_diagonal_conic_and_image(orc):
    """The off-diagonal term, which the axis-aligned pins leave at zero: a
    splat on the axis turned by 30 degrees about the view direction. On the
    axis the EWA Jacobian is (f/z) I, so the screen covariance is
    R2 diag(sx^2, sy^2) R2^T (f/z)^2 + 0.3 I; the conic (a, b, c) is its
    inverse, the radius that of the unrotated splat (same eigenvalues), and
    the image follows G = exp(-0.5 (a dx^2 + 2 b dx dy + c dy^2)) as the
    scanline formulation of App. A writes it."""
    W = H = 64
    f, z, sx, sy, th = 64.0, 3.0, 0.12, 0.04, np.pi / 6
    cam = scenegen.pinhole_camera(W, H, f, bg=(0.1, 0.2, 0.3))
    q = [np.cos(th / 2), 0.0, 0.0, np.sin(th / 2)]
    sc = _one([0.0, 0.0, z], np.log([sx, sy, 0.2]), quat=q, logit=1.3)
    r = orc.render_scene(sc, cam, (16, 16))
    sp = r["splats"]
    R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    S2 = (f / z) ** 2 * R2 @ np.diag([sx ** 2, sy ** 2]) @ R2.T + 0.3 * np.eye(2)
    det = S2[0, 0] * S2[1, 1] - S2[0, 1] ** 2
    a, b, c = S2[1, 1] / det, -S2[0, 1] / det, S2[0, 0] / det
    assert abs(b) > 0.1 * max(a, c)
    np.testing.assert_allclose(sp["conic"][0], [a, b, c], rtol=1e-12, atol=1e-15)
    lam = max((f * sx / z) ** 2, (f * sy / z) ** 2) + 0.3
    assert sp["radius"][0] == int(np.ceil(3 * np.sqrt(lam)))
    o = _sigmoid(1.3)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dx, dy = px - W / 2, py - H / 2
    rad = sp["radius"][0]
    t0, t1 = int(np.floor((W / 2 - rad) / 16)), int(np.floor((W / 2 + rad) / 16)) + 1
    inrect = (px // 16 >= t0) & (px // 16 < t1) & (py // 16 >= t0) & (py // 16 < t1)
    rgb = np.array([0.8, 0.5, 0.2])
    bg = np.array([0.1, 0.2, 0.3])

    def image(bb):
        G = np.exp(-0.5 * (a * dx ** 2 + 2 * bb * dx * dy + c * dy ** 2))
        al = np.minimum(0.99, o * G)
        al = np.where((al >= 1 / 255) & inrect, al, 0.0)
        return rgb[:, None, None] * al + (1 - al) * bg[:, None, None]

    np.testing.assert_allclose(r["image"], image(b), atol=1e-13)
    # the pin tells the orientation apart: the mirrored ellipse is far off
    assert np.abs(r["image"] - image(-b)).max() > 0.1


def test_covariance_in_a_turned_camera(orc):
    """Sec. 3's world covariance R(q) S S^T R(q)^T, q normalised first, seen by
    a camera whose rotation is the inverse of R(q): in camera coordinates the
    Gaussian is axis-aligned again, so on the optical axis its conic is the
    axis-aligned closed form. Taking the camera rotation transposed, or the
    quaternion conjugated, turns it by twice the angle instead; scaling q by
    3.7 changes nothing."""
    W, H, f, z = 96, 96, 80.0, 3.0
    sx, sy, sz = 0.09, 0.03, 0.2
    ph = 0.6
    Rc = np.array([[np.cos(ph), 0.0, -np.sin(ph)], [0.0, 1.0, 0.0], [np.sin(ph), 0.0, np.cos(ph)]])
    centre = np.array([0.2, 0.1, -1.5])
    cam = scenegen.pinhole_camera(W, H, f, R=Rc, t=-Rc @ centre)
    R32 = np.asarray(cam["R"], np.float64)
    mean = -R32.T @ np.asarray(cam["t"], np.float64) + R32.T @ np.array([0.0, 0.0, z])
    a = (f * sx / z) ** 2 + 0.3
    c = (f * sy / z) ** 2 + 0.3
    q = np.array([np.cos(ph / 2), 0.0, np.sin(ph / 2), 0.0])  # R(q) = Rc^T: a turn about y
    for scale in (1.0, 3.7):
        sp = orc.preprocess(_one(mean, np.log([sx, sy, sz]), quat=scale * q), cam)
        np.testing.assert_allclose(sp["uv"][0], [W / 2, H / 2], atol=1e-5)
        np.testing.assert_allclose(sp["conic"][0], [1 / a, 0.0, 1 / c], rtol=2e-6, atol=2e-7)
    # the Gaussian turned the other way is not axis-aligned in this camera
    sp = orc.preprocess(_one(mean, np.log([sx, sy, sz]), quat=q * [1, -1, -1, -1]), cam)
    assert abs(sp["conic"][0][0] - 1 / a) > 0.05 / a


def test_jacobian_clamp_beyond_the_field_of_view(orc):
    """The EWA Jacobian is taken at the centre with x/z clamped to
    +-1.3 W / (2 fx) (the 3DGS rule the paper's projection inherits), while
    the splat's screen position uses the unclamped centre. A splat at
    x/z = 1 with the limit at 0.832 (principal point moved to x = 0 so that
    it stays on screen): the conic's a takes the clamped x, u the true one."""
    W, H, f = 128, 96, 100.0
    cam = scenegen.pinhole_camera(W, H, f)
    cam["cx"] = 0.0
    z, x = 4.0, 4.0
    sx, sy, sz = 0.02, 0.03, 0.3
    sp = orc.preprocess(_one([x, 0.0, z], np.log([sx, sy, sz])), cam)
    lim = 1.3 * W / (2 * f)
    assert x / z > lim and sp["radius"][0] > 0
    a = (f * sx / z) ** 2 + (f * lim / z) ** 2 * sz ** 2 + 0.3
    c = (f * sy / z) ** 2 + 0.3
    np.testing.assert_allclose(sp["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(sp["uv"][0], [f * x / z, H / 2], rtol=1e-14)
    unclamped = (f * sx / z) ** 2 + (f * x / z ** 2) ** 2 * sz ** 2 + 0.3
    assert abs(1 / unclamped - sp["conic"][0][0]) > 0.1 / a


def test_radius_is_three_sigma_of_the_larger_eigenvalue(orc):
    """r = ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 - det))
    with m the mean of the 2D covariance's diagonal (the 3DGS rule the
    projection inherits). Axis-aligned, the eigenvalues are the diagonal
    itself; isotropic, the 0.1 floor lifts lambda_max by sqrt(0.1), which
    at a variance of 3.9 px^2 makes the radius 7 instead of 6."""
    W, H, f, z = 64, 64, 64.0, 3.0
    cam = scenegen.pinhole_camera(W, H, f)
    s_iso = np.sqrt(3.6) * z / f                           # (f s / z)^2 = 3.6, +0.3 = 3.9
    sp = orc.preprocess(_one([0.0, 0.0, z], [np.log(s_iso)] * 3), cam)
    np.testing.assert_allclose(1 / sp["conic"][0][0], 3.9, rtol=1e-12)
    assert int(np.ceil(3 * np.sqrt(3.9))) == 6
    assert sp["radius"][0] == int(np.ceil(3 * np.sqrt(3.9 + np.sqrt(0.1)))) == 7
    # axis-aligned, variances 9.3 and 1.3: the larger one, exactly
    sx, sy = 3.0 * z / f, 1.0 * z / f
    sp = orc.preprocess(_one([0.0, 0.0, z], np.log([sx, sy, 0.1])), cam)
    np.testing.assert_allclose(sp["conic"][0], [1 / 9.3, 0.0, 1 / 1.3], rtol=1e-12, atol=1e-16)
    assert sp["radius"][0] == int(np.ceil(3 * np.sqrt(9.3))) == 10
