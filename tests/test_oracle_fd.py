"""Finite-difference pins of the oracle's analytic backward.

Central differences in double precision. The loss is linear in the image,
L = sum_p w_p . I_p (for the end-to-end case w = dL/dI of the L1 loss at the
base point), so the difference is taken per pixel and the only error terms are
truncation O(h^2) and rounding O(eps |I| / h). A parameter whose +-h step
changes any discrete decision (which fragments are included, where a pixel
stops, a clamp, a tile rectangle, the sign of I - gt) is skipped and counted.
"""
import numpy as np

from paper_2503_01199_gb300 import scenegen

RTOL = 1e-6


def _check(an, fd, floor):
    """|fd - an| <= RTOL * max(|an|, floor)."""
    err = np.abs(fd - an)
    bound = RTOL * np.maximum(np.abs(an), floor)
    return err <= bound, err / np.maximum(np.abs(an), floor)


def _small_splat_scene(seed=0, W=48, H=40):
    d = scenegen.uniform_box_scene(300, 3, seed, W, H, focal=48.0)
    return d


def test_raster_backward_matches_fd(orc):
    d = _small_splat_scene()
    cam, tile = d["camera"], (16, 16)
    cam = dict(cam, bg=np.array([0.2, 0.1, 0.3], np.float32))
    base = orc.render_scene(d["scene"], cam, tile)
    sp = {k: base["splats"][k].copy() for k in ("uv", "conic", "opacity", "rgb", "depth")}
    vals, ranges = base["vals"], base["ranges"]
    w = np.random.default_rng(1).standard_normal(base["image"].shape)
    bw = orc.render_bwd(sp, vals, ranges, cam, w, tile)
    vis = np.flatnonzero(base["splats"]["radius"] > 0)
    pick = np.random.default_rng(2).choice(vis, 40, replace=False)
    h0 = orc.render_fwd(sp, vals, ranges, cam, tile)["hash"]
    # parameter k of splat j -> (array, index)
    slots = [("uv", 0), ("uv", 1), ("conic", 0), ("conic", 1), ("conic", 2), ("opacity", None),
             ("rgb", 0), ("rgb", 1), ("rgb", 2)]
    ok = skipped = 0
    scale = np.sqrt(np.mean(bw["grad9"][vis] ** 2, axis=0))
    for j in pick:
        for q, (name, c) in enumerate(slots):
            arr = sp[name]
            ref = (j, c) if c is not None else (j,)
            x0 = arr[ref]
            h = 1e-6 * max(1.0, abs(x0))
            arr[ref] = x0 + h
            fp = orc.render_fwd(sp, vals, ranges, cam, tile)
            arr[ref] = x0 - h
            fm = orc.render_fwd(sp, vals, ranges, cam, tile)
            arr[ref] = x0
            if fp["hash"] != h0 or fm["hash"] != h0:
                skipped += 1
                continue
            fd = np.sum(w * (fp["image"] - fm["image"])) / (2 * h)
            good, rel = _check(bw["grad9"][j, q], fd, 1e-3 * scale[q])
            assert good, (j, name, c, bw["grad9"][j, q], fd, rel)
            ok += 1
    assert ok > 300 and skipped < 0.1 * (ok + skipped)


def test_opacity_moments_single_splat_closed_form(orc):
    # one splat: I = c a + (1 - a) bg, so dI/da = c - bg and per pixel
    # g = dL/do = G sum_ch w_ch (c_ch - bg_ch) (unclamped). S, M, C are the
    # sum of g^2, the sum of g and the number of included pixels.
    W = H = 48
    cam = scenegen.pinhole_camera(W, H, 48.0, bg=(0.1, 0.2, 0.3))
    Y00 = 0.5 / np.sqrt(np.pi)
    rgb = np.array([0.7, 0.4, 0.9])
    sc = {"mean": np.array([[0.05, -0.03, 2.5]]), "log_scale": np.array([[-2.2, -2.6, -2.0]]),
          "quat": np.array([[0.9, 0.1, -0.3, 0.2]]), "logit": np.array([0.4]),
          "sh": ((rgb - 0.5) / Y00)[None, None, :], "sh_degree": 0}
    r = orc.render_scene(sc, cam)
    w = np.random.default_rng(3).standard_normal((3, H, W))
    bw = orc.render_bwd(r["splats"], r["vals"], r["ranges"], cam, w)
    sp = r["splats"]
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dx, dy = sp["uv"][0, 0] - px, sp["uv"][0, 1] - py
    A, B, C = sp["conic"][0]
    G = np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
    a = np.minimum(0.99, sp["opacity"][0] * G)
    inc = (a >= 1 / 255) & (r["last"] == 1)
    assert inc.sum() > 20 and (sp["opacity"][0] * G < 0.99).all()
    bg = np.asarray(cam["bg"], np.float64)  # stored as float32 by the generator
    g = G * np.einsum("chw,c->hw", w, sp["rgb"][0] - bg)
    g = g[inc]
    assert bw["C"][0] == inc.sum()
    np.testing.assert_allclose(bw["M"][0], g.sum(), rtol=1e-12)
    np.testing.assert_allclose(bw["S"][0], (g * g).sum(), rtol=1e-12)
    # C Var = S - M^2 / C equals the centred sum of squares
    cv = orc.opacity_variance(bw["S"], bw["M"], bw["C"])
    np.testing.assert_allclose(cv[0], g.size * np.var(g), rtol=1e-9)
    # M is the total opacity gradient
    np.testing.assert_allclose(bw["M"][0], bw["grad9"][0, 5], rtol=1e-12)


def test_moments_identities_on_a_scene(orc):
    d = _small_splat_scene(4)
    r = orc.render_scene(d["scene"], d["camera"])
    w = np.random.default_rng(5).standard_normal(r["image"].shape)
    bw = orc.render_bwd(r["splats"], r["vals"], r["ranges"], d["camera"], w)
    np.testing.assert_allclose(bw["M"], bw["grad9"][:, 5], rtol=1e-10, atol=1e-14)
    cv = orc.opacity_variance(bw["S"], bw["M"], bw["C"])
    assert (cv >= -1e-12 * np.maximum(bw["S"], 1e-30)).all()
    assert (cv[bw["C"] == 0] == 0).all()
    # total included fragments = sum over pixels of included counts
    assert bw["C"].sum() > 0


def _one_gauss(scene, i):
    return {k: (scene[k][i:i + 1] if k != "sh_degree" else scene[k]) for k in scene}


def test_preprocess_backward_matches_fd(orc):
    d = scenegen.uniform_box_scene(64, 3, 7, 96, 64, focal=80.0)
    sc = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in d["scene"].items()}
    cam = d["camera"]
    rng = np.random.default_rng(8)
    ok = skipped = 0
    # a few large Gaussians outside the 1.3 x FOV Jacobian clamp (|x/z| > 0.78,
    # |y/z| > 0.52 here) whose footprint still reaches the image
    sc["mean"][:4] = [[2.5, 0.0, 3.0], [-2.5, 0.2, 3.0], [0.1, 1.8, 3.0], [2.4, -1.8, 3.0]]
    sc["log_scale"][:4] = np.log(0.4)
    limx, limy = 1.3 * 96 / (2 * 80.0), 1.3 * 64 / (2 * 80.0)
    clamped = 0
    for i in range(sc["mean"].shape[0]):
        g1 = _one_gauss(sc, i)
        base = orc.preprocess(g1, cam)
        if base["radius"][0] == 0:
            continue
        m = sc["mean"][i]
        clamped += abs(m[0] / m[2]) > limx or abs(m[1] / m[2]) > limy
        g9 = rng.standard_normal((1, 9))
        an = orc.preprocess_bwd(g1, cam, g9)

        def out9(s):
            p = orc.preprocess(s, cam)
            return np.concatenate([p["uv"][0], p["conic"][0], [p["opacity"][0]], p["rgb"][0]]), p

        for name in ("mean", "log_scale", "quat", "logit", "sh"):
            arr = g1[name]
            for idx in np.ndindex(arr.shape):
                x0 = arr[idx]
                h = 1e-6 * max(1.0, abs(x0))
                arr[idx] = x0 + h
                op, pp = out9(g1)
                arr[idx] = x0 - h
                om, pm = out9(g1)
                arr[idx] = x0
                same = all((pp[k] == base[k]).all() and (pm[k] == base[k]).all() for k in ("radius", "rect"))
                same &= ((pp["rgb"] > 0) == (base["rgb"] > 0)).all() and ((pm["rgb"] > 0) == (base["rgb"] > 0)).all()
                if not same:
                    skipped += 1
                    continue
                fd = float(np.dot(g9[0], (op - om) / (2 * h)))
                good, rel = _check(an[name][idx], fd, 1e-4)
                assert good, (i, name, idx, an[name][idx], fd, rel)
                ok += 1
    assert ok > 2000 and skipped < 0.05 * ok
    assert clamped == 4


def test_end_to_end_l1_gradient_matches_fd(orc):
    # the finite-difference scene of the differentiation case: 1,024
    # Gaussians, SH degree 3, 64 x 64, fx = fy = 64
    d = scenegen.uniform_box_scene(1024, 3, 11, 64, 64, focal=64.0)
    sc = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in d["scene"].items()}
    cam, tgt = d["camera"], d["target"]
    res = orc.loss_and_grad(sc, cam, tgt)
    dLdI = orc.l1_loss(res["render"]["image"], tgt)[1]
    vis = np.flatnonzero(res["render"]["splats"]["radius"] > 0)
    pick = np.random.default_rng(12).choice(vis, 6, replace=False)
    names = ("mean", "log_scale", "quat", "logit", "sh")
    scale = {k: np.sqrt(np.mean(res["grad"][k][vis] ** 2)) for k in names}
    ok = skipped = 0
    for i in pick:
        for name in names:
            arr = sc[name]
            shape = arr.shape[1:]
            for sub in np.ndindex(shape):
                idx = (i,) + sub
                x0 = arr[idx]
                h = 1e-6 * max(1.0, abs(x0))
                arr[idx] = x0 + h
                rp = orc.loss_and_grad(sc, cam, tgt)
                arr[idx] = x0 - h
                rm = orc.loss_and_grad(sc, cam, tgt)
                arr[idx] = x0
                if rp["decisions"] != res["decisions"] or rm["decisions"] != res["decisions"]:
                    skipped += 1
                    continue
                fd = np.sum(dLdI * (rp["render"]["image"] - rm["render"]["image"])) / (2 * h)
                good, rel = _check(res["grad"][name][idx], fd, 1e-3 * scale[name])
                assert good, (i, name, sub, res["grad"][name][idx], fd, rel)
                ok += 1
    assert ok > 250 and skipped < 0.2 * (ok + skipped)
