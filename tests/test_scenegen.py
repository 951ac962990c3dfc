"""The synthetic bench input is what its recipe says: the surface scene
(90% of the means on 32 planes and 32 spheres within [-2, 2]^3 plus their
extent, 10% on a radius-20 shell; log-scales N(-4, 0.7); logits N(0, 1.5);
unit quaternions), seen by an orbit camera of radius 4 at 0.3 rad elevation
looking at the origin with fx = fy = 0.78 W. Seeded: the same seed gives the
same arrays."""
import numpy as np

from paper_2503_01199_gb300 import scenegen

N, W, H = 20_000, 1297, 840


def test_surface_scene_follows_its_recipe():
    d = scenegen.surface_scene(N, 3, 2, W, H)
    sc, cam = d["scene"], d["camera"]
    mean = sc["mean"].astype(np.float64)
    r = np.linalg.norm(mean, axis=1)
    n_shell = N // 10
    np.testing.assert_allclose(r[-n_shell:], 20.0, rtol=1e-6)
    # plane centres within 2 per axis plus half a diagonal of a side <= 2,
    # sphere centres plus radius <= 0.8, jitter 0.01
    assert np.abs(mean[:-n_shell]).max() < 2.0 + np.sqrt(2.0) + 0.1
    ls = sc["log_scale"].astype(np.float64)
    assert abs(ls.mean() + 4.0) < 0.02 and abs(ls.std() - 0.7) < 0.02
    lg = sc["logit"].astype(np.float64)
    assert abs(lg.mean()) < 0.05 and abs(lg.std() - 1.5) < 0.03
    np.testing.assert_allclose(np.linalg.norm(sc["quat"].astype(np.float64), axis=1), 1.0,
                               rtol=1e-6)
    assert sc["sh"].shape == (N, 16, 3) and sc["sh_degree"] == 3
    assert d["target"].shape == (3, H, W)
    # the orbit camera
    R = np.asarray(cam["R"], np.float64)
    c = -R.T @ np.asarray(cam["t"], np.float64)
    np.testing.assert_allclose(np.linalg.norm(c), 4.0, rtol=1e-6)
    np.testing.assert_allclose(abs(np.arcsin(c[1] / 4.0)), 0.3, rtol=1e-5)
    np.testing.assert_allclose(R[2], -c / np.linalg.norm(c), atol=1e-6)  # looks at the origin
    assert cam["fx"] == cam["fy"] == 0.78 * W
    assert (cam["width"], cam["height"]) == (W, H)


def test_surface_scene_is_seeded():
    a = scenegen.surface_scene(2000, 1, 7, 64, 48)
    b = scenegen.surface_scene(2000, 1, 7, 64, 48)
    c = scenegen.surface_scene(2000, 1, 8, 64, 48)
    for k in ("mean", "log_scale", "quat", "logit", "sh"):
        np.testing.assert_array_equal(a["scene"][k], b["scene"][k])
    assert not np.array_equal(a["scene"]["mean"], c["scene"]["mean"])
    np.testing.assert_array_equal(a["target"], b["target"])
