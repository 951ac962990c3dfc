"""Pins of the oracle's densification, opacity decay and moment sums
(Sec. 3.3), independent of how the oracle computes them."""
import numpy as np

from paper_2503_01199_gb300 import scenegen


def _state(n=300, deg=1, seed=0, extra=64):
    sc = scenegen.uniform_box_scene(n, deg, seed, 64, 64, with_target=False)["scene"]
    import oracle
    planes = oracle.scene_planes(sc)
    full = np.zeros((planes.shape[0], n + extra))
    full[:, :n] = planes
    rng = np.random.default_rng(seed + 1)
    m = np.zeros_like(full)
    v = np.zeros_like(full)
    m[:, :n] = rng.standard_normal((planes.shape[0], n))
    v[:, :n] = rng.uniform(0, 1, (planes.shape[0], n))
    return full, m, v, rng


def test_selection_is_the_k_largest_positive_metrics(orc):
    full, m, v, rng = _state()
    n = 300
    metric = rng.standard_normal(n)
    metric[::7] = metric[3]          # ties
    K = 40
    z = rng.standard_normal((K, 2, 3))
    r = orc.densify(full, m, v, metric, K, 1e9, z)   # split threshold never reached: clones
    cand = [i for i in range(n) if metric[i] > 0]
    want = sorted(cand, key=lambda i: (-metric[i], i))[:K]
    assert list(r["selected"]) == want and r["n"] == n + len(want)
    # fewer candidates than K: all of them
    r2 = orc.densify(full, m, v, np.where(np.arange(n) < 5, 1.0, -1.0), K, 1e9, z)
    assert list(r2["selected"]) == [0, 1, 2, 3, 4] and r2["n"] == n + 5


def test_clone_appends_an_exact_copy_with_fresh_moments(orc):
    full, m, v, rng = _state()
    n = 300
    metric = np.zeros(n)
    metric[[10, 50]] = [2.0, 1.0]
    r = orc.densify(full, m, v, metric, 8, 1e9, rng.standard_normal((8, 2, 3)))
    assert list(r["selected"]) == [10, 50]
    np.testing.assert_array_equal(r["planes"][:, n], full[:, 10])
    np.testing.assert_array_equal(r["planes"][:, n + 1], full[:, 50])
    np.testing.assert_array_equal(r["planes"][:, :n], full[:, :n])   # originals untouched
    np.testing.assert_array_equal(r["m"][:, :n], m[:, :n])
    assert not r["m"][:, n:n + 2].any() and not r["v"][:, n:n + 2].any()


def test_split_samples_lie_at_the_drawn_mahalanobis_distance(orc):
    # a split sample x satisfies (x - p)^T Sigma^-1 (x - p) = |z|^2 for the
    # original covariance Sigma = R S^2 R^T (any rotation / scale convention
    # error breaks it), and both samples get scales s / 1.6
    full, m, v, rng = _state(deg=0)
    n = 300
    metric = np.zeros(n)
    sel = [3, 77, 150, 299]
    metric[sel] = [4.0, 3.0, 2.0, 1.0]
    z = rng.standard_normal((4, 2, 3))
    r = orc.densify(full, m, v, metric, 4, 0.0, z)   # threshold 0: every selection splits
    for k, i in enumerate(sel):
        p = full[0:3, i]
        s = np.exp(full[3:6, i])
        q = full[6:10, i] / np.linalg.norm(full[6:10, i])
        w, x, y, zz = q
        # rotation matrix of a unit quaternion via its action on basis vectors
        def rot(vec):
            qv = np.array([x, y, zz])
            t = 2.0 * np.cross(qv, vec)
            return vec + w * t + np.cross(qv, t)
        Rm = np.stack([rot(e) for e in np.eye(3)], axis=1)
        Sig = Rm @ np.diag(s * s) @ Rm.T
        for h, row in enumerate((i, n + k)):
            d = r["planes"][0:3, row] - p
            assert abs(d @ np.linalg.solve(Sig, d) - z[k, h] @ z[k, h]) < 1e-9 * (1 + z[k, h] @ z[k, h])
            np.testing.assert_allclose(np.exp(r["planes"][3:6, row]), s / 1.6, rtol=1e-14)
            np.testing.assert_array_equal(r["planes"][6:, row], full[6:, i])
            assert not r["m"][:, row].any() and not r["v"][:, row].any()
    # z = 0 puts both samples on the centre
    r0 = orc.densify(full, m, v, metric, 1, 0.0, np.zeros((1, 2, 3)))
    np.testing.assert_allclose(r0["planes"][0:3, 3], full[0:3, 3], atol=0)
    np.testing.assert_allclose(r0["planes"][0:3, n], full[0:3, 3], atol=0)


def test_split_or_clone_follows_the_largest_scale(orc):
    full, m, v, rng = _state()
    n = 300
    metric = np.zeros(n)
    metric[[1, 2]] = [2.0, 1.0]
    smax = np.exp(full[3:6, :n]).max(axis=0)
    thr = 0.5 * (smax[1] + smax[2])
    r = orc.densify(full, m, v, metric, 2, thr, rng.standard_normal((2, 2, 3)))
    split_first = smax[1] > thr
    # the split one changed its own row, the cloned one did not
    assert (r["planes"][:, 1] != full[:, 1]).any() == split_first
    assert (r["planes"][:, 2] != full[:, 2]).any() == (smax[2] > thr)
    assert split_first != (smax[2] > thr)


def test_opacity_decay_halves_the_activated_opacity(orc):
    logit = np.linspace(-30, 30, 601)
    out = orc.opacity_decay(logit)
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    np.testing.assert_allclose(sig(out), 0.5 * sig(logit), rtol=1e-13)
    assert (np.diff(out) > 0).all()


def test_moments_accumulate_over_views(orc):
    rng = np.random.default_rng(3)
    n = 50
    S_acc, M_acc, C_acc = np.zeros(n), np.zeros(n), np.zeros(n, np.int64)
    want_S, want_M, want_C = np.zeros(n), np.zeros(n), np.zeros(n, np.int64)
    for _ in range(3):
        rows = np.sort(rng.choice(n, 20, replace=False)).astype(np.uint32)
        S, M = rng.uniform(0, 1, 20), rng.standard_normal(20)
        C = rng.integers(0, 9, 20)
        orc.moments_accumulate(rows, S, M, C, S_acc, M_acc, C_acc)
        np.add.at(want_S, rows, S)
        np.add.at(want_M, rows, M)
        np.add.at(want_C, rows, C)
    np.testing.assert_allclose(S_acc, want_S, rtol=1e-15)
    np.testing.assert_allclose(M_acc, want_M, rtol=1e-15)
    np.testing.assert_array_equal(C_acc, want_C)
