"""Pins of the oracle's Morton codes, sort, cluster cull, Adam and L1 loss.

Morton (Sec. 3.2.1): worked examples that follow from the definition of a
3-way bit interleave, the all-ones code, decode(encode) round trips and the
quantisation of the bounding-box corners. Sort: numpy's stable argsort.
Cluster-Cull-Compact (Sec. 3.2.2): the cull is conservative (every rendered
Gaussian sits in a visible cluster) and the image is unchanged by it.
Adam (Sec. 3.2.3): torch.optim.Adam in float64 on the all-visible case; rows
outside the visible clusters stay byte-identical.
"""
import numpy as np
import pytest

from paper_2503_01199_gb300 import scenegen


def _decode(code):
    x = y = z = 0
    for k in range(21):
        x |= ((code >> (3 * k)) & 1) << k
        y |= ((code >> (3 * k + 1)) & 1) << k
        z |= ((code >> (3 * k + 2)) & 1) << k
    return x, y, z


def test_morton_worked_examples(orc):
    assert orc.morton_interleave(1, 0, 0) == 1
    assert orc.morton_interleave(0, 1, 0) == 2
    assert orc.morton_interleave(0, 0, 1) == 4
    assert orc.morton_interleave(1, 1, 1) == 7
    assert orc.morton_interleave(2, 0, 0) == 8
    m = (1 << 21) - 1
    assert orc.morton_interleave(m, m, m) == (1 << 63) - 1
    assert orc.morton_interleave(m, 0, 0) == int("001" * 21, 2)


def test_morton_round_trip_and_order(orc):
    rng = np.random.default_rng(0)
    for _ in range(300):
        x, y, z = (int(a) for a in rng.integers(0, 1 << 21, 3))
        assert _decode(orc.morton_interleave(x, y, z)) == (x, y, z)
    # all 4-bit triples: the code is a bijection onto [0, 2^12)
    codes = {orc.morton_interleave(x, y, z) for x in range(16) for y in range(16) for z in range(16)}
    assert codes == set(range(1 << 12))


def test_morton_quantisation_corners(orc):
    mean = np.random.default_rng(1).uniform(-3, 5, (1000, 3)).astype(np.float32)
    codes = orc.morton_codes(mean)
    lo = np.argmin(mean, axis=0)
    hi = np.argmax(mean, axis=0)
    for k in range(3):
        q = [_decode(int(c))[k] for c in codes]
        assert q[lo[k]] == 0 and q[hi[k]] == (1 << 21) - 1
        assert min(q) == 0 and max(q) == (1 << 21) - 1
    # quantisation is monotone in each coordinate
    order = np.argsort(mean[:, 0], kind="stable")
    qx = np.array([_decode(int(c))[0] for c in codes])[order]
    assert (np.diff(qx.astype(np.int64)) >= 0).all()
    # a degenerate axis maps to 0
    flat = mean.copy()
    flat[:, 1] = 2.5
    assert all(_decode(int(c))[1] == 0 for c in orc.morton_codes(flat))


def test_stable_sort_matches_numpy(orc):
    rng = np.random.default_rng(2)
    for n, hi in [(1, 3), (1000, 7), (5000, 1 << 40), (3000, 1)]:
        keys = rng.integers(0, hi, n).astype(np.uint64)
        np.testing.assert_array_equal(orc.sort_u64_stable(keys), np.argsort(keys, kind="stable"))


@pytest.mark.parametrize("gen", ["box", "surface"])
def test_cluster_cull_is_conservative(orc, gen):
    if gen == "box":
        d = scenegen.uniform_box_scene(6000, 0, 3, 96, 64, focal=96.0)
        # move part of the scene behind / beside the camera
        d["scene"]["mean"][:2000, 0] += 6.0
        d["scene"]["mean"][2000:3000, 2] -= 6.0
    else:
        d = scenegen.surface_scene(40000, 0, 4, 128, 96)
    sc, cam = d["scene"], d["camera"]
    codes, perm = orc.morton_reorder(sc)
    sc = {k: (v[perm] if k != "sh_degree" else v) for k, v in sc.items()}
    cc = orc.cluster_cull(sc, cam, 128)
    assert 0 < cc["V"] < sc["mean"].shape[0]
    sp = orc.preprocess(sc, cam)
    rendered = np.flatnonzero(sp["radius"] > 0)
    assert np.isin(rendered, cc["map"]).all()
    # the image is identical with and without the cull
    full = orc.render_scene(sc, cam)
    sub = {k: (v[cc["map"]] if k != "sh_degree" else v) for k, v in sc.items()}
    part = orc.render_scene(sub, cam)
    np.testing.assert_array_equal(full["image"], part["image"])
    np.testing.assert_array_equal(full["last"], part["last"])
    # the map lists whole clusters in increasing order
    m = cc["map"].astype(np.int64)
    assert (np.diff(m) > 0).all()
    vis = np.flatnonzero(cc["visible"])
    expect = np.concatenate([np.arange(c * 128, min(c * 128 + 128, sc["mean"].shape[0])) for c in vis])
    np.testing.assert_array_equal(m, expect)


def test_cluster_behind_camera_is_culled(orc):
    cam = scenegen.pinhole_camera(64, 64, 64.0)
    n = 256
    mean = np.zeros((n, 3))
    mean[:128, 2] = -5.0   # cluster 0 behind the camera
    mean[128:, 2] = 5.0    # cluster 1 in front
    sc = {"mean": mean, "log_scale": np.full((n, 3), -3.0)}
    cc = orc.cluster_cull(sc, cam, 128)
    np.testing.assert_array_equal(cc["visible"], [0, 1])
    assert cc["V"] == 128


def test_adam_matches_torch_all_visible(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    nplanes, nrows = 7, 50
    p0 = rng.standard_normal((nplanes, nrows))
    lr = np.linspace(1e-3, 5e-2, nplanes)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    tp = [torch.tensor(p0[k].copy(), dtype=torch.float64, requires_grad=True) for k in range(nplanes)]
    opt = torch.optim.Adam([{"params": [tp[k]], "lr": float(lr[k])} for k in range(nplanes)],
                           betas=(0.9, 0.999), eps=1e-15)
    rows = np.arange(nrows, dtype=np.uint32)
    for step in range(1, 6):
        g = rng.standard_normal((nplanes, nrows))
        orc.adam(p, g, m, v, lr, step, rows)
        for k in range(nplanes):
            tp[k].grad = torch.tensor(g[k], dtype=torch.float64)
        opt.step()
        for k in range(nplanes):
            np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_sparse_rows_untouched(orc):
    rng = np.random.default_rng(4)
    p = rng.standard_normal((3, 300))
    m = rng.standard_normal((3, 300))
    v = rng.uniform(0, 1, (3, 300))
    before = (p.copy(), m.copy(), v.copy())
    rows = np.concatenate([np.arange(0, 128), np.arange(256, 300)]).astype(np.uint32)
    orc.adam(p, rng.standard_normal((3, 300)), m, v, np.array([0.1, 0.2, 0.3]), 3, rows)
    hidden = np.arange(128, 256)
    for a, b in zip((p, m, v), before):
        assert a[:, hidden].tobytes() == b[:, hidden].tobytes()
        assert not np.array_equal(a[:, rows], b[:, rows])


def test_l1_loss_and_gradient(orc):
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (3, 8, 9))
    tgt = img.copy()
    tgt[0, 0, 0] += 0.5
    tgt[1, 2, 3] -= 0.25
    L, g = orc.l1_loss(img, tgt)
    assert abs(L - 0.75 / img.size) < 1e-16
    n = img.size
    assert g[0, 0, 0] == -1.0 / n and g[1, 2, 3] == 1.0 / n
    assert np.count_nonzero(g) == 2   # sign(0) = 0


def test_cluster_cull_side_planes_closed_form(orc):
    """Sec. 3.2.2's cull against each of the five planes in turn: a cluster
    box whose nearest corner is a relative 1e-3 inside a plane is kept, one
    1e-3 outside is culled (camera turned and moved; closed forms in
    cull_cases). Deleting any plane keeps an outside cluster; transposing
    the camera rotation moves the boxes elsewhere."""
    import cull_cases as CC
    sc, want = CC.side_plane_scene()
    cc = orc.cluster_cull(sc, CC.camera(), CC.CLUSTER)
    np.testing.assert_array_equal(cc["visible"], want)
    assert (cc["flags"] == 0).all()
    assert cc["V"] == CC.CLUSTER * int(want.sum())


def test_cluster_cull_widening_by_three_largest_scales(orc):
    """The box is widened by 3 x the largest scale of each member: clusters
    whose centres all lie outside a side plane are kept exactly when one
    member's 3 s reaches it (s on the x, y or z axis; 3 s a relative 2e-3
    above or below the reach needed)."""
    import cull_cases as CC
    sc, want = CC.widening_scene()
    cc = orc.cluster_cull(sc, CC.camera(), CC.CLUSTER)
    np.testing.assert_array_equal(cc["visible"], want)
    assert (cc["flags"] == 0).all()
