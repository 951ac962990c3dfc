"""The bench workload at its full size, in the launch configuration the bench
times: the 3M-Gaussian surface scene (seed 2, SH 3, Morton-sorted) at
1297 x 840, one training iteration through the Trainer's calls. The oracle
checks sampled outputs one by one, and everything it can afford whole:

- a2: the visible clusters against the oracle's cluster cull of the same
  rows (clusters away from the test's rounding margin), and the map = the
  rows of the visible clusters in increasing order;
- a3: 4,000 sampled visible rows' splats against the oracle's preprocess of
  those Gaussians;
- a4: EVERY tile's list, bit for bit, against the oracle's binning of the
  kernels' own float32 splats;
- a5 / a7: 20 tiles (the 4 longest lists and 16 drawn at random) rendered
  by the oracle from the same splats and lists; the backward with dL/dI
  zero outside those tiles, so that every splat's gradient sums exactly the
  oracle's tiles (the fragment count C, which does not depend on dL/dI,
  for the splats listed in those tiles only);
- a9 + a10: the fused backward + Adam on sampled rows against the oracle's
  preprocess backward and Adam from the kernels' gradient rows.
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import pipeline as PL
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu

N, DEG, SEED, W, H = 3_000_000, 3, 2, 1297, 840
TILE = 16


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


@pytest.fixture(scope="module")
def run():
    d = scenegen.surface_scene(N, DEG, SEED, W, H)
    sc, cam = d["scene"], d["camera"]
    tr = PL.Trainer(sc, W, H, PL.StepConfig(tile=(TILE, TILE), pair_capacity=128_000_000))
    del sc, d
    tr.morton_reorder()
    cs = tr.render(cam)
    torch.cuda.synchronize()
    V, P = int(tr.d_V.item()), int(tr.d_P.item())
    out = {"tr": tr, "cam": cam, "cs": cs, "V": V, "P": P,
           "planes": tr.params[:, :tr.n].cpu().numpy(),
           "vis": tr.cluster_visible.cpu().numpy(),
           "map": tr.rowmap.cpu().numpy().view(np.uint32)[:V],
           "rec": tr.rec[:V].cpu().numpy(), "depth": tr.depth[:V].cpu().numpy(),
           "radius": tr.radius[:V].cpu().numpy(),
           "vals": tr.vals[:P].cpu().numpy().view(np.uint32),
           "ranges": tr.ranges.cpu().numpy().view(np.uint32),
           "image": tr.image.cpu().numpy(), "T": tr.finalT.cpu().numpy(),
           "last": tr.last.cpu().numpy()}
    yield out
    del out["tr"]
    torch.cuda.empty_cache()


def _scene_rows(planes, rows):
    p = planes[:, rows].astype(np.float64)
    return _scene_of(p)


def _scene_of(p):
    n = p.shape[1]
    return {"mean": p[0:3].T.copy(), "log_scale": p[3:6].T.copy(), "quat": p[6:10].T.copy(),
            "logit": p[10].copy(), "sh": p[11:].T.reshape(n, -1, 3).copy(), "sh_degree": DEG}


def _splats32(r):
    rec = r["rec"]
    return {"uv": rec[:, 0:2], "conic": rec[:, 2:5], "opacity": rec[:, 5], "rgb": rec[:, 6:9],
            "depth": r["depth"], "radius": r["radius"], "tau": rec[:, 9]}


def _sampled_tiles(r):
    ranges = r["ranges"].astype(np.int64)
    lens = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(7)
    longest = np.argsort(lens)[-4:]
    nonempty = np.flatnonzero(lens > 0)
    rand = rng.choice(np.setdiff1d(nonempty, longest), 16, replace=False)
    return np.sort(np.concatenate([longest, rand]))


def _tile_mask(tiles, gx):
    m = np.zeros((H, W), bool)
    for t in tiles:
        ty, tx = divmod(int(t), gx)
        m[ty * TILE:(ty + 1) * TILE, tx * TILE:(tx + 1) * TILE] = True
    return m


def test_fullsize_cull_and_map(orc, run):
    p = run["planes"]
    scene = {"mean": p[0:3].T.astype(np.float64), "log_scale": p[3:6].T.astype(np.float64)}
    ref = orc.cluster_cull(scene, run["cam"], 128)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(run["vis"][ok] != 0, ref["visible"][ok] != 0)
    n = p.shape[1]
    want = np.concatenate([np.arange(c * 128, min((c + 1) * 128, n))
                           for c in np.flatnonzero(run["vis"])])
    np.testing.assert_array_equal(run["map"], want)
    assert run["V"] == want.size and 0.5 * n < run["V"] < n


def test_fullsize_preprocess_sampled_rows(orc, run):
    js = np.random.default_rng(3).choice(run["V"], 4000, replace=False)
    rows = run["map"][js]
    op = orc.preprocess(_scene_rows(run["planes"], rows), run["cam"])
    rec = run["rec"][js]
    ok = op["flags"] == 0
    assert ok.mean() > 0.99
    rad = run["radius"][js]
    np.testing.assert_array_equal(rad[ok], op["radius"][ok])
    m = ok & (op["radius"] > 0)
    assert m.sum() > 1000
    np.testing.assert_allclose(rec[m, 0:2], op["uv"][m], rtol=1e-5, atol=2e-4)
    np.testing.assert_allclose(run["depth"][js][m], op["depth"][m], rtol=1e-6)
    np.testing.assert_allclose(rec[m, 5], op["opacity"][m], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(rec[m, 6:9], op["rgb"][m], rtol=1e-5, atol=1e-6)
    cn = np.linalg.norm(op["conic"][m], axis=1, keepdims=True)
    assert (np.abs(rec[m, 2:5] - op["conic"][m]) <= 1e-4 * cn).all()


def test_fullsize_every_tile_list_bit_exact(orc, run):
    sp = _splats32(run)
    _, _, P = U.check_bins(orc, run["vals"], run["ranges"], run["P"], sp, W, H, (TILE, TILE),
                           max_near_frac=1e-5)
    assert P > 10_000_000


def test_fullsize_raster_sampled_tiles(orc, run):
    orc.set_margins(*orc.MARGINS_SHARED_SPLATS)
    try:
        tr, cam = run["tr"], run["cam"]
        sp = _splats32(run)
        gx = -(-W // TILE)
        tiles = _sampled_tiles(run)
        rmask = np.zeros_like(run["ranges"])
        rmask[tiles] = run["ranges"][tiles]
        o = orc.render_fwd(sp, run["vals"], rmask, cam, (TILE, TILE))
        pix = _tile_mask(tiles, gx)
        ok = pix & (o["pixflags"] == 0)
        assert ok.sum() > 0.99 * pix.sum()
        assert np.abs(run["image"] - o["image"])[:, ok].max() <= 1e-5
        np.testing.assert_array_equal(run["last"][ok], o["last"][ok])
        np.testing.assert_allclose(run["T"][ok], o["T"][ok], rtol=2e-5, atol=1e-7)
        # backward with dL/dI on the sampled tiles only
        w = np.zeros((3, H, W), np.float32)
        w[:, pix] = np.random.default_rng(11).standard_normal((3, int(pix.sum()))) * 1e-3
        B.lgs_raster_bwd(tr.splats, tr.vals, tr.ranges, run["cs"], TILE, TILE, tr.finalT,
                         tr.last, U.t(w), tr.gacc)
        torch.cuda.synchronize()
        ga = tr.gacc[:run["V"]].cpu().numpy()
        ob = orc.render_bwd(sp, run["vals"], rmask, cam, w, (TILE, TILE))
        touched = np.unique(np.concatenate([run["vals"][rmask[t, 0]:rmask[t, 1]] for t in tiles]))
        assert touched.size > 1000
        for q in range(9):
            assert U.rel_l2(ga[:, q], ob["grad9"][:, q]) < 1e-3, q
        assert U.rel_l2(ga[:, 9], ob["S"]) < 1e-3
        assert U.rel_l2(ga[:, 10], ob["M"]) < 1e-3
        # C counts fragments whatever dL/dI is, so it matches for the splats
        # listed in sampled tiles only
        listed = np.concatenate([run["vals"][rmask[t, 0]:rmask[t, 1]] for t in tiles])
        only = (np.bincount(run["vals"], minlength=run["V"]) ==
                np.bincount(listed, minlength=run["V"])) & (np.bincount(listed, minlength=run["V"]) > 0)
        sok = (ob["sflags"] == 0) & only
        assert sok.sum() > 100
        np.testing.assert_array_equal(ga[:, 11].view(np.uint32)[sok], ob["C"][sok])
        others = np.setdiff1d(np.arange(run["V"]), touched)
        assert (ga[others][:, :11] == 0).all()
        run["touched"], run["gacc"] = touched, ga
    finally:
        orc.set_margins(*orc.MARGINS_END_TO_END)


def test_fullsize_fused_backward_adam_sampled_rows(orc, run):
    if "gacc" not in run:
        pytest.skip("needs the sampled-tile backward above")
    tr = run["tr"]
    g = tr.gaussians()
    B.lgs_preprocess_bwd_adam(g, tr.m, tr.v, tr.rowmap, tr.d_V, run["cs"], tr.gacc, tr.lr,
                              tr.cfg.beta1, tr.cfg.beta2, tr.cfg.eps, 1, splats=tr.splats)
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    js = np.sort(np.concatenate([rng.choice(run["touched"], 1500, replace=False),
                                 rng.choice(run["V"], 500, replace=False)]))
    js = np.unique(js)
    rows = run["map"][js]
    scene = _scene_rows(run["planes"], rows)
    g9 = run["gacc"][js, :9].astype(np.float64)
    ref_g = orc.grad_planes(orc.preprocess_bwd(scene, run["cam"], g9))
    p0 = np.ascontiguousarray(run["planes"][:, rows], dtype=np.float64)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    ref_g = np.ascontiguousarray(ref_g, dtype=np.float64)
    orc.adam(p, ref_g, m, v, np.asarray(tr.lr, np.float64), 1,
             np.arange(rows.size, dtype=np.uint32), tr.cfg.beta1, tr.cfg.beta2, tr.cfg.eps)
    gp = tr.params[:, rows].cpu().numpy().astype(np.float64)
    gm = tr.m[:, rows].cpu().numpy().astype(np.float64)
    for name, sl in (("mean", slice(0, 3)), ("log_scale", slice(3, 6)), ("quat", slice(6, 10)),
                     ("logit", slice(10, 11)), ("sh", slice(11, None))):
        assert U.rel_l2(gm[sl], m[sl]) < 1e-3, (name, "m")
    # parameters move by -lr sign(g) at step 1 where the sign is unambiguous
    clear = np.abs(ref_g) > 1e-3 * np.sqrt(np.mean(ref_g ** 2, axis=1, keepdims=True))
    np.testing.assert_allclose(gp[clear], p[clear], rtol=1e-6, atol=1e-7)
