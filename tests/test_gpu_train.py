"""GPU parity of the whole training step (a1..a10) and of the Adam kernels.

The oracle runs the same step in double precision: Morton re-sort, cluster
cull, preprocess of the visible rows, binning, forward, L1 loss, backward,
preprocess backward, variance metric and sparse Adam on the visible rows.
Integer results (permutation, compaction map, V) must match exactly; the
image 1e-5 max-abs on pixels no flagged decision touches; gradients,
moments and the variance metric 1e-3 relative L2. At step 1 Adam moves a
parameter by +-lr (the sign of its gradient), so parameters are compared
only where the oracle gradient is clear of rounding.
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import pipeline as PL
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def oracle_step(orc, scene, cam, target, tile=(16, 16), step=1, lr=None):
    codes, perm = orc.morton_reorder(scene)
    sc = {k: (np.asarray(v, np.float64)[perm] if k != "sh_degree" else v) for k, v in scene.items()}
    cc = orc.cluster_cull(sc, cam, 128)
    rows = cc["map"]
    sub = {k: (v[rows] if k != "sh_degree" else v) for k, v in sc.items()}
    r = orc.render_scene(sub, cam, tile)
    L, dL = orc.l1_loss(r["image"], target)
    bw = orc.render_bwd(r["splats"], r["vals"], r["ranges"], cam, dL, tile)
    g = orc.grad_planes(orc.preprocess_bwd(sub, cam, bw["grad9"]))
    n = scene["mean"].shape[0]
    planes = orc.scene_planes(sc)
    grads = np.zeros_like(planes)
    grads[:, rows] = g
    m, v = np.zeros_like(planes), np.zeros_like(planes)
    newp = planes.copy()
    # the kernel receives beta1, beta2 and the rates as float32: use the same values
    orc.adam(newp, grads, m, v, np.asarray(lr, np.float32).astype(np.float64), step, rows,
             beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
             eps=float(np.float32(1e-15)))
    metric = np.zeros(n)
    metric[rows] = orc.opacity_variance(bw["S"], bw["M"], bw["C"])
    # pixels a Gaussian can reach (alpha >= 1/255) in the tiles it may or may
    # not be listed in, when its radius or tile rectangle is within rounding
    bad = np.zeros((cam["height"], cam["width"]), bool)
    tw, th = tile
    gx, gy = -(-cam["width"] // tw), -(-cam["height"] // th)
    sp = r["splats"]
    px, py = np.meshgrid(np.arange(cam["width"]) + 0.5, np.arange(cam["height"]) + 0.5)
    for i in np.flatnonzero(sp["flags"] & 5):
        radii = (sp["radius"][i] - 1, sp["radius"][i], sp["radius"][i] + 1) if sp["flags"][i] & 1 \
            else (sp["radius"][i],)
        eps = (-2e-3, 2e-3) if sp["flags"][i] & 4 else (0.0,)
        cands = []
        for rad in radii:
            for du in eps:
                for dv in eps:
                    u, v = sp["uv"][i, 0] + du, sp["uv"][i, 1] + dv
                    x0, x1 = np.floor((u - rad) / tw), np.floor((u + rad) / tw) + 1
                    y0, y1 = np.floor((v - rad) / th), np.floor((v + rad) / th) + 1
                    cands.append([int(np.clip(a, 0, g)) for a, g in ((x0, gx), (y0, gy), (x1, gx), (y1, gy))])
        m_all = np.zeros((gy, gx), int)
        for x0, y0, x1, y1 in cands:
            m_all[y0:y1, x0:x1] += 1
        amb = (m_all > 0) & (m_all < len(cands))
        amb_px = np.kron(amb, np.ones((th, tw), bool))[:cam["height"], :cam["width"]]
        dx, dy = sp["uv"][i, 0] - px, sp["uv"][i, 1] - py
        A, Bq, C = sp["conic"][i]
        reach = sp["opacity"][i] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - Bq * dx * dy) >= 0.999 / 255
        bad |= amb_px & reach
    bad |= r["pixflags"] != 0
    return {"perm": perm, "map": rows, "V": cc["V"], "image": r["image"], "loss": L, "grads": grads,
            "params": newp, "m": m, "v": v, "metric": metric, "bad": bad, "planes0": planes,
            "sflags": bw["sflags"], "last": last_rows(r["last"], r["vals"], r["ranges"], rows, tile)}


def last_rows(last, vals, ranges, rowmap, tile=(16, 16)):
    """Gaussian row of each pixel's last composited splat (-1: none); list
    positions depend on the tile culling, the splat does not."""
    H, W = last.shape
    tw, th = tile
    gx = -(-W // tw)
    out = np.full((H, W), -1, np.int64)
    for t in range(ranges.shape[0]):
        ty, tx = divmod(t, gx)
        blk = last[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw]
        m = blk > 0
        ids = np.full(blk.shape, -1, np.int64)
        ids[m] = np.asarray(rowmap)[vals[ranges[t, 0] + blk[m] - 1]]
        out[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw] = ids
    return out


def _run_gpu_step(scene, cam, target, fused, tile=(16, 16)):
    tr = PL.Trainer(scene, cam["width"], cam["height"], PL.StepConfig(tile=tile))
    tgt = U.t(target)
    tr.step(cam, tgt, reorder=True, fused=fused)
    torch.cuda.synchronize()
    n = tr.n
    out = {"perm": tr.perm.cpu().numpy().view(np.uint32), "V": int(tr.d_V.item()),
           "map": tr.rowmap.cpu().numpy().view(np.uint32)[: int(tr.d_V.item())],
           "image": tr.image.cpu().numpy(), "loss": float(tr.loss.item()),
           "params": tr.params.cpu().numpy()[:, :n].astype(np.float64),
           "m": tr.m.cpu().numpy()[:, :n], "v": tr.v.cpu().numpy()[:, :n],
           "metric": tr.metric.cpu().numpy(), "lr": tr.lr}
    out["last"] = last_rows(tr.last.cpu().numpy(), tr.vals.cpu().numpy().view(np.uint32),
                            tr.ranges.cpu().numpy().view(np.uint32), out["map"], tile)
    if not fused:
        out["grads"] = tr.grad_planes.cpu().numpy()[:, :n]
    return out


@pytest.mark.parametrize("deg", [0, 3])
def test_full_step_config1(orc, deg):
    # 4,096 Gaussians, 128 x 128, fx = fy = 128, seed 0, L1 against a uniform target
    d = scenegen.uniform_box_scene(4096, deg, 0, 128, 128)
    sc, cam, tgt = d["scene"], d["camera"], d["target"]
    g = _run_gpu_step(sc, cam, tgt, fused=False)
    o = oracle_step(orc, sc, cam, tgt, lr=g["lr"])
    np.testing.assert_array_equal(g["perm"], o["perm"])
    assert g["V"] == o["V"]
    np.testing.assert_array_equal(g["map"], o["map"])
    ok = ~o["bad"]
    assert ok.mean() > 0.99
    err = np.abs(g["image"] - o["image"])[:, ok].max()
    assert err <= 1e-5, err
    np.testing.assert_array_equal(g["last"][ok], o["last"][ok])
    # the loss also sums the flagged pixels, so it is checked on shared
    # inputs in test_loss_l1_kernel_matches_oracle; here only loosely
    assert abs(g["loss"] - o["loss"]) <= 1e-4 * o["loss"]
    rows = o["map"]
    for name, sl in (("mean", slice(0, 3)), ("log_scale", slice(3, 6)), ("quat", slice(6, 10)),
                     ("logit", slice(10, 11)), ("sh", slice(11, None))):
        e = U.rel_l2(g["grads"][sl][:, rows], o["grads"][sl][:, rows])
        assert e < 1e-3, (name, e)
        e = U.rel_l2(g["m"][sl][:, rows], o["m"][sl][:, rows])
        assert e < 1e-3, (name, "m", e)
    assert U.rel_l2(g["metric"][rows], o["metric"][rows]) < 1e-3
    # parameters: rows outside visible clusters are untouched; visible rows
    # moved by -lr sign(g) where the gradient sign is unambiguous
    og = o["grads"]
    clear = np.abs(og) > 1e-3 * np.sqrt(np.mean(og[:, rows] ** 2, axis=1, keepdims=True))
    clear[:, np.setdiff1d(np.arange(og.shape[1]), rows)] = False
    np.testing.assert_allclose(g["params"][clear], o["params"][clear], rtol=1e-6, atol=1e-7)
    hidden = np.setdiff1d(np.arange(og.shape[1]), rows)
    np.testing.assert_array_equal(g["params"][:, hidden], o["planes0"][:, hidden].astype(np.float32))


def test_fused_backward_adam_equals_separate(orc):
    d = scenegen.uniform_box_scene(4096, 3, 2, 128, 128)
    sc, cam, tgt = d["scene"], d["camera"], d["target"]
    a = _run_gpu_step(sc, cam, tgt, fused=False)
    b = _run_gpu_step(sc, cam, tgt, fused=True)
    np.testing.assert_array_equal(a["perm"], b["perm"])
    np.testing.assert_allclose(b["m"], a["m"], rtol=1e-4, atol=1e-12)
    np.testing.assert_allclose(b["v"], a["v"], rtol=1e-4, atol=1e-20)
    assert np.mean(np.abs(b["params"] - a["params"]) > 1e-6) < 1e-3


@pytest.mark.parametrize("layout", ["clusters", "scattered", "unaligned_run"])
def test_fused_backward_adam_map_layouts(layout):
    """The fused call reaches rows through the map in both of its passes:
    consecutive, scattered and unaligned runs of visible rows must all give
    the separate path's result, and rows outside the map must stay
    byte-identical. The a8 metric it writes on request equals
    lgs_opacity_variance's bit for bit, on the mapped rows only."""
    d = scenegen.uniform_box_scene(1000, 3, 9, 96, 96, focal=96.0)
    sc, cam = d["scene"], d["camera"]
    rng = np.random.default_rng(10)
    if layout == "clusters":          # consecutive from row 0: all units bulk-copied
        rows = np.arange(0, 1000)
    elif layout == "scattered":       # not consecutive, V % 4 != 0
        rows = np.sort(rng.choice(1000, 397, replace=False))
    else:                             # consecutive but starting at row 2
        rows = np.arange(2, 902)
    V = rows.size
    grads = np.zeros((1000, 16), np.float32)
    grads[:V, :9] = rng.standard_normal((V, 9)).astype(np.float32) * 1e-2
    # S, M and the fragment count C (slots 9..11; some C = 0) for the a8
    # metric the fused call may write
    grads[:V, 9] = rng.uniform(0, 1e-3, V).astype(np.float32)
    grads[:V, 10] = rng.standard_normal(V).astype(np.float32) * 1e-2
    grads[:V, 11] = rng.integers(0, 40, V).astype(np.uint32).view(np.float32)
    lr = PL.lr_per_plane(3)
    metrics = []
    m0 = rng.standard_normal((59, 1000)).astype(np.float32) * 1e-3
    v0 = rng.uniform(0, 1e-4, (59, 1000)).astype(np.float32)
    out = []
    # the separate path, the fused call recomputing the colours, and the
    # fused call taking the colour clamp from the forward's splat records
    for mode in ("separate", "fused", "fused_records"):
        planes, n = U.planes_tensor(sc)
        m = torch.zeros_like(planes)
        v = torch.zeros_like(planes)
        m[:, :n] = U.t(m0)
        v[:, :n] = U.t(v0)
        g = B.gaussians_struct(planes, n, 3)
        cs = B.camera_struct(cam)
        mp = U.t(rows.astype(np.uint32).view(np.int32))
        dV = U.t(np.array([V], np.int32))
        gacc = U.t(grads)
        metric = torch.full((1000,), -7.0, dtype=torch.float32, device="cuda")
        if mode == "fused":
            B.lgs_preprocess_bwd_adam(g, m, v, mp, dV, cs, gacc, lr, 0.9, 0.999, 1e-15, 3,
                                      metric=metric)
        elif mode == "fused_records":
            rec = torch.empty((1000, B.SPLAT_FLOATS), dtype=torch.float32, device="cuda")
            depth = torch.empty(1000, dtype=torch.float32, device="cuda")
            radius = torch.empty(1000, dtype=torch.int32, device="cuda")
            sp = B.splats_struct(rec, depth, radius)
            B.lgs_preprocess(g, mp, dV, cs, 16, 16, sp)
            B.lgs_preprocess_bwd_adam(g, m, v, mp, dV, cs, gacc, lr, 0.9, 0.999, 1e-15, 3,
                                      splats=sp, metric=metric)
        else:
            gp = torch.zeros_like(planes)
            B.lgs_preprocess_bwd(g, mp, dV, cs, gacc, gp)
            B.lgs_adam_step(planes, gp, m, v, planes.shape[0], lr, 0.9, 0.999, 1e-15, 3, mp, dV, n)
            B.lgs_opacity_variance(gacc, mp, dV, n, metric)
        torch.cuda.synchronize()
        metrics.append(metric.cpu().numpy())
        out.append((planes.cpu().numpy()[:, :n], m.cpu().numpy()[:, :n], v.cpu().numpy()[:, :n]))
    pa, ma, va = out[0]
    hidden = np.setdiff1d(np.arange(1000), rows)
    # the metric of the fused call is lgs_opacity_variance's, bit for bit,
    # on the mapped rows only
    C = grads[:V, 11].view(np.uint32)
    assert (C == 0).any() and (metrics[0][rows] != 0).any()
    assert (metrics[0][hidden] == -7.0).all()
    for mb in metrics[1:]:
        np.testing.assert_array_equal(mb, metrics[0])
    for pb, mb, vb in out[1:]:
        np.testing.assert_array_equal(pb[:, hidden], pa[:, hidden])
        np.testing.assert_array_equal(mb[:, hidden], ma[:, hidden])
        np.testing.assert_allclose(mb[:, rows], ma[:, rows], rtol=1e-4, atol=1e-9)
        np.testing.assert_allclose(vb[:, rows], va[:, rows], rtol=1e-4, atol=1e-14)
        np.testing.assert_allclose(pb[:, rows], pa[:, rows], rtol=1e-5, atol=1e-6)


def test_loss_l1_kernel_matches_oracle(orc):
    img = scenegen.random_image(41, 3, 333, 257) * 1.2 - 0.1
    tgt = scenegen.random_image(42, 3, 333, 257)
    tgt[0, :5, :7] = img[0, :5, :7]  # exact ties: sign(0) = 0
    L, dL = orc.l1_loss(img, tgt)
    ti, tt = U.t(img), U.t(tgt)
    g = torch.empty_like(ti)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.lgs_loss_l1(ti, tt, g, loss)
    torch.cuda.synchronize()
    # FP32 sums: per thread, per block, then one atomic per block in an
    # unordered sequence (hundreds of blocks); each rounding is <= 2^-24 of
    # the running total, so allow 1e-5 relative (the image tolerance)
    assert abs(float(loss.item()) - L) <= 1e-5 * L
    np.testing.assert_array_equal(g.cpu().numpy(), dL.astype(np.float32))


def test_adam_kernel_matches_oracle(orc):
    rng = np.random.default_rng(7)
    nplanes, n = 14, 1000
    stride = 1024
    p = np.zeros((nplanes, stride), np.float32)
    p[:, :n] = rng.standard_normal((nplanes, n))
    gr = np.zeros_like(p)
    gr[:, :n] = rng.standard_normal((nplanes, n)) * 1e-2
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    m[:, :n] = rng.standard_normal((nplanes, n)) * 1e-3
    v[:, :n] = rng.uniform(0, 1e-4, (nplanes, n))
    rows = np.concatenate([np.arange(0, 128), np.arange(384, 1000)]).astype(np.uint32)
    lr = np.linspace(1e-4, 1e-2, nplanes).astype(np.float32)
    tp, tg, tm, tv = U.t(p), U.t(gr), U.t(m), U.t(v)
    trow = U.t(rows.view(np.int32))
    dV = U.t(np.array([rows.size], np.int32))
    B.lgs_adam_step(tp, tg, tm, tv, nplanes, lr, 0.9, 0.999, 1e-15, 5, trow, dV, n)
    torch.cuda.synchronize()
    P64c = np.ascontiguousarray(p[:, :n], np.float64)
    M64c = np.ascontiguousarray(m[:, :n], np.float64)
    V64c = np.ascontiguousarray(v[:, :n], np.float64)
    # the kernel receives beta1, beta2 and eps as float32: use the same values
    orc.adam(P64c, gr[:, :n].astype(np.float64), M64c, V64c, lr.astype(np.float64), 5, rows,
             beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
             eps=float(np.float32(1e-15)))
    np.testing.assert_allclose(tp.cpu().numpy()[:, :n], P64c, rtol=1e-6, atol=1e-7)
    # m and v are sums of two terms that can cancel; float32 rounds beta1,
    # beta2 and the terms, so the error is relative to the terms
    tm_scale = 0.9 * np.abs(m[:, :n]) + 0.1 * np.abs(gr[:, :n])
    tv_scale = 0.999 * v[:, :n] + 0.001 * gr[:, :n] ** 2
    assert (np.abs(tm.cpu().numpy()[:, :n] - M64c) <= 1e-6 * tm_scale + 1e-30).all()
    assert (np.abs(tv.cpu().numpy()[:, :n] - V64c) <= 1e-6 * tv_scale + 1e-30).all()
    hidden = np.arange(128, 384)
    assert tp.cpu().numpy()[:, hidden].tobytes() == p[:, hidden].tobytes()
    assert tm.cpu().numpy()[:, hidden].tobytes() == m[:, hidden].tobytes()
    assert tv.cpu().numpy()[:, hidden].tobytes() == v[:, hidden].tobytes()


def test_cull_does_not_change_the_image(orc):
    # the same render with the compaction map and with every row visible
    d = scenegen.uniform_box_scene(20000, 1, 8, 256, 192, focal=256.0)
    d["scene"]["mean"][:8000, 0] += 4.0
    tr = PL.Trainer(d["scene"], 256, 192)
    tr.morton_reorder()
    cs = B.camera_struct(d["camera"])
    tr.render(None, cs)
    torch.cuda.synchronize()
    img_cull = tr.image.cpu().numpy().copy()
    V = int(tr.d_V.item())
    assert V < tr.n
    # render every row (identity map, V = n)
    g = tr.gaussians()
    B.lgs_preprocess(g, None, None, cs, 16, 16, tr.splats)
    B.lgs_bin_sort(tr.splats, None, tr.n, cs, 16, 16, tr.vals, tr.d_P, tr.ranges, tr.ws_bin)
    B.lgs_raster_fwd(tr.splats, tr.vals, tr.ranges, cs, 16, 16, tr.image, tr.finalT, tr.last)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(tr.image.cpu().numpy(), img_cull)


def test_checkpoint_resume_continues_identically(tmp_path):
    """save() after two steps, load() into a fresh trainer: the next step
    gives the same parameters and moments as continuing (up to the order of
    the backward's float atomic additions)."""
    d = scenegen.surface_scene(20000, 3, 41, 160, 120)
    sc, cam, tgt = d["scene"], d["camera"], U.t(d["target"])
    a = PL.Trainer(sc, 160, 120)
    a.step(cam, tgt, reorder=True)
    a.step(cam, tgt, reorder=False)
    path = tmp_path / "ckpt.npz"
    a.save(path)
    b = PL.Trainer(sc, 160, 120)
    b.load(path)
    assert b.n == a.n and b.step_count == a.step_count
    a.step(cam, tgt, reorder=False)
    b.step(cam, tgt, reorder=False)
    torch.cuda.synchronize()
    for x, y in ((a.params, b.params), (a.m, b.m), (a.v, b.v)):
        np.testing.assert_allclose(y[:, :b.n].cpu().numpy(), x[:, :a.n].cpu().numpy(),
                                   rtol=1e-4, atol=1e-9)
