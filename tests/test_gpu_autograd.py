"""The rasterizer as a torch.autograd.Function: its gradient against the
oracle's analytic gradient and against finite differences of its own
forward.

The Function runs cull + compaction, preprocess, binning and the forward
raster; its backward runs the backward raster (transmittance recovered back
to front from the stored final T, nothing per fragment kept) and the
preprocess backward. Gradients must match the oracle within 1e-3 relative
L2 per parameter group.
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import autograd as AG
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu

GROUPS = (("mean", slice(0, 3)), ("log_scale", slice(3, 6)), ("quat", slice(6, 10)),
          ("logit", slice(10, 11)), ("sh", slice(11, None)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def oracle_grads(orc, scene, cam, target):
    """L1 loss gradient for every parameter plane, rows in storage order
    (cluster cull + compaction, no Morton re-sort)."""
    sc = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in scene.items()}
    cc = orc.cluster_cull(sc, cam, 128)
    rows = cc["map"]
    sub = {k: (v[rows] if k != "sh_degree" else v) for k, v in sc.items()}
    r = orc.render_scene(sub, cam)
    L, dL = orc.l1_loss(r["image"], target)
    bw = orc.render_bwd(r["splats"], r["vals"], r["ranges"], cam, dL)
    g = orc.grad_planes(orc.preprocess_bwd(sub, cam, bw["grad9"]))
    grads = np.zeros((g.shape[0], scene["mean"].shape[0]))
    grads[:, rows] = g
    metric = np.zeros(scene["mean"].shape[0])
    metric[rows] = orc.opacity_variance(bw["S"], bw["M"], bw["C"])
    return grads, rows, L, metric


def gpu_grads(scene, cam, target, precision="fp32"):
    planes, n = U.planes_tensor(scene)
    planes.requires_grad_(True)
    r = AG.GaussianRasterizer(n, scene["sh_degree"], cam["width"], cam["height"],
                              precision=precision)
    metric = torch.zeros(n, dtype=torch.float32, device="cuda")
    img = AG.rasterize(planes, cam, r, metric=metric)
    loss = (img - U.t(target, np.float32)).abs().mean()
    loss.backward()
    torch.cuda.synchronize()
    return (planes.grad.cpu().numpy()[:, :n].astype(np.float64), float(loss.item()),
            img.detach().cpu().numpy(), metric.cpu().numpy())


@pytest.mark.parametrize("case", ["config1_sh0", "fd_scene_sh3"])
def test_autograd_gradient_matches_oracle(orc, case):
    if case == "config1_sh0":   # 4,096 Gaussians, SH0, 128 x 128, seed 0
        d = scenegen.uniform_box_scene(4096, 0, 0, 128, 128)
    else:                       # 1,024 Gaussians, SH3, 64 x 64, fx = fy = 64
        d = scenegen.uniform_box_scene(1024, 3, 11, 64, 64, focal=64.0)
    sc, cam, tgt = d["scene"], d["camera"], d["target"]
    og, rows, oL, ometric = oracle_grads(orc, sc, cam, tgt)
    gg, gL, _, gmetric = gpu_grads(sc, cam, tgt)
    assert abs(gL - oL) <= 1e-4 * oL
    for name, sl in GROUPS:
        e = U.rel_l2(gg[sl][:, rows], og[sl][:, rows])
        assert e < 1e-3, (name, e)
    hidden = np.setdiff1d(np.arange(gg.shape[1]), rows)
    assert not gg[:, hidden].any()
    assert U.rel_l2(gmetric[rows], ometric[rows]) < 1e-3


def test_autograd_pending_forwards_keep_their_own_buffers():
    # two forwards on different cameras before either backward: each backward
    # must use its own saved lists, so the sum equals the two runs apart
    d = scenegen.uniform_box_scene(4096, 1, 5, 96, 80, focal=96.0)
    sc = d["scene"]
    c0 = d["camera"]
    cams = [c0, dict(c0, t=np.array([0.3, -0.2, 0.5], np.float32))]
    planes, n = U.planes_tensor(sc)
    r = AG.GaussianRasterizer(n, 1, 96, 80)
    w = [torch.randn((3, 80, 96), device="cuda", generator=torch.Generator("cuda").manual_seed(k))
         for k in range(2)]
    sep = []
    for k in range(2):
        p = planes.clone().requires_grad_(True)
        (AG.rasterize(p, cams[k], r) * w[k]).sum().backward()
        sep.append(p.grad.clone())
    p = planes.clone().requires_grad_(True)
    imgs = [AG.rasterize(p, cams[k], r) for k in range(2)]
    ((imgs[0] * w[0]).sum() + (imgs[1] * w[1]).sum()).backward()
    torch.cuda.synchronize()
    both = (sep[0] + sep[1]).cpu().numpy()
    assert np.abs(both).max() > 0
    np.testing.assert_allclose(p.grad.cpu().numpy(), both, rtol=1e-5,
                               atol=1e-6 * np.abs(both).max())


def test_autograd_matches_finite_differences(orc):
    """Central differences of the GPU forward (FP32) of L = sum w . I on the
    1,024-Gaussian SH3 64 x 64 scene; steps whose +-h changes a discrete
    decision in the oracle's render at the same parameters are skipped."""
    d = scenegen.uniform_box_scene(1024, 3, 11, 64, 64, focal=64.0)
    sc, cam = d["scene"], d["camera"]
    planes, n = U.planes_tensor(sc)
    r = AG.GaussianRasterizer(n, 3, 64, 64)
    w = np.random.default_rng(13).standard_normal((3, 64, 64))
    wt = U.t(w, np.float32)
    p = planes.clone().requires_grad_(True)
    (AG.rasterize(p, cam, r) * wt).sum().backward()
    an = p.grad.cpu().numpy().astype(np.float64)
    host = planes.cpu().numpy()

    def L_gpu(pl):
        with torch.no_grad():
            img = AG.rasterize(U.t(pl), cam, r).cpu().numpy().astype(np.float64)
        return float(np.sum(w * img))

    def decisions(pl):
        s = {"mean": pl[0:3, :n].T, "log_scale": pl[3:6, :n].T, "quat": pl[6:10, :n].T,
             "logit": pl[10, :n], "sh": pl[11:, :n].T.reshape(n, -1, 3), "sh_degree": 3}
        s = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in s.items()}
        res = orc.render_scene(s, cam)
        sp = res["splats"]
        return (res["hash"], sp["radius"].tobytes(), sp["rect"].tobytes(),
                (sp["rgb"] > 0).tobytes(), sp["flags"].tobytes(), res["pixflags"].any())

    base = decisions(host)
    vis = np.flatnonzero(np.abs(an[10, :n]) > 0)
    pick = np.random.default_rng(14).choice(vis, 6, replace=False)
    scale = {name: np.sqrt(np.mean(an[sl, :n][:, vis] ** 2)) for name, sl in GROUPS}
    errs, skipped = [], 0
    for i in pick:
        for name, sl in GROUPS:
            for k in range(*sl.indices(an.shape[0])):
                x0 = host[k, i]
                h = (1e-2 if name == "sh" else 2e-3) * max(1.0, abs(float(x0)))
                hp, hm = host.copy(), host.copy()
                hp[k, i] = np.float32(x0 + h)
                hm[k, i] = np.float32(x0 - h)
                if decisions(hp) != base or decisions(hm) != base:
                    skipped += 1
                    continue
                fd = (L_gpu(hp) - L_gpu(hm)) / (float(hp[k, i]) - float(hm[k, i]))
                err = abs(fd - an[k, i]) / max(abs(an[k, i]), 1e-2 * scale[name])
                assert err < 5e-2, (i, name, k, an[k, i], fd, err)
                errs.append(err)
    # FP32 forward: rounding of the two renders is O(1e-7) per touched pixel,
    # truncation O(h^2); the typical error is far below the worst
    errs = np.asarray(errs)
    assert errs.size > 150 and skipped < errs.size, (errs.size, skipped)
    assert np.median(errs) < 2e-3, np.quantile(errs, [0.5, 0.9, 1.0])
