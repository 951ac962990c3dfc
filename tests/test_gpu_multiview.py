"""Batched views: one persistent raster launch over the tiles of several
cameras of different sizes.

Each view's image must equal the single-view path bit for bit (the tile
code is the same, only the scheduling differs); the parameter gradient,
summed over views by the accumulating preprocess backward, equals the
sequential single-view path up to the order of float atomics, and the
oracle's sum over views within the gradient tolerance. A CUDA-graph replay
of the batched sequence gives the same results as running it eagerly, with
the views' front ends on one stream or spread over several.
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import pipeline as PL
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu

RES = [(160, 96), (96, 64), (200, 120), (128, 128), (160, 96), (96, 64)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def _setup(n=20000, seed=5, res=RES, streams=4):
    d = scenegen.uniform_box_scene(n, 3, seed, 64, 64, with_target=False)
    sc = d["scene"]
    cams = scenegen.orbit_cameras(3, res, radius=4.0, elevation=0.2, center=scenegen.BOX_CENTER)
    rng = np.random.default_rng(seed)
    tgts = [U.t(rng.uniform(0, 1, (3, h, w)).astype(np.float32)) for w, h in res]
    planes, n = U.planes_tensor(sc)
    return sc, cams, tgts, PL.MultiView(planes, n, 3, cams, tgts, pair_capacity=2_000_000,
                                        streams=streams)


def _snap(mv):
    torch.cuda.synchronize()
    return ([v["image"].cpu().numpy() for v in mv.views], mv.grad.cpu().numpy().copy())


@pytest.mark.parametrize("streams", [1, 3])
def test_batched_views_equal_sequential_and_graph_replay(streams):
    """With the front ends on one stream, and spread over 3 side streams
    (6 views: two per slot, sharing its workspaces in order)."""
    _, _, _, mv = _setup(streams=streams)
    assert mv.n_slots == streams
    mv.run_sequential()
    imgs_s, grad_s = _snap(mv)
    mv.run_batched()
    imgs_b, grad_b = _snap(mv)
    for a, b in zip(imgs_s, imgs_b):
        np.testing.assert_array_equal(a, b)
        assert a.max() > 0
    assert np.abs(grad_s).max() > 0
    assert U.rel_l2(grad_b, grad_s) < 1e-5
    mv.capture()
    for v in mv.views:
        v["image"].zero_()
    mv.grad.zero_()
    mv.replay()
    imgs_g, grad_g = _snap(mv)
    for a, b in zip(imgs_s, imgs_g):
        np.testing.assert_array_equal(a, b)
    assert U.rel_l2(grad_g, grad_s) < 1e-5


def test_batched_gradient_sums_the_oracle_views(orc):
    res = [(96, 64), (128, 96)]
    sc, cams, tgts, mv = _setup(n=4096, seed=8, res=res)
    mv.run_batched()
    torch.cuda.synchronize()
    got = mv.grad.cpu().numpy()[:, :4096].astype(np.float64)
    want = np.zeros_like(got)
    for cam, tgt in zip(cams, tgts):
        sc64 = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in sc.items()}
        cc = orc.cluster_cull(sc64, cam, 128)
        rows = cc["map"]
        sub = {k: (v[rows] if k != "sh_degree" else v) for k, v in sc64.items()}
        r = orc.render_scene(sub, cam)
        _, dL = orc.l1_loss(r["image"], tgt.cpu().numpy())
        bw = orc.render_bwd(r["splats"], r["vals"], r["ranges"], cam, dL)
        want[:, rows] += orc.grad_planes(orc.preprocess_bwd(sub, cam, bw["grad9"]))
    for sl in (slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, None)):
        assert U.rel_l2(got[sl], want[sl]) < 1e-3
