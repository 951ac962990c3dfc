"""The allocation-free cluster cull (lgs_cluster_cull_compact_noalloc) gives
the same results as lgs_cluster_cull_compact with a caller workspace.

It exists for callers that cannot call cudaMalloc or hand out a workspace
(code inside another framework's memory pool, code that must not
synchronise the device, hosts that forbid allocation at frame time); its
scratch is a fixed array inside the library. The check runs two calls in a
row on different scenes and cameras, so a second call must not depend on
what the first one left in that shared array; the outputs are integers and
float bounds produced by the same kernels, so they must match exactly.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu


def _run(fn, sc, cam, cs=128, with_ws=False):
    planes, n = U.planes_tensor(sc)
    g = B.gaussians_struct(planes, n, sc["sh_degree"])
    ncl = -(-n // cs)
    aabb = torch.full((ncl, 6), -7.0, dtype=torch.float32, device="cuda")
    vis = torch.full((ncl,), 7, dtype=torch.int32, device="cuda")
    rowmap = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    dV = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    if with_ws:
        ws = torch.empty(B.lgs_ccc_workspace_size(n, cs), dtype=torch.uint8, device="cuda")
        fn(g, B.camera_struct(cam), cs, aabb, vis, rowmap, dV, ws)
    else:
        fn(g, B.camera_struct(cam), cs, aabb, vis, rowmap, dV)
    torch.cuda.synchronize()
    V = int(dV.item())
    return {"V": V, "map": rowmap.cpu().numpy()[:V], "vis": vis.cpu().numpy(),
            "aabb": aabb.cpu().numpy()}


def test_noalloc_cull_matches_workspace_version_twice():
    U.need_gpu()
    cases = []
    d1 = scenegen.uniform_box_scene(40000, 0, 31, 320, 240, focal=320.0)
    d1["scene"]["mean"][:15000, 0] += 5.0          # a block of culled clusters
    cases.append((d1["scene"], d1["camera"]))
    d2 = scenegen.surface_scene(100003, 1, 32, 640, 360)
    R, t = np.asarray(d2["camera"]["R"], np.float64), np.asarray(d2["camera"]["t"], np.float64)
    behind = -R.T @ t - 10.0 * R[2]                 # 10 units behind the camera
    d2["scene"]["mean"][20000:40000] = (behind + 0.1 * np.random.default_rng(33).standard_normal(
        (20000, 3))).astype(np.float32)
    cases.append((d2["scene"], d2["camera"]))
    for sc, cam in cases:                          # two calls in a row
        ref = _run(B.lgs_cluster_cull_compact, sc, cam, with_ws=True)
        got = _run(B.lgs_cluster_cull_compact_noalloc, sc, cam)
        assert 0 < ref["V"] < sc["mean"].shape[0]
        assert got["V"] == ref["V"]
        np.testing.assert_array_equal(got["map"], ref["map"])
        np.testing.assert_array_equal(got["vis"], ref["vis"])
        np.testing.assert_array_equal(got["aabb"], ref["aabb"])


def test_noalloc_cull_rejects_more_clusters_than_its_scratch_holds():
    U.need_gpu()
    L = B.load()
    planes = torch.zeros((14, 8), dtype=torch.float32, device="cuda")
    g = B.gaussians_struct(planes, 8, 0)
    g.n = (B.NOALLOC_MAX_CLUSTERS + 1) * 128       # descriptor only: nothing is read
    g.stride = g.n
    cam = B.camera_struct(scenegen.pinhole_camera(64, 64, 64.0))
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = L.lgs_cluster_cull_compact_noalloc(ctypes.byref(g), ctypes.byref(cam), 128, None, None,
                                            dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == B.LGS_ERR_TOO_LARGE
