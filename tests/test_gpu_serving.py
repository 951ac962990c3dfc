"""The render server on the GPU.

- Each request's image is the same when rendered alone (one slot, nothing
  else in flight) and in the mix (several slots, requests of different
  scenes and resolutions overlapping on the device): bit-identical, since
  no kernel of the forward path depends on timing.
- The pose read from device memory (graph replay) gives the same image as
  the pose given on the host.
- With the colour coefficients stored in BF16, the render equals the oracle's
  render of the same scene with its coefficients rounded to BF16
  (1e-5 max-abs on unflagged pixels, the FP32 image tolerance).
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import scenegen
from paper_2503_01199_gb300 import serving as SV

import gpu_util as U

pytestmark = pytest.mark.gpu

RES = [(96, 64), (160, 96), (200, 120)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


@pytest.fixture(scope="module")
def scenes():
    return [SV.ResidentScene(scenegen.uniform_box_scene(n, 3, seed, 64, 64, with_target=False)["scene"])
            for n, seed in ((20000, 10), (50000, 11))]


@pytest.mark.parametrize("grouped", [False, True])
def test_each_request_same_alone_and_in_the_mix(scenes, grouped):
    # grouped: requests admitted together share one batched raster launch
    reqs = scenegen.render_requests(7, 0.04, 1500.0, len(scenes), RES)
    assert len(reqs) > 30
    mix = SV.serve(scenes, reqs, hbm_budget_bytes=1 << 40, resolutions=RES,
                   pair_capacity=4_000_000, keep_images=True, max_slots=4, grouped=grouped)
    st = mix["stats"]
    assert st["requests"] == len(reqs) and st["pair_overflow"] == 0
    assert st["max_inflight"] > 1          # requests did overlap
    if grouped:
        assert st["max_group"] > 1         # and some shared a launch
    alone = SV.GpuExecutor(scenes, 1, RES, 4_000_000, use_graphs=False, keep_images=True)
    for r in mix["completed"]:
        q = {"scene": r["scene"], "camera": r["camera"]}
        alone.start(0, q)
        alone.slots[0].event.synchronize()
        alone.finish(0, q)
        np.testing.assert_array_equal(r["image"], q["image"])
        assert np.isfinite(q["image"]).all() and q["image"].max() > 0


@pytest.mark.parametrize("grouped", [False, True])
def test_slot_classes_and_overflow_retry(scenes, grouped):
    """Slots of three classes (one per resolution); the smallest class's pair
    capacity is set below what some of its requests need, so those are run
    again in a larger class. Every request completes once, with an image
    bit-identical to its render alone, and none is returned truncated."""
    reqs = scenegen.render_requests(8, 0.05, 1500.0, len(scenes), RES)
    alone = SV.GpuExecutor(scenes, 1, RES, 4_000_000, use_graphs=False, keep_images=True)
    need = {}
    for i, r in enumerate(reqs):
        q = {"scene": r["scene"], "camera": r["camera"]}
        alone.start(0, q)
        alone.slots[0].event.synchronize()
        assert alone.finish(0, q)
        need[i] = (q["pairs"], q["image"])
    small = [need[i][0] for i, r in enumerate(reqs) if r["camera"]["width"] == RES[0][0]]
    cap0 = int(np.median(small))                      # about half of them overflow
    classes = [(96, 64, cap0), (160, 96, 4_000_000), (200, 120, 4_000_000)]
    for i, r in enumerate(reqs):
        r["i"] = i
    max_n = max(sc.n for sc in scenes)
    budget = 2 * sum(SV.slot_bytes(max_n, w, h, cap) for w, h, cap in classes)
    out = SV.serve(scenes, reqs, hbm_budget_bytes=budget, resolutions=RES,
                   pair_capacity=4_000_000, keep_images=True, classes=classes, grouped=grouped)
    st = out["stats"]
    assert st["requests"] == len(reqs) and st["pair_overflow"] == 0
    assert st["retries"] == sum(p > cap0 for p in small) > 0
    assert len(st["slot_classes"]) == 3 and st["slots"] >= 6
    assert st["slot_classes"][0]["slot_bytes"] < st["slot_classes"][2]["slot_bytes"]
    ex = out["executor"]
    for r in out["completed"]:
        slot = ex.slots[r["slot"]]
        w, h = r["camera"]["width"], r["camera"]["height"]
        assert slot.fits(w, h) and r["pairs"] <= slot.cap
        np.testing.assert_array_equal(r["image"], need[r["i"]][1])


def test_device_pose_equals_host_pose(scenes):
    cam = scenegen.orbit_camera(4.0, 1.1, 0.2, 160, 96, center=scenegen.BOX_CENTER)
    ex_graph = SV.GpuExecutor(scenes, 1, [(160, 96)], 4_000_000, use_graphs=True, keep_images=True)
    ex_plain = SV.GpuExecutor(scenes, 1, [(160, 96)], 4_000_000, use_graphs=False, keep_images=True)
    for si in range(len(scenes)):
        out = []
        for ex in (ex_graph, ex_plain):
            q = {"scene": si, "camera": cam}
            ex.start(0, q)
            ex.slots[0].event.synchronize()
            ex.finish(0, q)
            out.append(q["image"])
        np.testing.assert_array_equal(out[0], out[1])


def test_bf16_colour_storage_matches_oracle_with_rounded_coefficients(orc):
    d = scenegen.uniform_box_scene(4096, 3, 12, 128, 128, with_target=False)
    sc, cam = d["scene"], d["camera"]
    planes, n = U.planes_tensor(sc)
    sh16 = planes[11:].to(torch.bfloat16).contiguous()
    geom = planes[:11].contiguous()
    g = B.gaussians_struct(geom, n, 3, sh16=sh16)
    cs = B.camera_struct(cam)
    rec = torch.zeros((n, 12), dtype=torch.float32, device="cuda")
    depth = torch.zeros(n, dtype=torch.float32, device="cuda")
    radius = torch.zeros(n, dtype=torch.int32, device="cuda")
    sp = B.splats_struct(rec, depth, radius)
    B.lgs_preprocess(g, None, None, cs, 16, 16, sp)
    torch.cuda.synchronize()
    rounded = dict(sc, sh=sh16.float().cpu().numpy()[:, :n].T.reshape(n, -1, 3))
    o = orc.preprocess({k: (np.asarray(v, np.float64) if k != "sh_degree" else v)
                        for k, v in rounded.items()}, cam)
    r = rec.cpu().numpy()
    vis = o["radius"] > 0
    np.testing.assert_array_equal(radius.cpu().numpy() > 0, vis)
    np.testing.assert_allclose(r[vis, 6:9], o["rgb"][vis], rtol=0, atol=2e-6)
    # the same call with the coefficients as float32 planes differs only by
    # the rounding of the coefficients
    g32 = B.gaussians_struct(planes, n, 3)
    rec32 = torch.zeros_like(rec)
    B.lgs_preprocess(g32, None, None, cs, 16, 16, B.splats_struct(rec32, depth, radius))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rec32.cpu().numpy()[:, :6], r[:, :6])
