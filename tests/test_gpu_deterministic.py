"""The bit-reproducible backward (lgs_raster_bwd_deterministic): the
cross-tile accumulation of Sec. 3.1's reduction made order-independent by
exact fixed-point integer sums.

- Two calls on the same inputs give identical bits, with the float warp
  sum and with the integer warp reduction, and at the full-size
  bench workload.
- The values are the oracle's within the FP32 gradient tolerance, and the
  float-atomic path's within the rounding of its atomics.
"""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import scenegen

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def _det(dev, w, precision):
    n = dev["n"]
    gacc = torch.full((max(n, 1), 16), 7.0, dtype=torch.float32, device="cuda")  # overwritten
    ws = torch.empty(B.lgs_raster_bwd_det_workspace_size(max(n, 1)), dtype=torch.uint8,
                     device="cuda")
    ws.fill_(0xA5)                                                              # any contents
    B.lgs_raster_bwd_deterministic(dev["splats"], dev["vals"], dev["ranges"], dev["cam"], 16, 16,
                                   dev["T"], dev["last"], U.t(w), gacc, ws, precision=precision)
    torch.cuda.synchronize()
    return gacc.cpu().numpy()[:n]


@pytest.mark.parametrize("reduce_int", [False, True])
def test_deterministic_backward_is_bit_reproducible_and_matches(orc, reduce_int):
    cam = scenegen.pinhole_camera(200, 150, 200.0, bg=(0.1, 0.2, 0.3))
    sp = U.random_splat_dict(3000, 41, 200, 150, max_radius=30)
    W, H = cam["width"], cam["height"]
    w = np.random.default_rng(42).standard_normal((3, H, W)).astype(np.float32) * 1e-3
    prec = B.LGS_FP32 | (B.LGS_WARP_REDUCE_INT if reduce_int else 0)
    g = U.gpu_raster(sp, cam, dLdI=w, precision=prec)
    a = _det(g["dev"], w, prec)
    b = _det(g["dev"], w, prec)
    assert a.tobytes() == b.tobytes()
    assert B.lgs_get_det_overflow() == 0
    np.testing.assert_array_equal(a[:, 12:], 0.0)
    np.testing.assert_array_equal(a[:, 10], a[:, 5])                  # M = the opacity sum
    np.testing.assert_array_equal(a[:, 11].view(np.uint32), g["C"])    # integer counts
    vals, ranges, P = orc.bin_splats(sp["uv"][:, 0], sp["uv"][:, 1], sp["radius"], sp["depth"], W, H,
                                     (16, 16), conic=sp["conic"], tau=sp["tau"])
    ob = orc.render_bwd(sp, vals, ranges, cam, w, (16, 16))
    for q in range(9):
        assert U.rel_l2(a[:, q], ob["grad9"][:, q]) < 1e-3, q
        assert U.rel_l2(a[:, q], g["grad9"][:, q]) < 1e-5, q
    assert U.rel_l2(a[:, 9], ob["S"]) < 1e-3 and U.rel_l2(a[:, 10], ob["M"]) < 1e-3


def test_deterministic_backward_at_full_size():
    """The 3M-Gaussian surface scene at 1297 x 840 (2.7M splats, 22M pairs):
    identical bits over two calls, and the float-atomic path within its
    rounding."""
    from paper_2503_01199_gb300 import pipeline as PL
    d = scenegen.surface_scene(3_000_000, 3, 2, 1297, 840)
    tr = PL.Trainer(d["scene"], 1297, 840, PL.StepConfig(pair_capacity=128_000_000))
    tgt, cam = U.t(d["target"]), d["camera"]
    del d
    tr.morton_reorder()
    cs = tr.render(cam)
    tr.backward(cs, tgt)
    torch.cuda.synchronize()
    V = int(tr.d_V.item())
    ref = tr.gacc[:V].cpu().numpy()
    ws = torch.empty(B.lgs_raster_bwd_det_workspace_size(tr.n), dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(2):
        gacc = torch.empty_like(tr.gacc)
        B.lgs_raster_bwd_deterministic(tr.splats, tr.vals, tr.ranges, cs, 16, 16, tr.finalT,
                                       tr.last, tr.dLdI, gacc, ws)
        torch.cuda.synchronize()
        outs.append(gacc[:V].cpu().numpy())
    assert outs[0].tobytes() == outs[1].tobytes()
    assert B.lgs_get_det_overflow() == 0
    for q in range(11):
        assert U.rel_l2(outs[0][:, q], ref[:, q]) < 1e-5, q
    np.testing.assert_array_equal(outs[0][:, 11].view(np.uint32), ref[:, 11].view(np.uint32))
    del tr
    torch.cuda.empty_cache()
