"""Edge cases of the training step and graph capture.

- Every Gaussian culled (camera looking away): V = 0, the image is the
  background, no pair is listed, nothing is updated.
- One Gaussian on a 1 x 1 image; a ragged image smaller than a tile.
- The whole a2-a10 iteration captured in a CUDA graph (no host sync, no
  allocation inside the library) replays to the eager result.
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


def test_everything_culled():
    d = scenegen.uniform_box_scene(2000, 1, 4, 64, 48, focal=64.0)
    cam = dict(d["camera"], R=np.diag([-1.0, 1.0, -1.0]).astype(np.float32))   # looks away
    tr = PL.Trainer(d["scene"], 64, 48)
    before = tr.params.clone()
    tr.step(cam, U.t(d["target"]), reorder=False)
    torch.cuda.synchronize()
    assert int(tr.d_V.item()) == 0 and int(tr.d_P.item()) == 0
    bg = np.asarray(cam["bg"], np.float32)
    np.testing.assert_array_equal(tr.image.cpu().numpy(),
                                  np.broadcast_to(bg[:, None, None], (3, 48, 64)))
    np.testing.assert_array_equal(tr.params.cpu().numpy(), before.cpu().numpy())


@pytest.mark.parametrize("W,H,n", [(1, 1, 1), (13, 7, 50), (17, 33, 400)])
def test_tiny_images_match_oracle(orc, W, H, n):
    d = scenegen.uniform_box_scene(n, 0, 6 + n, W, H, focal=float(max(W, H)))
    tr = PL.Trainer(d["scene"], W, H)
    tr.render(d["camera"])
    torch.cuda.synchronize()
    o = orc.render_scene(d["scene"], d["camera"])
    ok = o["pixflags"] == 0
    err = np.abs(tr.image.cpu().numpy() - o["image"])[:, ok]
    assert err.size == 0 or err.max() <= 1e-5


def test_iteration_captured_in_a_cuda_graph():
    d = scenegen.uniform_box_scene(8192, 3, 7, 160, 120, focal=160.0)
    cam, tgt = d["camera"], U.t(d["target"])
    eager = PL.Trainer(d["scene"], 160, 120)
    graphed = PL.Trainer(d["scene"], 160, 120)
    cs = B.camera_struct(cam)
    for tr in (eager, graphed):
        tr.morton_reorder()
        tr.render(None, cs)               # first calls outside any capture
        tr.backward(cs, tgt)
    torch.cuda.synchronize()
    eager.step(cs, tgt, reorder=False)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        graphed.step(cs, tgt, reorder=False)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(graphed.image.cpu().numpy(), eager.image.cpu().numpy())
    assert abs(float(graphed.loss.item()) - float(eager.loss.item())) <= 1e-6
    a, b = eager.params.cpu().numpy(), graphed.params.cpu().numpy()
    # Adam's first step moves a parameter by about lr sign(g): compare where
    # the two runs' float atomics cannot flip a sign
    close = np.abs(a - b) <= 1e-6 + 1e-6 * np.abs(a)
    assert close.mean() > 0.999


def test_pair_overflow_raises_in_training_and_autograd():
    """A pair capacity below what the binning needs cuts the tile lists; the
    Trainer's periodic check and the autograd backward both raise instead of
    training on them, and a large enough capacity trains normally."""
    from paper_2503_01199_gb300 import autograd as AG
    d = scenegen.uniform_box_scene(3000, 0, 31, 96, 96, focal=96.0)
    tgt = U.t(d["target"])
    B.lgs_get_overflow()                      # clear the shared flag
    tr = PL.Trainer(d["scene"], 96, 96, PL.StepConfig(pair_capacity=100, overflow_check_every=1))
    with pytest.raises(B.LgsError, match="pair_capacity"):
        tr.step(d["camera"], tgt, reorder=False)
    ok = PL.Trainer(d["scene"], 96, 96, PL.StepConfig(overflow_check_every=1))
    ok.step(d["camera"], tgt, reorder=False)
    planes, n = U.planes_tensor(d["scene"])
    small = AG.GaussianRasterizer(n, 0, 96, 96, pair_capacity=100)
    img = AG.rasterize(planes.requires_grad_(True), d["camera"], small)
    with pytest.raises(B.LgsError, match="pair_capacity"):
        img.sum().backward()
    B.lgs_get_overflow()
    big = AG.GaussianRasterizer(n, 0, 96, 96)
    planes.grad = None
    AG.rasterize(planes, d["camera"], big).sum().backward()
    assert planes.grad is not None and torch.isfinite(planes.grad).all()
