"""The bounds-checked debug build (liblgs_debug.so, LGS_DEBUG): run in a
child process with LGS_DEBUG=1 so that the binding loads it.

- A whole training step (Morton re-sort, cull, preprocess, binning, both
  raster passes, loss, variance, separate preprocess backward and Adam) of
  the 4,096-Gaussian scene passes every check: no failed check is
  recorded, and the image equals the release build's.
- A tile list holding a splat index beyond the splat rows: the raster's
  check catches it before the record is read, skips that entry, and
  lgs_get_debug_error reports site 1 (LGS_ERR_BOUNDS); the release build
  would read past the records.
"""
import json
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

import gpu_util as U

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parents[1]

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, "tests")
from paper_2503_01199_gb300 import binding as B, pipeline as PL, scenegen
import gpu_util as U
L = B.load()
out = {"debug": int(L.lgs_debug_build())}
d = scenegen.uniform_box_scene(4096, 1, 0, 128, 128)
tr = PL.Trainer(d["scene"], 128, 128)
tr.step(d["camera"], U.t(d["target"]), reorder=True, fused=False)
torch.cuda.synchronize()
out["step_error"] = B.lgs_get_debug_error()
out["image"] = tr.image.cpu().numpy().ravel()[::97].tolist()
# a list entry past the splat rows, in the middle of a tile's list
P = int(tr.d_P.item())
ranges = tr.ranges.cpu().numpy().view(np.uint32)
t = int(np.argmax(ranges[:, 1] - ranges[:, 0]))
bad = tr.vals.clone()
bad[int(ranges[t, 0]) + 1] = tr.rec.shape[0] + 5
img = torch.zeros_like(tr.image)
B.lgs_raster_fwd(tr.splats, bad, tr.ranges, B.camera_struct(d["camera"]), 16, 16, img,
                 torch.zeros_like(tr.finalT), torch.zeros_like(tr.last))
torch.cuda.synchronize()
code = B.lgs_get_debug_error()
out["bad_site"] = code >> 32
out["after"] = B.lgs_get_debug_error()
print(json.dumps(out))
'''


def _child(debug: bool):
    env = dict(os.environ, LGS_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def test_debug_build_checks_pass_on_a_valid_step_and_catch_a_bad_list():
    dbg = _child(True)
    assert dbg["debug"] == 1
    assert dbg["step_error"] == 0
    assert dbg["bad_site"] == 1                 # tile-list splat index
    assert dbg["after"] == 0                    # cleared by the read
    rel = _release_image()
    np.testing.assert_array_equal(np.asarray(dbg["image"]), np.asarray(rel))


def _release_image():
    code = CHILD.split("# a list entry past the splat rows")[0] + "print(json.dumps(out))\n"
    env = dict(os.environ, LGS_DEBUG="0")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["debug"] == 0 and out["step_error"] == 0
    return out["image"]
