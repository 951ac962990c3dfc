"""The give-up path of the bounded device waits (the decoupled look-backs of
the radix sort and of the binning's item kernel).

With the wait limit at 0, every look-back that meets a predecessor that has
not yet published gives up at once: the call still ends, its result is
wrong but every write stays inside its output (a given-up look-back uses a
prefix no larger than the true one; the workspace starts zeroed, so slots
left unwritten hold valid splat indices), the timeout count is non-zero and
lgs_get_wait_timeouts returns LGS_ERR_TIMEOUT. With the default limit
restored, the next call is exact again. Nothing here reads the wrong lists
on the device afterwards.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def _bin(s, W, H):
    n = s["uv"].shape[0]
    rec, d, r = U.pack_splats(s["uv"][:, 0], s["uv"][:, 1], s["conic"], s["opacity"], s["rgb"],
                              s["depth"], s["radius"], tau=s["tau"])
    sp = B.splats_struct(rec, d, r)
    cam = {"R": np.eye(3), "t": np.zeros(3), "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0,
           "width": W, "height": H, "znear": 0.2, "bg": np.zeros(3)}
    gx, gy = -(-W // 16), -(-H // 16)
    cap = 60 * n
    vals = torch.zeros(cap, dtype=torch.int32, device="cuda")
    dP = torch.zeros(1, dtype=torch.int64, device="cuda")
    ranges = torch.zeros((gx * gy, 2), dtype=torch.int32, device="cuda")
    ws = torch.zeros(B.lgs_bin_sort_workspace_size(n, cap, gx * gy), dtype=torch.uint8,
                     device="cuda")
    B.lgs_bin_sort(sp, None, n, B.camera_struct(cam), 16, 16, vals, dP, ranges, ws, tile_cull=1)
    torch.cuda.synchronize()
    P = int(dP.item())
    return (vals.cpu().numpy().view(np.uint32)[:min(P, cap)], ranges.cpu().numpy().view(np.uint32),
            P)


def test_wait_that_gives_up_is_reported_and_the_next_call_is_exact(orc):
    W, H = 1297, 840
    s = U.random_splat_dict(300000, 61, W, H, max_radius=40)
    L = B.load()
    B.lgs_get_wait_timeouts()                     # clear
    try:
        B.lgs_set_wait_limit(0)
        _bin(s, W, H)
        count = ctypes.c_uint32(0)
        assert L.lgs_get_wait_timeouts(ctypes.byref(count)) == B.LGS_ERR_TIMEOUT
        assert count.value > 0
    finally:
        B.lgs_set_wait_limit(B.LGS_DEFAULT_WAIT_LIMIT)
    assert B.lgs_get_wait_timeouts() == 0         # cleared by the read
    vals, ranges, P = _bin(s, W, H)
    assert B.lgs_get_wait_timeouts() == 0
    U.check_bins(orc, vals, ranges, P, s, W, H)
