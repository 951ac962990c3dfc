"""The radix sort behind the Morton re-sort, the depth order and the
densification selection (onesweep with decoupled look-back), on sizes that
span one tile, a ragged tail and thousands of tiles: the permutation must be
numpy's stable argsort of the keys, and no bounded look-back wait may give
up."""
import numpy as np
import pytest
import torch

from paper_2503_01199_gb300 import binding as B

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


@pytest.mark.parametrize("n", [1, 4095, 4097, 100_003, 5_000_000])
def test_morton_sort_is_the_stable_argsort(orc, n):
    rng = np.random.default_rng(n)
    mean = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    if n > 3:
        mean[::7] = mean[3]                                # equal codes: stability
    stride = (n + 127) // 128 * 128
    src = np.zeros((3, stride), np.float32)
    src[:, :n] = mean.T
    ts, td = U.t(src), torch.zeros((3, stride), dtype=torch.float32, device="cuda")
    codes = torch.zeros(n, dtype=torch.int64, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lgs_morton_workspace_size(n), dtype=torch.uint8, device="cuda")
    B.lgs_morton_reorder(ts, td, n, 3, codes, perm, ws)
    torch.cuda.synchronize()
    want_codes = orc.morton_codes(mean)
    want = np.argsort(want_codes, kind="stable")
    np.testing.assert_array_equal(perm.cpu().numpy().view(np.uint32), want)
    np.testing.assert_array_equal(codes.cpu().numpy().view(np.uint64), want_codes[want])
    assert B.lgs_get_wait_timeouts() == 0
