"""The unit-rate microbenchmarks do the work their operation counts claim:
the reductions land exactly (every row float counts its adds), the FMA
chains follow their closed form, the ex2 chain stays in its interval (it
converges to -1, an attracting fixed point of x <- 2^x - 1.5)."""
import numpy as np
import pytest

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    U.need_gpu()


def test_peak_red_count_is_exact():
    import torch
    from paper_2503_01199_gb300 import binding as B
    rows = torch.zeros((1000, 16), dtype=torch.float32, device="cuda")
    n = B.lgs_peak_red(rows, rows.shape[0], 3, 5)
    torch.cuda.synchronize()
    r = rows.cpu().numpy()
    assert n == 3 * 8 * 12 * 5
    assert r.sum() == n                      # small integers: exact in FP32
    assert (r[:, 12:] == 0).all()            # lanes 12..31 add nothing
    # each (warp, iteration) adds 1 to floats 0..11 of one row
    assert (r[:, :12] == r[:, :1]).all()


@pytest.mark.parametrize("packed", [False, True])
def test_peak_ffma_follows_the_closed_form(packed):
    import torch
    from paper_2503_01199_gb300 import binding as B
    out = torch.empty(2 * B.PEAK_THREADS, dtype=torch.float32, device="cuda")
    iters = 4
    n = B.lgs_peak_ffma(out, 2, iters, packed)
    torch.cuda.synchronize()
    assert n == 2 * B.PEAK_THREADS * B.PEAK_UNROLL * iters * (2 if packed else 1)
    a, b, k = 0.9990234375, 1.0e-3, B.PEAK_UNROLL * iters
    tid = np.arange(B.PEAK_THREADS, dtype=np.float64)

    def chain(x0):  # x_k = a^k x0 + b (1 - a^k) / (1 - a)
        return a ** k * x0 + b * (1 - a ** k) / (1 - a)

    x0 = np.float32(0.001) * tid.astype(np.float32)
    want = chain(x0) + chain(0.5) if packed else chain(x0)
    got = out.cpu().numpy().reshape(2, -1)
    for blk in range(2):
        np.testing.assert_allclose(got[blk], want, rtol=1e-4, atol=1e-5)


def test_peak_ex2_stays_in_its_interval():
    import torch
    from paper_2503_01199_gb300 import binding as B
    out = torch.empty(4 * B.PEAK_THREADS, dtype=torch.float32, device="cuda")
    n = B.lgs_peak_ex2(out, 4, 3)
    torch.cuda.synchronize()
    assert n == 4 * B.PEAK_THREADS * B.PEAK_UNROLL * 3
    x = out.cpu().numpy()
    assert np.isfinite(x).all() and (x >= -1.001).all() and (x <= 0.5).all()
