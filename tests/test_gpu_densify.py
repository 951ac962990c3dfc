"""Densification, opacity decay and moment sums on the GPU against the oracle
(Sec. 3.3). Selection and copies are exact; split samples and decayed
logits are FP32 evaluations of the oracle's double-precision values."""
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


def test_densify_matches_oracle(orc):
    n, K, deg = 3000, 300, 1
    sc = scenegen.uniform_box_scene(n, deg, 21, 64, 64, with_target=False)["scene"]
    stride = PL.round_up(n + K, 128)
    planes32 = np.zeros((B.num_planes(deg), stride), np.float32)
    planes32[:, :n] = PL.pack_planes(sc)
    rng = np.random.default_rng(22)
    m32 = np.zeros_like(planes32)
    v32 = np.zeros_like(planes32)
    m32[:, :n] = rng.standard_normal((planes32.shape[0], n)).astype(np.float32)
    v32[:, :n] = rng.uniform(0, 1, (planes32.shape[0], n)).astype(np.float32)
    metric = rng.standard_normal(n).astype(np.float32)
    metric[::11] = metric[5]                                  # ties
    smax = np.exp(planes32[3:6, :n]).max(axis=0)
    split = float(np.float32(np.median(smax)))                 # about half split, half clone
    normals = rng.standard_normal((K, 2, 3)).astype(np.float32)
    tp, tm, tv = U.t(planes32), U.t(m32), U.t(v32)
    g = B.gaussians_struct(tp, n, deg)
    d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    sel = torch.zeros(K, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lgs_densify_workspace_size(n), dtype=torch.uint8, device="cuda")
    B.lgs_densify(g, tm, tv, U.t(metric), K, split, U.t(normals), d_n, sel, ws)
    torch.cuda.synchronize()
    o = orc.densify(planes32.astype(np.float64), m32.astype(np.float64), v32.astype(np.float64),
                    metric.astype(np.float64), K, split, normals.astype(np.float64))
    n_new = int(d_n.item())
    assert n_new == o["n"] == n + K
    gsel = sel.cpu().numpy()[:K].astype(np.int64)
    np.testing.assert_array_equal(gsel, o["selected"])
    P, Mg, Vg = tp.cpu().numpy(), tm.cpu().numpy(), tv.cpu().numpy()
    split_rows = [i for i in gsel if np.exp(planes32[3:6, i].astype(np.float64)).max() > split]
    assert 0 < len(split_rows) < K
    changed = set(split_rows) | set(range(n, n + K))
    keep = np.array([i for i in range(n) if i not in changed])
    np.testing.assert_array_equal(P[:, keep], planes32[:, keep])
    np.testing.assert_array_equal(Mg[:, keep], m32[:, keep])
    rows = sorted(changed)
    # colour, rotation, opacity planes are copies: exact
    np.testing.assert_array_equal(P[6:, rows], o["planes"][6:, rows].astype(np.float32))
    np.testing.assert_allclose(P[3:6, rows], o["planes"][3:6, rows], rtol=0, atol=1e-6)
    np.testing.assert_allclose(P[0:3, rows], o["planes"][0:3, rows], rtol=0, atol=2e-6)
    np.testing.assert_array_equal(Mg[:, rows], o["m"][:, rows].astype(np.float32))
    np.testing.assert_array_equal(Vg[:, rows], o["v"][:, rows].astype(np.float32))


def test_opacity_decay_matches_oracle(orc):
    logit = np.linspace(-40, 40, 4001).astype(np.float32)
    planes = np.zeros((14, 4096), np.float32)
    planes[10, :logit.size] = logit
    tp = U.t(planes)
    B.lgs_opacity_decay(B.gaussians_struct(tp, logit.size, 0))
    torch.cuda.synchronize()
    got = tp.cpu().numpy()[10, :logit.size].astype(np.float64)
    want = orc.opacity_decay(logit.astype(np.float64))
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    np.testing.assert_allclose(sig(got), sig(want), rtol=2e-6, atol=0)
    assert (np.diff(got) >= 0).all()


def test_moments_sum_over_views_and_metric(orc):
    n = 5000
    rng = np.random.default_rng(30)
    S = torch.zeros(n, dtype=torch.float32, device="cuda")
    M = torch.zeros_like(S)
    C = torch.zeros(n, dtype=torch.int32, device="cuda")
    S64, M64, C64 = np.zeros(n), np.zeros(n), np.zeros(n, np.int64)
    for _ in range(3):
        V = int(rng.integers(1000, 4000))
        rows = np.sort(rng.choice(n, V, replace=False)).astype(np.uint32)
        g = np.zeros((n, 16), np.float32)
        g[:V, 9] = rng.uniform(0, 1, V)
        g[:V, 10] = rng.standard_normal(V)
        cnt = rng.integers(0, 50, V).astype(np.uint32)
        g[:V, 11] = cnt.view(np.float32)
        B.lgs_moments_accumulate(U.t(g), U.t(rows.view(np.int32)), U.t(np.array([V], np.int32)), n,
                                 S, M, C)
        orc.moments_accumulate(rows, g[:V, 9], g[:V, 10], cnt.astype(np.int64), S64, M64, C64)
    metric = torch.zeros_like(S)
    B.lgs_moments_metric(S, M, C, n, metric)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.cpu().numpy(), C64)
    np.testing.assert_allclose(S.cpu().numpy(), S64, rtol=1e-6)
    want = orc.opacity_variance(S64, M64, C64)
    assert U.rel_l2(metric.cpu().numpy(), want) < 1e-5


def test_trainer_densify_grows_and_resorts():
    d = scenegen.uniform_box_scene(4096, 1, 3, 96, 96, focal=96.0)
    tr = PL.Trainer(d["scene"], 96, 96, capacity=4096 + 512)
    tr.track_moments = True
    tgt = U.t(d["target"])
    for _ in range(3):
        tr.step(d["camera"], tgt, reorder=False)
    added = tr.densify(400, split_scale=0.05, seed=1)
    torch.cuda.synchronize()
    assert 0 < added <= 400 and tr.n == 4096 + added
    codes = tr.codes.cpu().numpy()[:tr.n].astype(np.uint64)
    assert (np.diff(codes.astype(np.float64)) >= 0).all()      # Morton order after the re-sort
    loss = tr.step(d["camera"], tgt, reorder=False)
    torch.cuda.synchronize()
    assert np.isfinite(float(loss.item()))
    assert np.isfinite(tr.params.cpu().numpy()[:, :tr.n]).all()
