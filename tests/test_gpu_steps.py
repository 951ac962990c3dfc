"""GPU parity of each hot-path step against the CPU oracle, called through
the C ABI (via the binding) on seeded inputs shared by both sides.

Tolerances:
  * integer work (Morton codes, sort permutations, tile lists and ranges,
    compaction maps, radii, last-contributor indices, fragment counts):
    bit-exact, except where the oracle flags a decision within rounding of
    its threshold (counted, and required to be rare);
  * images: 1e-5 max-abs on unflagged pixels;
  * gradients: 1e-3 relative L2 (atomic summation order);
  * preprocess outputs (single precision against double): relative 1e-5 on
    positions and colours, 1e-4 of the conic's norm (the 2x2 inverse
    amplifies rounding by its condition number).
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


# ---------------------------------------------------------------------------
# a3 preprocess
# ---------------------------------------------------------------------------
def _cmp_preprocess(gp, op, flags):
    ok = flags == 0
    vis_o = op["radius"] > 0
    vis_g = gp["radius"] > 0
    assert (vis_o[ok] == vis_g[ok]).all()
    np.testing.assert_array_equal(gp["radius"][ok], op["radius"][ok])
    m = ok & vis_o & vis_g
    assert m.sum() > 0.5 * vis_o.sum()
    np.testing.assert_allclose(gp["uv"][m], op["uv"][m], rtol=1e-5, atol=2e-4)
    np.testing.assert_allclose(gp["depth"][m], op["depth"][m], rtol=1e-6)
    np.testing.assert_allclose(gp["opacity"][m], op["opacity"][m], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(gp["rgb"][m], op["rgb"][m], rtol=1e-5, atol=1e-6)
    cn = np.linalg.norm(op["conic"][m], axis=1, keepdims=True)
    assert (np.abs(gp["conic"][m] - op["conic"][m]) <= 1e-4 * cn).all()
    return int((~ok).sum())


@pytest.mark.parametrize("deg", [0, 3])
def test_preprocess_matches_oracle(orc, deg):
    d = scenegen.uniform_box_scene(4096, deg, 0, 128, 128)
    op = orc.preprocess(d["scene"], d["camera"])
    gp = U.gpu_preprocess(d["scene"], d["camera"])
    flagged = _cmp_preprocess(gp, op, op["flags"])
    assert flagged < 10


def test_preprocess_through_map_and_device_count(orc):
    d = scenegen.surface_scene(6000, 3, 1, 320, 200)
    rng = np.random.default_rng(0)
    rowmap = rng.permutation(6000)[:4000].astype(np.uint32)
    V = 3500
    op = orc.preprocess(d["scene"], d["camera"])
    gp = U.gpu_preprocess(d["scene"], d["camera"], rowmap=rowmap, V=V)
    sel = rowmap[:V]
    sub = {k: op[k][sel] for k in op}
    _cmp_preprocess(gp, sub, sub["flags"])


def test_preprocess_backward_matches_oracle(orc):
    d = scenegen.uniform_box_scene(3000, 3, 3, 160, 120)
    sc, cam = d["scene"], d["camera"]
    sc["log_scale"][:50] += 2.5   # some large Gaussians to reach the clamp branch
    g9 = np.random.default_rng(1).standard_normal((3000, 9)).astype(np.float32)
    ref = orc.grad_planes(orc.preprocess_bwd(sc, cam, g9))
    planes, n = U.planes_tensor(sc)
    g = B.gaussians_struct(planes, n, 3)
    gacc = np.zeros((n, 16), np.float32)
    gacc[:, :9] = g9
    out = torch.zeros_like(planes)
    B.lgs_preprocess_bwd(g, None, None, B.camera_struct(cam), U.t(gacc), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()[:, :n]
    # per parameter group: 1e-3 relative L2
    for name, sl in (("mean", slice(0, 3)), ("log_scale", slice(3, 6)), ("quat", slice(6, 10)),
                     ("logit", slice(10, 11)), ("sh", slice(11, None))):
        e = U.rel_l2(got[sl], ref[sl])
        assert e < 1e-3, (name, e)


# ---------------------------------------------------------------------------
# a1 Morton, a2 cluster cull + compaction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gen,n", [("box", 50000), ("surface", 70001)])
def test_morton_reorder_bit_exact(orc, gen, n):
    d = (scenegen.uniform_box_scene(n, 1, 4, 64, 64) if gen == "box"
         else scenegen.surface_scene(n, 1, 5, 64, 64))
    sc = d["scene"]
    codes_ref, perm_ref = orc.morton_reorder(sc)
    planes, n_ = U.planes_tensor(sc)
    dst = torch.zeros_like(planes)
    codes = torch.zeros(n, dtype=torch.int64, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lgs_morton_workspace_size(n), dtype=torch.uint8, device="cuda")
    B.lgs_morton_reorder(planes, dst, n, planes.shape[0], codes, perm, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(codes.cpu().numpy().view(np.uint64), codes_ref)
    np.testing.assert_array_equal(perm.cpu().numpy().view(np.uint32), perm_ref)
    src = planes.cpu().numpy()
    np.testing.assert_array_equal(dst.cpu().numpy()[:, :n], src[:, :n][:, perm_ref])


@pytest.mark.parametrize("gen", ["box", "surface"])
def test_cluster_cull_compact_matches_oracle(orc, gen):
    if gen == "box":
        d = scenegen.uniform_box_scene(30000, 0, 6, 200, 150)
        d["scene"]["mean"][:10000, 0] += 5.0
        d["scene"]["mean"][10000:15000, 2] -= 5.0
    else:
        d = scenegen.surface_scene(100003, 0, 7, 320, 240)
    sc, cam = d["scene"], d["camera"]
    _, perm = orc.morton_reorder(sc)
    sc = {k: (v[perm] if k != "sh_degree" else v) for k, v in sc.items()}
    ref = orc.cluster_cull(sc, cam, 128)
    planes, n = U.planes_tensor(sc)
    g = B.gaussians_struct(planes, n, 0)
    ncl = -(-n // 128)
    aabb = torch.zeros((ncl, 6), dtype=torch.float32, device="cuda")
    vis = torch.zeros(ncl, dtype=torch.int32, device="cuda")
    rowmap = torch.zeros(n, dtype=torch.int32, device="cuda")
    dV = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lgs_ccc_workspace_size(n, 128), dtype=torch.uint8, device="cuda")
    B.lgs_cluster_cull_compact(g, B.camera_struct(cam), 128, aabb, vis, rowmap, dV, ws)
    torch.cuda.synchronize()
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    vis_g = vis.cpu().numpy()
    np.testing.assert_array_equal(vis_g[ok], ref["visible"][ok])
    np.testing.assert_allclose(aabb.cpu().numpy(), ref["aabb"], rtol=1e-5, atol=1e-5)
    V = int(dV.item())
    # the map lists whole visible clusters in increasing order
    vv = np.flatnonzero(vis_g)
    expect = np.concatenate([np.arange(c * 128, min(c * 128 + 128, n)) for c in vv]) if vv.size else np.zeros(0)
    assert V == expect.size
    np.testing.assert_array_equal(rowmap.cpu().numpy()[:V].view(np.uint32), expect.astype(np.uint32))
    if ok.all():
        assert V == ref["V"]
        np.testing.assert_array_equal(rowmap.cpu().numpy()[:V].view(np.uint32), ref["map"])


@pytest.mark.parametrize("case", ["side_planes", "widening"])
def test_cluster_cull_closed_form_cases(orc, case):
    """The closed-form cull cases of the oracle's pins (each of the five
    planes, a relative 1e-3 inside and outside; the 3 x largest-scale
    widening 2e-3 above and below the reach needed) through the kernel:
    the same flags as the closed form and the oracle."""
    import cull_cases as CC
    geo, want = CC.side_plane_scene() if case == "side_planes" else CC.widening_scene()
    n = geo["mean"].shape[0]
    quat = np.zeros((n, 4), np.float32)
    quat[:, 0] = 1.0
    sc = {"mean": geo["mean"].astype(np.float32), "log_scale": geo["log_scale"].astype(np.float32),
          "quat": quat, "logit": np.zeros(n, np.float32), "sh": np.zeros((n, 1, 3), np.float32),
          "sh_degree": 0}
    cam = CC.camera()
    ref = orc.cluster_cull(sc, cam, CC.CLUSTER)
    np.testing.assert_array_equal(ref["visible"], want)
    planes, n = U.planes_tensor(sc)
    g = B.gaussians_struct(planes, n, 0)
    ncl = -(-n // CC.CLUSTER)
    aabb = torch.zeros((ncl, 6), dtype=torch.float32, device="cuda")
    vis = torch.zeros(ncl, dtype=torch.int32, device="cuda")
    rowmap = torch.zeros(n, dtype=torch.int32, device="cuda")
    dV = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lgs_ccc_workspace_size(n, CC.CLUSTER), dtype=torch.uint8, device="cuda")
    B.lgs_cluster_cull_compact(g, B.camera_struct(cam), CC.CLUSTER, aabb, vis, rowmap, dV, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(vis.cpu().numpy(), want)
    assert int(dV.item()) == CC.CLUSTER * int(want.sum())


# ---------------------------------------------------------------------------
# a4 bin sort
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cull", [0, 1])
@pytest.mark.parametrize("n,W,H,tile", [(4096, 128, 128, (16, 16)), (50000, 1297, 840, (16, 16)),
                                        (3000, 200, 77, (16, 16)), (1, 64, 64, (16, 16)),
                                        (20000, 1600, 1063, (16, 16))])
def test_bin_sort_bit_exact(orc, n, W, H, tile, cull):
    s = U.random_splat_dict(n, 10 + n, W, H, max_radius=40)
    s["radius"][::13] = 0
    s["tau"][::17] = -np.inf                        # splats that reach no pixel
    vals, ranges, P = U.gpu_bin(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], W, H, tile,
                                conic=s["conic"], tau=s["tau"], cull=cull)
    U.check_bins(orc, vals, ranges, P, s, W, H, tile, cull=cull)


def test_bin_keys_of_the_tile_lists():
    """lgs_bin_keys: every pair's 64-bit key is (tile << 32 | depth bits of
    its splat), non-decreasing within each tile's range (the depth order
    of the list); an empty binning writes nothing."""
    import torch
    from paper_2503_01199_gb300 import binding as B
    cam = scenegen.pinhole_camera(200, 150, 200.0)
    sp = U.random_splat_dict(3000, 31, 200, 150, max_radius=30)
    g = U.gpu_raster(sp, cam)
    dev, P = g["dev"], int(g["P"])
    keys = torch.full((P + 1,), -1, dtype=torch.int64, device="cuda")
    B.lgs_bin_keys(dev["splats"], dev["vals"], dev["ranges"], keys)
    torch.cuda.synchronize()
    k = keys.cpu().numpy().view(np.uint64)
    assert k[P] == np.uint64(0xffffffffffffffff)               # nothing past the pairs
    vals, ranges = g["vals"], g["ranges"].reshape(-1, 2)
    depth_bits = sp["depth"].astype(np.float32).view(np.uint32).astype(np.uint64)
    seen = 0
    for t, (r0, r1) in enumerate(ranges):
        seg = k[r0:r1]
        assert (seg >> np.uint64(32) == np.uint64(t)).all()
        assert (seg & np.uint64(0xffffffff) == depth_bits[vals[r0:r1]]).all()
        assert (seg[1:] >= seg[:-1]).all()                     # unsigned: no np.diff
        seen += r1 - r0
    assert seen == P > 0


@pytest.mark.parametrize("cull", [0, 1])
def test_bin_sort_large_and_degenerate_splats(orc, cull):
    """Splats up to 600 px: groups of 32 splats with more tile rows than the
    shared-memory spans hold and more super-tile items than the staged
    output holds (the per-lane and direct-write paths of the item kernel);
    conics whose det is 0 or negative after rounding (the per-tile box test);
    thin ellipses (an axis ratio up to 1000)."""
    W, H = 1297, 840
    s = U.random_splat_dict(4000, 77, W, H, max_radius=600)
    conic = s["conic"].astype(np.float64)
    A, C = conic[:, 0], conic[:, 2]
    conic[::7, 1] = np.sqrt(A[::7] * C[::7])            # det = 0 (rounds to 0 or below)
    conic[3::11, 1] = 1.5 * np.sqrt(A[3::11] * C[3::11])  # det < 0
    thin = np.arange(5, 4000, 13)
    conic[thin, 0] *= 1e3                                # axis ratio up to ~1000
    s["conic"] = conic.astype(np.float32)
    s["radius"][::29] = 0
    vals, ranges, P = U.gpu_bin(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], W, H,
                                (16, 16), conic=s["conic"], tau=s["tau"], cull=cull,
                                cap=64_000_000)
    _, _, rP = U.check_bins(orc, vals, ranges, P, s, W, H, (16, 16), cull=cull)
    assert rP > 100_000
    assert B.lgs_get_wait_timeouts() == 0


def test_bin_sort_empty_and_device_count(orc):
    s = U.random_splat_dict(5000, 3, 300, 200)
    s["radius"][:] = 0
    vals, ranges, P = U.gpu_bin(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], 300, 200)
    assert P == 0 and (ranges == 0).all()
    s = U.random_splat_dict(5000, 4, 300, 200)
    V = 1234
    vals, ranges, P = U.gpu_bin(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], 300, 200, V=V)
    rv, rr, rP = orc.bin_splats(s["uv"][:V, 0], s["uv"][:V, 1], s["radius"][:V], s["depth"][:V], 300, 200)
    assert P == rP
    U.assert_same_tile_lists(vals, ranges, rv, rr)


def test_bin_sort_overflow_is_reported(orc):
    s = U.random_splat_dict(2000, 5, 256, 256)
    B.lgs_get_overflow()  # clear
    _, _, rP = orc.bin_splats(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], 256, 256)
    vals, ranges, P = U.gpu_bin(s["uv"][:, 0], s["uv"][:, 1], s["radius"], s["depth"], 256, 256,
                                cap=rP // 3)
    assert P == rP
    assert B.lgs_get_overflow() == rP
    assert B.lgs_get_overflow() == 0


# ---------------------------------------------------------------------------
# a5 forward, a7 backward on shared float32 splats
# ---------------------------------------------------------------------------
@pytest.fixture
def shared_margins(orc):
    # both sides read the same float32 splats: only the exponent's rounding
    # and exp() separate the kernel's alpha from the oracle's
    orc.set_margins(*orc.MARGINS_SHARED_SPLATS)
    yield
    orc.set_margins(*orc.MARGINS_END_TO_END)


def _raster_case(orc, sp, cam, tile=(16, 16), seed=0, min_ok=0.995):
    W, H = cam["width"], cam["height"]
    w = np.random.default_rng(seed).standard_normal((3, H, W)).astype(np.float32) * 1e-3
    g = U.gpu_raster(sp, cam, tile, dLdI=w)
    vals, ranges, P = U.check_bins(orc, g["vals"], g["ranges"], g["P"], sp, W, H, tile)
    o = orc.render_fwd(sp, vals, ranges, cam, tile)
    ok = o["pixflags"] == 0
    assert ok.mean() > min_ok, ok.mean()
    err = np.abs(g["image"] - o["image"])[:, ok].max()
    assert err <= 1e-5, err
    np.testing.assert_array_equal(U.last_ids(g["last"], g["vals"], g["ranges"], W, tile)[ok],
                                  U.last_ids(o["last"], vals, ranges, W, tile)[ok])
    np.testing.assert_allclose(g["T"][ok], o["T"][ok], rtol=2e-5, atol=1e-7)
    ob = orc.render_bwd(sp, vals, ranges, cam, w, tile)
    names = ["du", "dv", "dA", "dB", "dC", "do", "dr", "dg", "db"]
    for q, nm in enumerate(names):
        e = U.rel_l2(g["grad9"][:, q], ob["grad9"][:, q])
        assert e < 1e-3, (nm, e)
    assert U.rel_l2(g["S"], ob["S"]) < 1e-3
    assert U.rel_l2(g["M"], ob["M"]) < 1e-3
    sok = ob["sflags"] == 0
    np.testing.assert_array_equal(g["C"][sok], ob["C"][sok])
    assert (g["pad"] == 0).all()
    return g, o, ob


def test_tile_culling_keeps_the_image_bit_identical(orc):
    cam = scenegen.pinhole_camera(320, 240, 320.0, bg=(0.2, 0.3, 0.1))
    sp = U.random_splat_dict(20000, 25, 320, 240, max_radius=40)
    w = np.random.default_rng(26).standard_normal((3, 240, 320)).astype(np.float32) * 1e-3
    a = U.gpu_raster(sp, cam, dLdI=w, cull=0)
    b = U.gpu_raster(sp, cam, dLdI=w, cull=1)
    assert b["P"] < 0.8 * a["P"]
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["T"], b["T"])
    # the last contributor is the same splat (list positions differ)
    np.testing.assert_array_equal(U.last_ids(a["last"], a["vals"], a["ranges"], 320),
                                  U.last_ids(b["last"], b["vals"], b["ranges"], 320))
    for q in range(9):
        assert U.rel_l2(b["grad9"][:, q], a["grad9"][:, q]) < 1e-5
    np.testing.assert_array_equal(a["C"], b["C"])


def test_raster_random_splats(orc, shared_margins):
    cam = scenegen.pinhole_camera(200, 150, 200.0, bg=(0.1, 0.2, 0.3))
    sp = U.random_splat_dict(3000, 21, 200, 150, max_radius=30)
    _raster_case(orc, sp, cam)


def test_raster_config1_scene(orc, shared_margins):
    # the 4,096-Gaussian, 128 x 128 case: oracle splats rounded to float32
    d = scenegen.uniform_box_scene(4096, 0, 0, 128, 128)
    sp = U.f32_splats(orc.preprocess(d["scene"], d["camera"]))
    _raster_case(orc, sp, d["camera"])


def test_raster_ragged_image_and_empty_tiles(orc, shared_margins):
    cam = scenegen.pinhole_camera(77, 45, 60.0, bg=(0.5, 0.25, 0.125))
    sp = U.random_splat_dict(60, 22, 40, 20, max_radius=12)   # only the top-left has splats
    g, o, _ = _raster_case(orc, sp, cam)
    bg = np.array([0.5, 0.25, 0.125], np.float32)
    empty = o["last"] == 0
    assert empty.sum() > 1000
    np.testing.assert_array_equal(g["image"][:, empty], np.broadcast_to(bg[:, None], (3, empty.sum())))


def test_raster_dense_opaque_stack(orc, shared_margins):
    # many overlapping high-opacity splats: long lists, early termination and
    # the 0.99 clamp (opacities above 0.99 clamp near their centres)
    cam = scenegen.pinhole_camera(96, 96, 96.0)
    sp = U.random_splat_dict(4000, 23, 96, 96, max_radius=24)
    sp["opacity"] = np.random.default_rng(24).uniform(0.9, 1.0, 4000).astype(np.float32)
    sp["tau"] = U.tau_of(sp["opacity"])   # the record's tau follows its opacity
    # two clamped splats leave T = (1 - 0.99)^2, exactly the 1e-4 stop
    # threshold, which rounding decides: those pixels are flagged
    _raster_case(orc, sp, cam, min_ok=0.9)


def test_raster_backward_integer_warp_reduction(orc, shared_margins):
    # the integer warp sums (Sec. 3.1) give the oracle's gradients within the
    # FP32 tolerance and the float warp sums within the truncation bound
    cam = scenegen.pinhole_camera(200, 150, 200.0, bg=(0.1, 0.2, 0.3))
    sp = U.random_splat_dict(3000, 27, 200, 150, max_radius=30)
    W, H = cam["width"], cam["height"]
    w = np.random.default_rng(28).standard_normal((3, H, W)).astype(np.float32) * 1e-3
    f = U.gpu_raster(sp, cam, dLdI=w)
    g = U.gpu_raster(sp, cam, dLdI=w, precision=B.LGS_WARP_REDUCE_INT)
    np.testing.assert_array_equal(f["image"], g["image"])
    vals, ranges, P = orc.bin_splats(sp["uv"][:, 0], sp["uv"][:, 1], sp["radius"], sp["depth"], W, H,
                                     (16, 16), conic=sp["conic"], tau=sp["tau"])
    ob = orc.render_bwd(sp, vals, ranges, cam, w, (16, 16))
    for q in range(9):
        assert U.rel_l2(g["grad9"][:, q], ob["grad9"][:, q]) < 1e-3, q
        assert U.rel_l2(g["grad9"][:, q], f["grad9"][:, q]) < 1e-5, q
    assert U.rel_l2(g["S"], ob["S"]) < 1e-3 and U.rel_l2(g["M"], ob["M"]) < 1e-3
    np.testing.assert_array_equal(g["C"], f["C"])
