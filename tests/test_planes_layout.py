"""The host side of the parameter layout include/lgs.h fixes: plane k of
Gaussian i at data[k * stride + i], planes 0..2 centre, 3..5 log-scale,
6..9 quaternion (w, x, y, z), 10 opacity logit, 11 + 3k + ch SH coefficient
k of channel ch; 11 + 3 (deg + 1)^2 planes. Checked against the header's
own macro and the per-plane learning rates."""
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2503_01199_gb300 import binding as B
from paper_2503_01199_gb300 import pipeline as PL
from paper_2503_01199_gb300 import scenegen

ROOT = Path(__file__).resolve().parents[1]


def _header_num_planes(deg: int) -> int:
    """The header's LGS_NUM_PLANES(deg), whose text is checked to be
    11 + 3 (deg + 1)^2."""
    text = (ROOT / "include" / "lgs.h").read_text()
    m = re.search(r"#define LGS_NUM_PLANES\(deg\)\s*(\(.*\))", text)
    assert " ".join(m.group(1).split()) == "(11 + 3 * ((deg) + 1) * ((deg) + 1))"
    return 11 + 3 * (deg + 1) * (deg + 1)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_pack_follows_the_header_order(deg):
    d = scenegen.uniform_box_scene(37, deg, 5, 64, 48)
    sc = d["scene"]
    p = PL.pack_planes(sc)
    assert p.shape == (_header_num_planes(deg), 37) == (B.num_planes(deg), 37)
    assert p.dtype == np.float32 and p.flags.c_contiguous
    f32 = lambda a: np.asarray(a, np.float32)
    np.testing.assert_array_equal(p[0:3], f32(sc["mean"]).T)
    np.testing.assert_array_equal(p[3:6], f32(sc["log_scale"]).T)
    np.testing.assert_array_equal(p[6:10], f32(sc["quat"]).T)     # w, x, y, z
    np.testing.assert_array_equal(p[10], f32(sc["logit"]))
    sh = f32(sc["sh"])
    K = (deg + 1) ** 2
    assert sh.shape == (37, K, 3)
    for k in range(K):
        for ch in range(3):
            np.testing.assert_array_equal(p[11 + 3 * k + ch], sh[:, k, ch])
    back = PL.unpack_planes(p, deg)
    for key in ("mean", "log_scale", "quat", "logit", "sh"):
        np.testing.assert_array_equal(back[key], f32(sc[key]))
    assert back["sh_degree"] == deg


def test_header_counts_and_learning_rate_groups():
    assert _header_num_planes(0) == 14 and _header_num_planes(3) == 59
    lr = PL.lr_per_plane(3)
    assert len(lr) == 59
    D = PL.DEFAULT_LR
    assert lr[0:3] == [D["mean"]] * 3 and lr[3:6] == [D["log_scale"]] * 3
    assert lr[6:10] == [D["quat"]] * 4 and lr[10] == D["logit"]
    assert lr[11:14] == [D["sh_dc"]] * 3 and lr[14:] == [D["sh_rest"]] * 45
    assert len(PL.lr_per_plane(0)) == 14
    assert PL.lr_per_plane(1, {"mean": 1.0})[0:3] == [1.0] * 3
