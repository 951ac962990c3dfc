"""The C-ABI library builds, loads and exports every entry point that
include/lgs.h declares, and the Python binding wraps exactly those. No
compute call is made (no GPU needed)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared() -> set[str]:
    text = (ROOT / "include" / "lgs.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(lgs_[a-z0-9_]+)\s*\(", text))


def test_header_declares_the_hot_path():
    names = declared()
    for step in ("lgs_morton_reorder", "lgs_cluster_cull_compact", "lgs_preprocess",
                 "lgs_bin_sort", "lgs_raster_fwd", "lgs_raster_bwd", "lgs_opacity_variance",
                 "lgs_preprocess_bwd", "lgs_adam_step"):
        assert step in names


def test_library_exports_every_declared_symbol():
    from paper_2503_01199_gb300 import binding as B
    B.load()
    lib = ctypes.CDLL(str(B.library_path()))
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(B.ENTRY_POINTS) == declared()
    assert B.lgs_version().startswith("lgs")


def test_invalid_arguments_are_rejected_without_a_gpu():
    from paper_2503_01199_gb300 import binding as B
    L = B.load()
    # null pointers / sizes are refused before anything is enqueued
    assert L.lgs_loss_l1(None, None, 0, None, None, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_morton_reorder(None, None, 0, 0, 0, None, None, None, 0, None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_adam_step(None, None, None, None, 0, 0, None, 0.9, 0.999, 1e-15, 1, None, None, 0,
                           None) == B.LGS_ERR_INVALID_ARG
    assert L.lgs_bin_sort_workspace_size(1000, 100000, 64) > 100000 * 6
