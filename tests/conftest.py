"""Shared pytest setup: the ``gpu`` marker and repo-root imports.

Tests marked ``gpu`` need a CUDA device and the compiled CUDA library; the
rest run on any CPU (``-m "not gpu"``).

With LGS_DEBUG=1 in the environment the binding loads the bounds-checked
build, and after every ``gpu`` test the library's failed-check word is read
(it synchronises the device and clears the word): a test whose kernels
failed a bounds check fails, naming the check's site and source line.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _debug_build_checks(request):
    yield
    if not os.environ.get("LGS_DEBUG") or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2503_01199_gb300 import binding as B
    if getattr(B, "_lib", None) is None:  # the test loaded no library
        return
    code = B.lgs_get_debug_error()
    assert code == 0, f"bounds check failed: site {code >> 32}, line {code & 0xffffffff}"
