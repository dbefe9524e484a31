"""The bounds-checked build (DSE_CHECK_BOUNDS, the substitute for a device
memory checker): it compiles from the same sources into its own library and
exports the same entry points; in the normal build the probe reports that
no checks are compiled."""
import ctypes as C
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2602_06986_gb300 import _build

    return _build.build(checked=True)


def test_checked_build_exports_every_entry_point(checked_lib):
    from paper_2602_06986_gb300 import dse

    lib = C.CDLL(checked_lib)
    for name in dse.EXPORTS:
        assert hasattr(lib, name), name


def test_normal_build_has_no_checks():
    from paper_2602_06986_gb300 import _build, dse

    _build.build()
    assert dse.bounds_probe(5, 3) == dse.EINVAL
    assert b"not a bounds-checked build" in dse.lib().dse_last_error()


def test_checked_library_is_selected_by_the_environment(checked_lib):
    code = "from paper_2602_06986_gb300 import dse; print(dse.LIB_PATH)"
    env = dict(os.environ, DSE_LIB_VARIANT="checked")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == checked_lib
