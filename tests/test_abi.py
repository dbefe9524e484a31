"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every entry point include/dse.h declares; without a GPU every computing call
fails loudly with DSE_ECUDA (there is no CPU fallback)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dse.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dse_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def dse():
    from paper_2602_06986_gb300 import _build

    _build.build()
    from paper_2602_06986_gb300 import dse as m

    m.lib()
    return m


def test_every_declared_symbol_is_exported(dse):
    names = declared_functions()
    assert "dse_build_space" in names and "dse_sis_screen" in names and "dse_topk_fetch" in names
    lib = C.CDLL(dse.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(dse.EXPORTS) == set(names)


def test_struct_layouts_match_header(dse):
    # sizes implied by the header's field lists (LP64)
    assert C.sizeof(dse.SpaceDesc) == 8 * 2 + 4 * 2 + 8 + 8 + 4 * 2 + 8 + 8 + 4 * 4 + 8 * 2 + 8 + 8 * 2
    assert C.sizeof(dse.ScreenDesc) == 8 + 8 + 4 * 2 + 8 + 4 * 2 + 8 * 2 + 8 + 4 * 2 + 8 + 8 + 8
    assert C.sizeof(dse.Stats) == 8 + 8 * 6 + 8 * 4 + 4 * 2 + 8 + 8 * 3 + 8 * 4 + 8 + 8 + 4 * 2
    assert C.sizeof(dse.Expr) == 4 * 2 + 8 * 2
    assert C.sizeof(dse.RefitDesc) == 8 + 4 * 2 + 8 + 8 + 8 + 4 * 2 + 8
    assert C.sizeof(dse.BatchItem) == 8 + 8 + 4 * 2
    assert C.sizeof(dse.BatchDesc) == 8 + 4 * 2 + 8
    assert C.sizeof(dse.LoopDesc) == 8 + 4 * 2 + 8 + 4 * 2 + 8 + 4 * 2 + 8
    assert C.sizeof(dse.L0Desc) == 8 + 4 * 2 + 8 + 8 + 4 * 2 + 8
    assert C.sizeof(dse.LoopResult) == 8 * 4 + 8 * 4 + 8 * 20 + 4 * C.sizeof(dse.Stats)


def test_version_and_null_arguments(dse):
    assert "sm_103a" in dse.version()
    L = dse.lib()
    assert L.dse_build_space(None, None) == dse.EINVAL
    assert b"null" in L.dse_last_error()
    assert L.dse_sis_screen(None, None, None) == dse.EINVAL
    assert L.dse_topk_fetch(None, 0, None, None, None, 0, None) == dse.EINVAL
    assert L.dse_sis_screen_batched(None, 0, None, None) == dse.EINVAL
    assert L.dse_batch_rescreen(None, None, 0) == dse.EINVAL
    assert L.dse_batch_fetch(None, 0, None, None, None, 0, None) == dse.EINVAL
    assert L.dse_batch_stats(None, 0, None) == dse.EINVAL
    L.dse_batch_free(None)
    assert L.dse_residual_loop(None, None, None, None, None) == dse.EINVAL
    assert L.dse_l0_search(None, None, None, None, None, None) == dse.EINVAL


def test_invalid_descriptor_rejected_before_device(dse):
    X = np.ones((2, 4))
    with pytest.raises(dse.DseError) as e:
        dse.Space(X, None, 0, 2)  # empty op mask
    assert e.value.status == dse.EINVAL
    with pytest.raises(dse.DseError) as e:
        dse.Space(X, None, 1 << 8, 9)  # rung beyond the supported maximum
    assert e.value.status == dse.EINVAL
    with pytest.raises(dse.DseError) as e:
        dse.Space(X, None, 1 << 8, 2, fmax_max=float("inf"))
    assert e.value.status == dse.EINVAL


def test_no_cpu_fallback(dse):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X = np.random.default_rng(0).uniform(0.5, 2, size=(3, 8))
    with pytest.raises(dse.DseError) as e:
        dse.Space(X, None, 1 << 8, 2)
    assert e.value.status == dse.ECUDA
    # the wait probe and the peak probe need the device too
    assert dse.check_wait(10, arrive=True) == dse.ECUDA
    with pytest.raises(dse.DseError) as e:
        dse.measure_peaks()
    assert e.value.status == dse.ECUDA
    assert dse.check_wait(0, arrive=True) == dse.EINVAL


def test_binding_constants_match_header(dse):
    """Every DSE_* constant the binding mirrors has the header's value."""
    import re

    text = open(HEADER).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define DSE_(\w+) (\d+)", text)}
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"DSE_(\w+) = (\d+)", text)}
    for name in ("FLAG_TIMING", "FLAG_DEDUP", "FLAG_DIRECT", "FLAG_TIMING_MAIN", "PATH_CUDA_CORE", "PATH_TENSOR",
                 "PATH_GRAM", "PATH_GRAM_MT"):
        assert getattr(dse, name) == defines[name], name
    for name in ("PREC_FP32", "PREC_FP64"):
        assert getattr(dse, name) == enums[name], name
