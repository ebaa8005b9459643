"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (CPU only)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*(dl_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_07607_gb300 import build as B, dl
    B.build()
    return dl.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dl_store_create", "dl_sim_join", "dl_topk_join", "dl_result_pairs", "dl_result_free"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_07607_gb300 import dl
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(dl.EXPORTS) == sorted(set(dl.EXPORTS))
    assert set(names) == set(dl.EXPORTS), set(names) ^ set(dl.EXPORTS)


def test_version_and_defaults(lib):
    from paper_1812_07607_gb300 import dl
    assert b"sm_103a" in lib.dl_version()
    o = dl.dl_join_opts()
    lib.dl_join_opts_default(ctypes.byref(o))
    assert o.precision == dl.DL_PREC_AUTO and o.self_mode == dl.DL_SELF_UPPER and o.out_capacity == 0


def test_argument_validation_without_gpu(lib):
    """Null handles and bad arguments are rejected before any CUDA work."""
    from paper_1812_07607_gb300 import dl
    h = ctypes.c_void_p()
    assert lib.dl_sim_join(None, None, 0, 0.1, None, ctypes.byref(h)) == dl.DL_EINVAL
    assert lib.dl_store_create(ctypes.byref(h), None, None, 5, 0, 0, None) == dl.DL_EINVAL
    assert lib.dl_store_create(ctypes.byref(h), None, None, 5, 2000, 0, None) == dl.DL_EINVAL
    assert lib.dl_store_create(None, None, None, 5, 8, 0, None) == dl.DL_EINVAL
    assert b"d=" in lib.dl_last_error() or b"out" in lib.dl_last_error()


def test_no_cpu_fallback():
    """Without a usable GPU the library fails loudly instead of computing on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_1812_07607_gb300 import build as B, dl
    B.build()
    with pytest.raises(dl.DLError) as ei:
        dl.Store(np.arange(4, dtype=np.int64), np.ones((4, 8), np.float32))
    assert ei.value.status == dl.DL_ECUDA


def test_further_rows_validation_without_gpu(lib):
    """The further rows' entry points reject bad arguments before any CUDA work."""
    from paper_1812_07607_gb300 import dl
    h = ctypes.c_void_p()
    c = ctypes.c_int64()
    ms = ctypes.c_float()
    # colour histograms: bin counts outside [1, 256] or d > 1024, negative sizes, NULL inputs
    for bins in ((0, 1, 1), (257, 1, 1), (16, 16, 8)):
        assert lib.dl_color_hist(None, 1, 8, 8, None, 1, *bins, None, None, None) == dl.DL_EINVAL
    assert lib.dl_color_hist(None, -1, 8, 8, None, 1, 4, 4, 4, None, None, None) == dl.DL_EINVAL
    assert lib.dl_color_hist(None, 1, 8, 8, None, 3, 4, 4, 4, None, ctypes.byref(ms), None) == dl.DL_EINVAL
    assert lib.dl_color_hist(None, 1, 8, 8, None, 0, 4, 4, 4, None, None, None) == dl.DL_OK   # no boxes: no work
    # components: negative sizes, n >= 2^31, NULL arrays; an empty graph needs no GPU
    assert lib.dl_components(-1, None, None, 0, None, ctypes.byref(c), None) == dl.DL_EINVAL
    assert lib.dl_components(1 << 31, None, None, 0, None, ctypes.byref(c), None) == dl.DL_EINVAL
    assert lib.dl_components(5, None, None, 3, None, ctypes.byref(c), None) == dl.DL_EINVAL
    assert lib.dl_components(0, None, None, 0, None, ctypes.byref(c), None) == dl.DL_OK and c.value == 0
    # dedup and clustering: NULL stores and bad plans / cluster counts
    assert lib.dl_dedup(None, 0, 0.1, None, 0, 0, None, None, ctypes.byref(c)) == dl.DL_EINVAL
    assert lib.dl_store_cluster(None, 4, 2, ctypes.byref(h), None) == dl.DL_EINVAL
    # the new metrics are part of the join's metric enum; an unknown metric is rejected
    assert lib.dl_sim_join(None, None, 2, 0.1, None, ctypes.byref(h)) == dl.DL_EINVAL
    assert lib.dl_last_error()
