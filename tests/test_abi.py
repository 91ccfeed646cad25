"""The C-ABI library builds, loads and exports every entry point include/mms.h
declares; host-side logic (planner, workspace sizing, argument checks) runs
without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mms.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1702_07961_gb300 import _build_lib
    import paper_1702_07961_gb300 as mms
    _build_lib.build()
    return mms.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mms_\w+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for must in ["mms_sort_keys", "mms_sort_pairs", "mms_sort_workspace_bytes", "mms_tile_sort",
                 "mms_splitter", "mms_merge_pass", "mms_status_string"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in mms.h but not exported"


def test_tile_geometry(lib):
    import paper_1702_07961_gb300 as mms
    assert mms.tile_items(mms.KEY_U32) == 8192
    assert mms.tile_items(mms.KEY_F32) == 8192
    assert mms.tile_items(mms.KEY_U64) == 4096


@pytest.mark.parametrize("base", [0, 8192, 16384, 65536])
def test_planner_round_count_is_ceil_log_k(base):
    """ceil(log_K(N / run)) merge rounds (Sec. 6.2), run = the base case's runs."""
    import math
    import paper_1702_07961_gb300 as mms
    for n in [1, 8192, 8193, 10**6, 10**8, 2**28]:
        run = mms.base_run_items(mms.KEY_U32, n, base_items=base)
        assert run == (base or 8192)
        runs = -(-n // run)
        for K in [2, 4, 8, 16, 32]:
            want = 0 if runs <= 1 else math.ceil(math.log(runs) / math.log(K) - 1e-12)
            got = mms.plan(mms.KEY_U32, n, K, base_items=base)
            assert len(got) == want and all(k == K for k in got)
        auto = mms.plan(mms.KEY_U32, n, base_items=base)
        prod = 1
        for k in auto:
            assert 2 <= k <= 32
            prod *= k
        assert prod >= runs and (not auto or prod // min(auto) < runs)


def test_base_run_items(lib):
    """Runs of the base case: one CTA tile by default, 2, 4 or 8 tiles (a
    cluster) on request for 4-byte keys; invalid settings give 0."""
    import paper_1702_07961_gb300 as mms
    assert mms.base_run_items(mms.KEY_U32, 10**8) == 8192
    assert mms.base_run_items(mms.KEY_F32, 8193) == 8192
    assert mms.base_run_items(mms.KEY_U64, 10**8) == 4096
    assert mms.base_run_items(mms.KEY_U32, 10**8, tile_items=4096) == 4096
    assert mms.base_run_items(mms.KEY_U32, 10**8, tile_items=8192, base_items=32768) == 32768
    assert mms.base_run_items(mms.KEY_F32, 10**8, base_items=16384) == 16384
    assert mms.base_run_items(mms.KEY_U32, 10**8, base_items=65536) == 65536
    assert mms.base_run_items(mms.KEY_U32, 10**8, base_items=12288) == 0
    assert mms.base_run_items(mms.KEY_U64, 10**8, base_items=16384) == 0
    assert mms.base_run_items(mms.KEY_U32, 10**8, tile_items=4096, base_items=32768) == 0


def test_workspace_grows_with_n(lib):
    import paper_1702_07961_gb300 as mms
    a = mms.workspace_bytes(mms.KEY_U32, 10**6)
    b = mms.workspace_bytes(mms.KEY_U32, 2 * 10**6)
    c = mms.workspace_bytes(mms.KEY_U64, 10**6)
    assert 4 * 10**6 < a < b and c > a
    assert mms.workspace_bytes(mms.KEY_U32, 10**6, True) >= a + 4 * 10**6


def test_argument_checks_need_no_gpu(lib):
    # null keys, keys not aligned to the key size, bad fanout: rejected before any CUDA call
    assert lib.mms_sort_keys(0, None, 100, None, 0, None) == 1
    assert lib.mms_sort_keys(0, ctypes.c_void_p(2), 100, None, 0, None) == 1       # u32 at 2 bytes
    assert lib.mms_sort_keys(1, ctypes.c_void_p(4), 100, None, 0, None) == 1       # u64 at 4 bytes
    assert lib.mms_sort_pairs(0, ctypes.c_void_p(256), ctypes.c_void_p(6), 100, None, 0, None) == 1
    assert lib.mms_tile_sort(2, ctypes.c_void_p(258), ctypes.c_void_p(256), 100, None) == 1
    assert lib.mms_sort_keys(7, ctypes.c_void_p(256), 100, None, 0, None) == 1
    assert lib.mms_sort_keys(0, None, 1, None, 0, None) == 0       # n <= 1 is a no-op
    assert lib.mms_splitter(2, ctypes.c_void_p(256), 100, 8192, 4, ctypes.c_void_p(256), None) == 2
    assert lib.mms_splitter(0, ctypes.c_void_p(256), 100, 1000, 4, ctypes.c_void_p(256), None) == 1
    assert lib.mms_splitter(0, ctypes.c_void_p(256), 100, 8192, 33, ctypes.c_void_p(256), None) == 1
    assert lib.mms_status_string(5) == b"device-side wait timed out"


def test_splitter_rows_count_tiles(lib):
    import paper_1702_07961_gb300 as mms
    # two full groups of 4 runs of 8192 and a ragged third group of 1.5 runs
    n = 2 * 4 * 8192 + 8192 + 4096
    assert mms.splitter_rows(mms.KEY_U32, n, 8192, 4) == 4 + 4 + 2
