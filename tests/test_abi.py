"""The C-ABI library loads and exports every entry point include/wg.h declares
(no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(wg_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2607_17571_gb300 import build
    try:
        return build.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this machine
        if os.path.exists(build.LIB):
            return build.LIB
        pytest.skip(f"libwg.so cannot be built here: {e}")


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("wg_relation_load", "wg_tc", "wg_sg", "wg_submit", "wg_poll", "wg_result_copy"):
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2607_17571_gb300 import wg
    assert sorted(wg.SIGNATURES) == declared_functions()
    wg.load_library(lib_path)


def test_binding_struct_sizes_match_header():
    from paper_2607_17571_gb300 import wg
    # sizes fixed by the field lists in wg.h (natural alignment, LP64)
    assert ctypes.sizeof(wg.wg_opts) == 32
    assert ctypes.sizeof(wg.wg_status) == 48
    assert ctypes.sizeof(wg.wg_request) == 48
    assert ctypes.sizeof(wg.wg_kernel_stat) == 56


def test_init_without_gpu_fails_cleanly(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_17571_gb300 import wg
    with pytest.raises(wg.WgError):
        wg.Context(0, torch_memory=False)
