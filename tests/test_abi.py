"""The C ABI: the library builds for sm_103a and exports every declared entry point.

Runs on the CPU (nvcc cross-compiles; the library loads without a GPU since
it links the CUDA runtime statically).  No compute call is made.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flowtree.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = re.findall(r"\b(ft_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("ft_build_quadtree", "ft_embed_docs", "ft_quadtree_scan", "ft_flowtree_batch",
                 "ft_flowtree_backward", "ft_knn", "ft_flowtree_plain", "ft_topk_f32"):
        assert must in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_1910_04126_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1910_04126_gb300 import _ffi
    assert set(declared_functions()) <= set(_ffi.SIGNATURES)
