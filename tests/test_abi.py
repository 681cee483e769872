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


def _null_args(argtypes):
    import ctypes as C
    out = []
    for a in argtypes:
        if a is None or a is C.c_void_p or a is C.c_char_p or (isinstance(a, type) and issubclass(a, C._Pointer)):
            out.append(None)
        else:
            out.append(a(0))
    return out


def test_entry_points_reject_null_handles_before_touching_the_gpu():
    # Every status-returning entry point validates its handles and pointers on
    # the host first: called with NULL / zero arguments (here, on a machine
    # without a GPU) each returns FT_EINVAL, and every *_workspace_size returns
    # 0, without a CUDA call.
    from paper_1910_04126_gb300 import _ffi
    lib = _ffi.load()
    status_fns, size_fns = [], []
    for name in declared_functions():
        res, args = _ffi.SIGNATURES[name]
        if res is None or name == "ft_status_string":
            continue
        fn = getattr(lib, name)
        r = fn(*_null_args(fn.argtypes or []))
        if name.endswith("_workspace_size"):
            size_fns.append(name)
            assert r == 0, name
        else:
            status_fns.append(name)
            assert r == -1, (name, r)  # FT_EINVAL
    assert "ft_flowtree_batch" in status_fns and "ft_knn" in status_fns and "ft_read_probe" in status_fns
    assert "ft_flowtree_backward_workspace_size" in size_fns


def test_status_strings_name_every_code():
    from paper_1910_04126_gb300 import _ffi
    lib = _ffi.load()
    for code, name in _ffi.STATUS.items():
        assert lib.ft_status_string(code).decode().split(":")[0] == name
    assert lib.ft_status_string(-99).decode() == "unknown ft_status"


def _header_struct_fields(name):
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return re.findall(r"\b(u?int\d+_t|float|double)\s+([a-z_0-9]+)\s*;", m.group(1))


def test_binding_structs_match_the_header():
    """The ctypes mirrors of the header's by-value structs have the same fields, in order, with the same widths."""
    import ctypes as C
    from paper_1910_04126_gb300 import _ffi
    width = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint32_t": C.c_uint32, "uint64_t": C.c_uint64,
             "float": C.c_float, "double": C.c_double}
    for cname, py in (("ft_flowtree_config", _ffi.FlowtreeConfig), ("ft_tree_info", _ffi.TreeInfo),
                      ("ft_docs_info", _ffi.DocsInfo)):
        fields = _header_struct_fields(cname)
        assert [n for _, n in fields] == [n for n, _ in py._fields_], cname
        assert all(width[t] is ct for (t, _), (_, ct) in zip(fields, py._fields_)), cname
    assert "deep_loads" in [n for n, _ in _ffi.FlowtreeConfig._fields_]
