"""The C-ABI library builds, loads and exports every symbol ``include/srk.h``
declares; the Python binding exposes the same names (CPU only: no compute
call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srk.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srk_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("srk_graph_load", "srk_graph_free", "srk_single_source",
                     "srk_multi_source", "srk_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_the_same_names(lib):
    import paper_2304_04015_gb300 as srk
    for name in declared_functions():
        assert callable(getattr(srk, name)), name


def test_last_error_starts_empty(lib):
    lib.srk_last_error.restype = ctypes.c_char_p
    assert lib.srk_last_error() in (b"",)


def test_graph_load_refuses_both_layouts(lib):
    import numpy as np
    import paper_2304_04015_gb300 as srk
    rp = np.array([0, 1], dtype=np.int32)
    col = np.array([0], dtype=np.int32)
    out = ctypes.c_void_p()
    flags = srk.SRK_ADJ_NARROW | srk.SRK_ADJ_WIDE
    assert lib.srk_graph_load(rp.ctypes.data_as(ctypes.c_void_p),
                              col.ctypes.data_as(ctypes.c_void_p), 1, 1, flags, None,
                              ctypes.byref(out)) == srk.SRK_EINVAL
    lib.srk_last_error.restype = ctypes.c_char_p
    assert b"exclude each other" in lib.srk_last_error()


def test_graph_load_rejects_bad_arguments_without_touching_the_device(lib):
    # argument checks run before any CUDA call
    import paper_2304_04015_gb300 as srk
    out = ctypes.c_void_p()
    assert lib.srk_graph_load(None, None, 0, 0, 0, None, ctypes.byref(out)) == srk.SRK_EINVAL
    assert lib.srk_graph_load(None, None, 5, -1, 0, None, ctypes.byref(out)) == srk.SRK_EINVAL
    assert lib.srk_graph_load(None, None, 5, 0, 0, None, None) == srk.SRK_EINVAL
    assert b"out is null" in lib.srk_last_error()
    assert lib.srk_single_source(None, 0, ctypes.c_double(0.6), ctypes.c_double(0.1),
                                 ctypes.c_uint64(1), None, None, None, None, None) == srk.SRK_EINVAL


def test_null_handles_are_refused_on_the_host(lib):
    # every entry point checks its handle or output pointer before any CUDA
    # call; releasing NULL is allowed
    import paper_2304_04015_gb300 as srk
    L = srk._lib
    n, m, lay, adm = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    src = (ctypes.c_int32 * 1)(0)
    eps = (ctypes.c_double * 1)(0.1)
    report = srk.SrkServerReport()
    assert L.srk_graph_free(None) == srk.SRK_OK
    assert L.srk_linear_ctx_free(None) == srk.SRK_OK
    assert L.srk_server_destroy(None) == srk.SRK_OK

    def refused(rc, msg):
        assert rc == srk.SRK_EINVAL and msg in L.srk_last_error()

    refused(L.srk_graph_info(None, ctypes.byref(n), ctypes.byref(m)), b"null graph")
    refused(L.srk_graph_layout(None, ctypes.byref(lay)), b"null argument")
    refused(L.srk_single_source_noalloc(None, 0, 0.6, 0.1, 1, None, None, None, None, None),
            b"null graph")
    refused(L.srk_multi_source(None, ctypes.cast(src, ctypes.c_void_p), 1, 0.6,
                               ctypes.cast(eps, ctypes.c_void_p), 1, None, None, None, None),
            b"null graph")
    refused(L.srk_linear_fwd(None, None, 0, 0.6, 3, None, None, None), b"null graph")
    refused(L.srk_linear_bwd(None, None, None, None), b"null context")
    refused(L.srk_server_create(None, 0, 0, 1, 0.0, None), b"out is null")
    refused(L.srk_server_submit(None, 0, 0, 0.6, 0.1, 1, None, 0, ctypes.byref(adm)),
            b"null server")
    refused(L.srk_server_drain(None), b"null server")
    refused(L.srk_server_stats(None, ctypes.byref(report)), b"null argument")
    refused(L.srk_probe_gather(None, 0, 1, 1, None, None, None), b"bad arguments")


def test_build_entry_point():
    import __graft_entry__ as g
    g.build()
