"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/lbem.h declares.

No compute call is made here (no GPU needed).
"""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G

    G.build()
    from paper_1108_2651_gb300 import lbem

    return lbem.load()


def test_header_declares_the_boundary():
    from paper_1108_2651_gb300 import lbem

    names = lbem.header_symbols()
    for required in ("lbem_create", "lbem_set_medium", "lbem_step", "lbem_fields"):
        assert required in names
    assert len(names) >= 25


def test_every_declared_symbol_is_exported(lib):
    from paper_1108_2651_gb300 import lbem

    missing = [n for n in lbem.header_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1108_2651_gb300 import lbem

    for n in lbem.header_symbols():
        assert n in lbem._SIGS, n
        assert callable(getattr(lbem, n)), n


def test_last_error_is_callable_without_a_gpu(lib):
    assert isinstance(lib.lbem_last_error(), bytes)


def test_descriptor_layout_matches_header():
    from paper_1108_2651_gb300 import lbem

    # int dim, nx, ny, nz, storage; double c_ref2; void* stream  (LP64)
    assert lbem.Desc.c_ref2.offset == 24 and lbem.Desc.stream.offset == 32
    assert ctypes.sizeof(lbem.Desc) == 40


def test_product_path_refuses_to_run_without_the_library(tmp_path):
    from paper_1108_2651_gb300 import lbem

    saved = lbem._lib
    lbem._lib = None
    try:
        with pytest.raises(OSError):
            lbem.load(str(tmp_path / "missing.so"))
    finally:
        lbem._lib = saved
