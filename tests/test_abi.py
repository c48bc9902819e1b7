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


@pytest.mark.parametrize("kw,msg", [
    (dict(dim=4, nx=8, ny=8), "dim"),
    (dict(dim=2, nx=0, ny=8), "sizes"),
    (dict(dim=2, nx=8, ny=-1), "sizes"),
    (dict(dim=3, nx=8, ny=8, nz=0), "sizes"),
    (dict(dim=2, nx=8, ny=8, storage=9), "storage"),
    (dict(dim=3, nx=8, ny=8, nz=8, storage=1), "3D"),
    (dict(dim=2, nx=1 << 29, ny=1), "too large"),
])
def test_create_rejects_invalid_descriptors_before_touching_the_device(lib, kw, msg):
    """Descriptor validation happens on the host, before any CUDA call, so it is testable without a GPU."""
    from paper_1108_2651_gb300 import lbem

    args = dict(dim=2, nx=8, ny=8, nz=1, storage=0)
    args.update(kw)
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_create(args["dim"], args["nx"], args["ny"], args.get("nz", 1), args["storage"])
    assert e.value.status == 1 and msg in str(e.value)


def test_null_handles_are_rejected(lib):
    from paper_1108_2651_gb300 import lbem

    d = ctypes.c_double
    for f, extra in (("lbem_step", [1]), ("lbem_sync", []), ("lbem_set_graphs", [1]), ("lbem_set_variant", [0]),
                     ("lbem_check_guards", []), ("lbem_batch_step", [1]), ("lbem_set_stream", [None]),
                     ("lbem_info", [None, None]), ("lbem_set_medium", [None, None]),
                     ("lbem_set_medium_aniso", [None, d(1.0), d(1.0)]), ("lbem_set_fields", [None, None]),
                     ("lbem_set_sources", [0, None, None, None, 0]), ("lbem_set_receivers", [0, None, None, 0]),
                     ("lbem_set_boundaries", [None, 0, d(0.0)]), ("lbem_get_boundaries", [None, None, None]),
                     ("lbem_set_dispersion", [None, None, None]), ("lbem_set_watchdog", [0, d(2.0)]),
                     ("lbem_set_temporal_blocking", [2, 0]), ("lbem_get_temporal_blocking", [None, None, None]),
                     ("lbem_time", [None]), ("lbem_fields", [None, None]), ("lbem_energy_flux", [None, None]),
                     ("lbem_traces", [None, None]), ("lbem_diagnostics", [None]), ("lbem_save_state", [None]),
                     ("lbem_load_state", [None, 0]), ("lbem_rows", [0, 0, 1, None, 0]),
                     ("lbem_forward_record", [2, 1]), ("lbem_adjoint", [None, None, None]),
                     ("lbem_autotune", [1, None]), ("lbem_get_variant", [None, None]),
                     ("lbem_batch_autotune", [1, None]), ("lbem_batch_set_variant", [0]),
                     ("lbem_batch_get_variant", [None, None]), ("lbem_halo_out", [1, None, None]),
                     ("lbem_halo_in", [1, None, None])):
        assert getattr(lib, f)(None, *extra) == 1, f
        assert "null" in lbem.lbem_last_error() or "bad argument" in lbem.lbem_last_error(), f


def test_wait_limit_rejects_bad_values_before_touching_the_device(lib):
    from paper_1108_2651_gb300 import lbem

    for v in (-1.0, float("nan"), float("inf"), 1e9):
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_wait_limit(v)
        assert e.value.status == 1 and "seconds" in str(e.value)
