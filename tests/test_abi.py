"""The C-ABI library loads on a CPU-only host and exports every entry point
that include/gpa.h declares (no compute calls: there is no GPU here)."""
import ctypes

import numpy as np

import synth


def test_library_exports_every_declared_symbol():
    import paper_2009_04061_gb300 as g
    lib = g.library()
    names = g.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    for core in ("gpa_create", "gpa_load_program", "gpa_ingest_samples", "gpa_blame", "gpa_advise"):
        assert core in names


def test_status_strings_and_default_arch():
    import paper_2009_04061_gb300 as g
    lib = g.library()
    assert lib.gpa_status_string(0) == b"ok"
    assert lib.gpa_status_string(-4).startswith(b"reaching")
    lat, fl = g.gpa_arch_default()
    # the workload generator's opcode table is the library's default table
    slat, sfl = synth.default_arch()
    assert np.array_equal(lat, slat) and np.array_equal(fl, sfl)


def test_invalid_arguments_are_rejected_without_a_device():
    import paper_2009_04061_gb300 as g
    lib = g.library()
    assert lib.gpa_create(None, None, None) == -1
    assert lib.gpa_destroy(None) == -1
    assert lib.gpa_arch_default(None) == -1
    assert lib.gpa_launch_count(None) == -1


def test_advice_buffers_are_checked_before_use():
    """Reusable advice arrays must match the program's shapes and dtypes; a mismatch is
    refused before the library sees a pointer."""
    import numpy as np
    import pytest
    from paper_2009_04061_gb300 import gpa
    shape = (3, 2, 5)
    b = gpa.advice_buffers(shape)
    assert gpa._advice_out(shape, b) is b
    assert b["hot"].shape == (3, gpa.NUM_OPT, 5, 6) and b["line_stall"].shape == (5,)
    bad = dict(b, speedup=np.zeros((3, gpa.NUM_OPT), np.float32))
    with pytest.raises(ValueError):
        gpa._advice_out(shape, bad)
    with pytest.raises(ValueError):
        gpa._advice_out((4, 2, 5), b)
