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
