"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute calls here (no GPU in this environment); only entry points that
validate arguments on the host are exercised.
"""
import ctypes as C
import glob
import os
import re

import pytest

from paper_1209_4008_gb300 import build, gf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gf.load()


def test_header_declares_the_method_entry_points():
    names = declared_functions()
    for required in ("gf_create", "gf_overrelax", "gf_anneal", "gf_functional", "gf_theta",
                     "gf_destroy", "gf_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = declared_functions()
    missing = [n for n in names if n not in gf.SIGNATURES]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    h = C.c_void_p()
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 5), 0, C.byref(h)) == gf.GF_EINVAL
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 0), 0, C.byref(h)) == gf.GF_EINVAL
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), 7, C.byref(h)) == gf.GF_EINVAL
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), 0, C.byref(h)) == gf.GF_OK
    try:
        assert lib.gf_set_option(h, b"precision", 1.0) == gf.GF_OK
        assert lib.gf_set_option(h, b"precision", 5.0) == gf.GF_EINVAL
        assert lib.gf_set_option(h, b"storage64", 12.0) == gf.GF_OK
        assert lib.gf_set_option(h, b"threads_per_site", 3.0) == gf.GF_EINVAL
        assert lib.gf_set_option(h, b"no_such_option", 1.0) == gf.GF_EINVAL
        assert b"no_such_option" in lib.gf_last_error(h)
        v = C.c_double()
        assert lib.gf_get_option(h, b"storage64", C.byref(v)) == gf.GF_OK and v.value == 12
        # resident-field calls without a field report a state error, not a crash
        assert lib.gf_or_half_sweep(h, 0, 1.7) == gf.GF_ESTATE
        assert lib.gf_or_half_sweep(h, 0, 2.5) in (gf.GF_EINVAL, gf.GF_ESTATE)
    finally:
        assert lib.gf_destroy(h) == gf.GF_OK
    assert lib.gf_destroy(None) == gf.GF_OK
    assert lib.gf_error_string(gf.GF_ENOTCONVERGED) == b"GF_ENOTCONVERGED"


def test_host_side_checks_of_the_added_paths(lib):
    """Options and entry points of the OR readings, register budgets, per-
    timeslice stopping, the maximally Abelian gauge and generation: argument
    and state errors are reported without touching a GPU."""
    h = C.c_void_p()
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), gf.GF_MAG, C.byref(h)) == gf.GF_OK
    try:
        for key, bad, good in ((b"or_variant", 3.0, 2.0), (b"acc_registers", 200.0, 168.0)):
            assert lib.gf_set_option(h, key, bad) == gf.GF_EINVAL
            assert lib.gf_set_option(h, key, good) == gf.GF_OK
        # not in the maximally Abelian gauge
        assert lib.gf_set_option(h, b"theta_per_timeslice", 1.0) == gf.GF_EINVAL
        assert lib.gf_set_option(h, b"fp64_arith", 1.0) == gf.GF_EINVAL
        assert lib.gf_set_option(h, b"stochastic_p", 0.5) == gf.GF_EINVAL
        assert b"maximally Abelian" in lib.gf_last_error(h)
        F = (C.c_double * 4)()
        assert lib.gf_measure_timeslices(h, F, F) == gf.GF_EINVAL  # not in this gauge
        assert lib.gf_wilson_update(h, 0, 0, 6.0, 0, 1, 0) == gf.GF_ESTATE
    finally:
        lib.gf_destroy(h)
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), gf.GF_COULOMB, C.byref(h)) == gf.GF_OK
    try:
        assert lib.gf_set_option(h, b"theta_per_timeslice", 1.0) == gf.GF_OK
        F = (C.c_double * 4)()
        assert lib.gf_measure_timeslices(h, F, F) == gf.GF_ESTATE  # no resident field
        assert lib.gf_generate(h, None, 6.0, 1, 1, 1, 0) == gf.GF_EINVAL  # no field
        assert lib.gf_generate(h, None, -1.0, 1, 1, 1, 0) == gf.GF_EINVAL
    finally:
        lib.gf_destroy(h)


def test_fp32_restarts_option_host_side(lib):
    """The restart option's range, and the policy it needs (tracked gauge and
    reunitarisation at every check), are checked before any device work."""
    import numpy as np
    h = C.c_void_p()
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), gf.GF_LANDAU, C.byref(h)) == gf.GF_OK
    try:
        for bad in (-1.0, 17.0, 1.5):
            assert lib.gf_set_option(h, b"fp32_restarts", bad) == gf.GF_EINVAL
        assert lib.gf_set_option(h, b"fp32_restarts", 2.0) == gf.GF_OK
        v = C.c_double()
        assert lib.gf_get_option(h, b"fp32_restarts", C.byref(v)) == gf.GF_OK and v.value == 2
        assert lib.gf_set_option(h, b"precision", float(gf.GF_MIXED)) == gf.GF_OK
        U = np.zeros(4 ** 4 * 72)
        it, F, th = C.c_int(), C.c_double(), C.c_double()
        for key, val in ((b"track_gauge", 0.0), (b"reunitarize_every", 2.0)):
            assert lib.gf_set_option(h, key, val) == gf.GF_OK
            rc = lib.gf_overrelax(h, U.ctypes.data, 1.7, 1e-12, 10, C.byref(it), C.byref(F), C.byref(th))
            assert rc == gf.GF_EINVAL and b"fp32_restarts" in lib.gf_last_error(h)
            assert lib.gf_set_option(h, key, 1.0) == gf.GF_OK
    finally:
        lib.gf_destroy(h)


def documented_options():
    """Option keys listed in the gf_set_option documentation of include/gf.h."""
    text = open(os.path.join(ROOT, "include", "gf.h")).read()
    block = text[text.index("int gf_create"):text.index("int gf_set_option")]
    return re.findall(r'^\s*\*\s+"(\w+)"', block, flags=re.M)


def test_every_documented_option_round_trips(lib):
    """Each documented option is known to gf_get_option, and setting it to the
    value read back is accepted (the documentation and the parser agree)."""
    keys = documented_options()
    assert len(keys) >= 20
    h = C.c_void_p()
    assert lib.gf_create((C.c_int * 4)(4, 4, 4, 4), gf.GF_LANDAU, C.byref(h)) == gf.GF_OK
    try:
        for key in keys:
            v = C.c_double()
            assert lib.gf_get_option(h, key.encode(), C.byref(v)) == gf.GF_OK, key
            assert lib.gf_set_option(h, key.encode(), v.value) == gf.GF_OK, (key, v.value)
    finally:
        lib.gf_destroy(h)


def test_batch_handle_host_side(lib):
    b = gf.gf_batch_create([(4, 4, 4, 4), (8, 8, 8, 8)], gf.GF_LANDAU)
    gf.gf_batch_set_option(b, "precision", gf.GF_FP64)
    gf.gf_batch_set_option(b, "check_every", 10)
    with pytest.raises(gf.GFError):
        gf.gf_batch_set_option(b, "threads_per_site", 3)
    with pytest.raises(gf.GFError):
        gf.gf_batch_set_option(b, "no_such_option", 1)
    gf.gf_batch_destroy(b)
    with pytest.raises(gf.GFError):
        gf.gf_batch_create([(4, 4, 4, 5)])
    h = C.c_void_p()
    assert lib.gf_batch_create(0, (C.c_int * 4)(4, 4, 4, 4), 0, C.byref(h)) == gf.GF_EINVAL


def test_binding_argument_counts_match_header():
    text = ""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text += re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(gf_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    for name, (_, argtypes) in gf.SIGNATURES.items():
        assert name in protos, name
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])


def test_noalloc_binding_refuses_mistyped_tensors(lib):
    """The allocation-free measurement reads U and writes two doubles at raw
    addresses; the binding refuses tensors of the wrong type or size before
    the library sees them, and the library refuses what it cannot hold."""
    import torch
    U = torch.zeros(4 ** 4 * 72, dtype=torch.float64)
    out = torch.zeros(2, dtype=torch.float64)
    for bad_u, bad_out in ((U, torch.zeros(2, dtype=torch.float32)), (U, torch.zeros(1, dtype=torch.float64)),
                           (U[:-2], out), (U.float(), out)):
        with pytest.raises(ValueError):
            gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, bad_u, bad_out)
    dims = (C.c_int * 4)
    assert lib.gf_measure_noalloc(dims(4, 4, 4, 4), gf.GF_LANDAU, None, None, None) == gf.GF_EINVAL
    # host memory is never accepted (no staging copy without an allocation)
    assert lib.gf_measure_noalloc(dims(4, 4, 4, 4), gf.GF_LANDAU, U.data_ptr(), out.data_ptr(), None) \
        in (gf.GF_EINVAL, gf.GF_ECUDA)  # ECUDA where no driver is present
    assert lib.gf_measure_noalloc(dims(4, 4, 4, 4), 7, U.data_ptr(), out.data_ptr(), None) == gf.GF_EINVAL
    assert lib.gf_measure_noalloc(dims(64, 64, 64, 64), 0, U.data_ptr(), out.data_ptr(), None) == gf.GF_EINVAL
