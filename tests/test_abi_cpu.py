"""The C-ABI library loads and exports every entry point of include/lrs.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lrs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lrs_create", "lrs_destroy", "lrs_load_orbitals", "lrs_set_sites",
                     "lrs_set_frequency_quadrature", "lrs_project", "lrs_build_chi0", "lrs_solve_w",
                     "lrs_get_chi0", "lrs_get_w", "lrs_backward", "lrs_stats", "lrs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2005_07834_gb300 import lrs
    lib = ctypes.CDLL(lrs.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(lrs.exported_symbols()) <= set(declared_functions())


def test_argument_errors_without_device():
    from paper_2005_07834_gb300 import lrs
    assert lrs.lrs_create(None, 0, 0, None) == lrs.LRS_ERR_ARG
    assert b"NULL" in lrs.lrs_last_error()
    ctx = ctypes.c_void_p()
    assert lrs.lrs_create(ctypes.byref(ctx), 0, 99, None) == lrs.LRS_ERR_ARG
    assert lrs.lrs_load_orbitals(None, None, 0, None, None, 0, None, 0, None, None, None) == lrs.LRS_ERR_ARG
    assert lrs.lrs_build_chi0(None, 0, None) == lrs.LRS_ERR_ARG
    assert lrs.lrs_destroy(None) == lrs.LRS_OK
    assert lrs.lrs_version().startswith(b"lrs")


def header_constants():
    src = open(os.path.join(ROOT, "include", "lrs.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(LRS_[A-Z0-9_]+)\s+(-?\d+)\b", src)}


def test_binding_constants_match_the_header():
    """Every integer constant of include/lrs.h that the binding names has the header's value
    (option codes, solver and update modes, lanes, precisions, error codes)."""
    from paper_2005_07834_gb300 import lrs
    consts = header_constants()
    assert {"LRS_OPT_DYSON_LANES", "LRS_OPT_DYSON_UPDATE", "LRS_UPDATE_TC", "LRS_SOLVER_SPD"} <= set(consts)
    checked = 0
    for name, value in consts.items():
        if hasattr(lrs, name):
            assert getattr(lrs, name) == value, name
            checked += 1
    assert checked >= 20
