"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/hpg.h; the Python binding declares the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpg.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpg_[a-z_0-9]+)\s*\(", src)) - {"hpg_field_fn"})


@pytest.fixture(scope="module")
def libpath():
    from paper_2412_13733_gb300 import build, hpg
    if not os.path.exists(hpg.LIB_PATH):
        build.build()
    return hpg.LIB_PATH


def test_header_declares_the_boundary():
    names = declared()
    for must in ["hpg_create", "hpg_destroy", "hpg_problem_create", "hpg_set_rhs", "hpg_set_constraint",
                 "hpg_set_dirichlet", "hpg_set_alpha_schedule", "hpg_set_params", "hpg_solve", "hpg_solve_batch",
                 "hpg_get_u", "hpg_get_psi", "hpg_get_stats", "hpg_eval_u", "hpg_status_str"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2412_13733_gb300 import hpg
    assert set(declared()) <= set(hpg.SIGNATURES)
    hpg.lib()      # loads and binds every signature


def test_host_only_calls_without_gpu(libpath):
    from paper_2412_13733_gb300 import hpg
    L = hpg.lib()
    assert L.hpg_status_str(0) == b"HPG_OK"
    assert L.hpg_status_str(7) == b"HPG_ERR_NOT_SPD"
    p = hpg.default_params()
    assert p.newton_tol == 1e-10 and p.krylov_max == 150
    # a NULL output pointer is rejected, never dereferenced
    assert L.hpg_create(None, 0, None) == 1
