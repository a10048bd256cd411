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


def struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/hpg.h, in order."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    bodies = dict((n, body) for body, n in re.findall(r"typedef struct\s*\{([^{}]*)\}\s*(\w+)\s*;", src))
    assert name in bodies, name
    fields = []
    for decl in bodies[name].split(";"):
        decl = decl.strip()
        if not decl:
            continue
        head, *rest = [t.strip() for t in decl.split(",")]
        fields.append(re.sub(r"\[.*\]", "", head.split()[-1]).lstrip("*"))
        fields.extend(re.sub(r"\[.*\]", "", r).lstrip("*") for r in rest)
    return fields


@pytest.mark.parametrize("cname,pyname", [("hpg_params", "hpg_params"), ("hpg_stats", "hpg_stats")])
def test_binding_structs_mirror_header(cname, pyname):
    """The ctypes structures lay out the same fields, in the same order, as the C header."""
    from paper_2412_13733_gb300 import hpg
    py = [f[0] for f in getattr(hpg, pyname)._fields_]
    assert py == struct_fields(cname)


def test_default_params_keep_fp64_orthogonalisation(libpath):
    from paper_2412_13733_gb300 import hpg
    p = hpg.default_params()
    assert p.krylov_f32 == 0 and p.strategy == hpg.HPG_SCHUR and p.precision == hpg.HPG_FP64
