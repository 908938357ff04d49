"""The C-ABI library loads and exports every function include/dgsl.h declares
(no compute calls)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgsl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgsl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dgsl_build_operators", "dgsl_apply_schur", "dgsl_cg_solve",
                     "dgsl_query_maps", "dgsl_destroy_operator", "dgsl_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(dgsl_lib):
    for name in declared_functions():
        assert hasattr(dgsl_lib, name), name


def test_version_string(dgsl_lib):
    assert b"sm_103a" in dgsl_lib.dgsl_version()
