"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (CPU only: nothing here calls into the GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1604_06525_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b(opt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["opt_problem_create_grid", "opt_problem_create_graph", "opt_solve_gn",
                     "opt_solve_lm", "opt_pcg_init", "opt_pcg_step", "opt_apply_jtj",
                     "opt_eval_jtf", "opt_problem_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1604_06525_gb300 import api
    bound = {n for n, _, _ in api._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings_without_gpu(lib):
    lib.opt_status_str.restype = ctypes.c_char_p
    assert lib.opt_status_str(0) == b"OPT_OK"
    assert lib.opt_status_str(1) == b"OPT_ERR_INVALID_ARG"
    assert lib.opt_status_str(99) == b"OPT_ERR_UNKNOWN"


def test_null_arguments_are_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    out = ctypes.c_void_p(1)
    assert lib.opt_problem_create_grid(None, None, ctypes.byref(out)) == 1
    assert out.value is None
    assert lib.opt_problem_create_graph(None, None, ctypes.byref(out)) == 1
    assert lib.opt_solve_gn(None, None, None) == 1
    assert lib.opt_problem_destroy(None) == 0
    assert lib.opt_problem_create_grid_f64(None, None, ctypes.byref(out)) == 1
    assert lib.opt_problem_create_graph_f64(None, None, ctypes.byref(out)) == 1
    assert lib.opt_solve_lm_f64(None, None, None) == 1
    assert lib.opt_apply_jtj_f64(None, None, None, ctypes.c_double(0.0), None) == 1
    assert lib.opt_problem_destroy_f64(None) == 0
    assert lib.opt_server_set_max_active(None, 4) == 1


def test_library_is_built_for_sm103a():
    # the fat binary must carry sm_103a code; cuobjdump-free check: the build
    # command pins the one -gencode
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
