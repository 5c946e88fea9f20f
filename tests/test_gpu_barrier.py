"""The grid-wide barrier of the persistent PCG loop and the mbarrier wait of
the tensor-copy staging never wait without bound: a wait that cannot complete
gives up, reports a timeout and leaves the context usable."""
import ctypes
import time

import pytest

from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1604_06525_gb300 import build, api as api_mod
    build.build()
    api_mod.load_library()
    return api_mod


def test_barrier_completes(api):
    lib = api.load_library()
    t = ctypes.c_int32(-1)
    assert lib.opt_selftest_grid_barrier(0, 200, ctypes.byref(t)) == 0
    assert t.value == 0


def test_barrier_wait_is_bounded_and_context_survives(api):
    lib = api.load_library()
    t = ctypes.c_int32(-1)
    t0 = time.perf_counter()
    assert lib.opt_selftest_grid_barrier(1, 3, ctypes.byref(t)) == 0
    assert t.value == 1
    assert time.perf_counter() - t0 < 10.0
    # invalid arguments are refused before any device work
    assert lib.opt_selftest_grid_barrier(-1, 3, ctypes.byref(t)) == 1
    assert lib.opt_selftest_grid_barrier(0, 0, ctypes.byref(t)) == 1
    assert lib.opt_selftest_grid_barrier(0, 3, None) == 1
    # the context still runs a persistent solve
    prob = synth.warp_problem(300, 40, 6, seed=171)
    g = api.Problem(prob)
    r = g.solve_gn(2, 6, persistent=1)
    assert r["status"] == "OPT_OK"


def test_staging_wait_is_bounded_and_context_survives(api):
    lib = api.load_library()
    t = ctypes.c_int32(-1)
    assert lib.opt_selftest_staging_wait(1, ctypes.byref(t)) == 0
    assert t.value == 0
    t0 = time.perf_counter()
    assert lib.opt_selftest_staging_wait(0, ctypes.byref(t)) == 0
    assert t.value == 1
    assert time.perf_counter() - t0 < 10.0
    assert lib.opt_selftest_staging_wait(2, ctypes.byref(t)) == 1
    assert lib.opt_selftest_staging_wait(1, None) == 1
    # the context still runs a solve staged by tensor copies (128-pixel tiles)
    prob = synth.poisson_problem(300, 40, seed=172)
    g = api.Problem(prob, tile_w=128)
    rep = g.solve_gn(2, 5)
    assert rep["E_history"][-1] < rep["E_history"][0]
    g.close()
