"""Degenerate and extreme inputs through the C ABI, against the float64 oracle:
the largest grid extents the planner accepts (and the first it rejects), zero
PCG iterations, graphs without edges or with a single vertex, images whose
pixels are all excluded or all fixed -- for the float32 path, the float64
solver and embedded deformation."""
import numpy as np
import pytest

import oracle
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


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def relE(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


@pytest.mark.parametrize("W,H", [(32767, 1), (1, 32767), (32767, 2)])
@pytest.mark.parametrize("f64", [False, True])
def test_largest_grid_extents(api, W, H, f64):
    """W or H = 32767, the largest extent the planner accepts (one row of
    tiles, or one column of ragged 128-wide tiles)."""
    import torch
    prob = synth.warp_problem(W, H, 20, seed=5)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = (api.ProblemF64 if f64 else api.Problem)(prob)
    dt = torch.float64 if f64 else torch.float32
    p = np.random.default_rng(3).standard_normal(prob.n_unknowns)
    q, _ = gp.apply_jtj(torch.as_tensor(p, dtype=dt, device="cuda"))
    J = e.jacobian(x)
    assert rel(q.cpu().numpy(), J.T @ (J @ p)) <= (1e-12 if f64 else 1e-5)
    ref = oracle.gauss_newton(e, x, 2, 5)
    rep = gp.solve_gn(2, 5)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= (1e-10 if f64 else 1e-4)
    gp.close()


@pytest.mark.parametrize("W,H", [(32768, 1), (1, 32768), (0, 5)])
def test_first_rejected_extent(api, W, H):
    import torch
    ok = synth.warp_problem(4, 4, 1, seed=1)
    d, x, keep = api.make_descriptor(ok, "cuda")
    d.W, d.H = W, H
    import ctypes
    h = ctypes.c_void_p()
    assert api.load_library().opt_problem_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert h.value is None
    torch.cuda.synchronize()


@pytest.mark.parametrize("f64", [False, True])
def test_zero_pcg_iterations(api, f64):
    """inner = 0: the step is 0, GN keeps x, LM rejects every step (zero
    predicted decrease) and grows lambda by nu = 2, 4, 8, ..."""
    prob = synth.warp_problem(20, 10, 3, seed=5)
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    gp = (api.ProblemF64 if f64 else api.Problem)(prob)
    rep = gp.solve_gn(2, 0)
    ref = oracle.gauss_newton(e, x0, 2, 0)
    assert rep["pcg_done"] == 0 == ref.pcg_done
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= 1e-6
    np.testing.assert_array_equal(gp.x.cpu().numpy().reshape(-1), x0.astype(gp.x.cpu().numpy().dtype))
    rep = gp.solve_lm(3, 0, lambda0=1e-3)
    ref = oracle.levenberg_marquardt(e, x0, 3, 0)
    assert rep["accepted"] == 0 == sum(ref.accepted)
    assert rep["lambda_final"] == pytest.approx(ref.lambda_final, rel=1e-12)
    gp.close()


@pytest.mark.parametrize("kind", ["mesh", "embedded", "mesh_f64"])
def test_graph_without_edges(api, kind):
    """No edges: only the fit rows (and, for embedded deformation, the column
    constraints) remain; LM moves the handles onto their targets."""
    import torch
    base = synth.mesh_problem(1, seed=3, handle_frac=0.2)
    if kind == "embedded":
        eb = synth.embedded_problem(1, seed=3, handle_frac=0.2, x0_noise=0.05)
        prob = synth.EmbeddedProblem(eb.V, eb.urshape, eb.v0[:0], eb.v1[:0], eb.x0, eb.handle_idx, eb.handle_target)
    else:
        prob = synth.MeshProblem(base.V, base.urshape, base.v0[:0], base.v1[:0], base.x0, base.handle_idx,
                                 base.handle_target)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    f64 = kind.endswith("f64")
    gp = (api.ProblemF64 if f64 else api.Problem)(prob)
    p = np.random.default_rng(2).standard_normal(prob.n_unknowns)
    dt = torch.float64 if f64 else torch.float32
    for lam in (0.0, 0.3):
        _, diag, _ = oracle.jtf_diag(e, x)
        q, _ = gp.apply_jtj(torch.as_tensor(p, dtype=dt, device="cuda"), lam)
        qref = oracle.apply_jtj(e, x, p, lam, np.clip(diag, 1e-6, 1e32))
        assert rel(q.cpu().numpy(), qref) <= (1e-12 if f64 else 1e-5)
    ref = oracle.levenberg_marquardt(e, x, 2, 10)
    rep = gp.solve_lm(2, 10)
    assert rep["accepted"] == int(sum(ref.accepted)) == 2
    assert relE(rep["E_history"][0], ref.E_history[0]) <= 1e-5
    # after one step E is ~1e-6 of E0 while the unknowns are not small: the
    # residuals cancel, and the float32 (float64) rounding of x and delta
    # allows the first-order bound of tests/lm_tolerance.py (~1e-3 here)
    from lm_tolerance import energy_rounding_bound, U32, U64
    x1 = oracle.levenberg_marquardt(e, x, 1, 10).x
    bound = energy_rounding_bound(e, x, x1, u=U64 if f64 else U32)
    assert relE(rep["E_history"][1], ref.E_history[1]) <= max(1e-4 if not f64 else 1e-12, bound)
    assert rep["E_final"] <= 1e-6 * ref.E_history[0]
    gp.close()


@pytest.mark.parametrize("kind", ["mesh", "embedded", "mesh_f64"])
def test_single_vertex_graph(api, kind):
    """One vertex, no edges, no handles.  ARAP: E = 0 and J^T F = 0, PCG stops
    at once (r.z = 0), x stays.  Embedded deformation: only the six column
    constraints of a non-orthonormal matrix; LM drives them to 0."""
    U = np.zeros((3, 1), np.float32)
    none = np.zeros(0, np.int32)
    if kind == "embedded":
        x0 = np.zeros((12, 1), np.float32)
        x0[3:12, 0] = (np.eye(3) + 0.1 * np.arange(9).reshape(3, 3) / 9).reshape(-1)
        prob = synth.EmbeddedProblem(1, U, none, none, x0, none, np.zeros((0, 3), np.float32))
    else:
        prob = synth.MeshProblem(1, U, none, none, np.full((6, 1), 0.3, np.float32), none,
                                 np.zeros((0, 3), np.float32))
    e = oracle.make_energy(prob)
    gp = (api.ProblemF64 if kind.endswith("f64") else api.Problem)(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 3, 10)
    rep = gp.solve_lm(3, 10)
    assert relE(rep["E_history"][0], ref.E_history[0]) <= 1e-5 or ref.E_history[0] == rep["E_history"][0] == 0.0
    if kind == "embedded":
        assert rep["accepted"] == int(sum(ref.accepted))
        assert rep["E_final"] <= 1e-6 * ref.E_history[0]
    else:
        assert rep["E_final"] == 0.0 and rep["pcg_done"] == 0
        np.testing.assert_array_equal(gp.x.cpu().numpy(), prob.x0.astype(gp.x.cpu().numpy().dtype))
    gp.close()


@pytest.mark.parametrize("f64", [False, True])
def test_all_pixels_excluded_or_fixed(api, f64):
    """Every warp pixel masked (no residual, handles dropped) or every
    Poisson pixel fixed (no unknown): E = 0, nothing moves."""
    w = synth.warp_problem(9, 8, 0, seed=5, mask=np.ones((8, 9), np.uint8))
    p = synth.poisson_problem(12, 10, seed=4)
    p.mask = np.ones((10, 12), np.uint8)
    for prob in (w, p):
        gp = (api.ProblemF64 if f64 else api.Problem)(prob)
        rep = gp.solve_gn(2, 5)
        assert rep["E_history"] == [0.0, 0.0, 0.0] and rep["pcg_done"] == 0
        np.testing.assert_array_equal(gp.x.cpu().numpy(), prob.x0.astype(gp.x.cpu().numpy().dtype))
        gp.close()
