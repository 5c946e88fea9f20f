"""Parity of the full float64 solver (opt_*_f64 through the C ABI) against the
float64 oracle.

Both sides compute in float64 and differ only in the order of their sums, so
the bars are rounding-level: J^T J p, J^T F and diag(J^T J) <= 1e-12 relative
(norm-wise), energies <= 1e-12, whole GN / LM trajectories <= 1e-9 per outer
iteration, identical iteration and acceptance counts.  Sizes span ragged
grids, masks, the degenerate 1 x N grids and small meshes with one-way edges.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_PRODUCT = 1e-12
TOL_ENERGY = 1e-12
TOL_TRAJ = 1e-9


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


def perturbed(prob, scale, seed):
    rng = np.random.default_rng(seed)
    x = prob.x0.astype(np.float64).copy()
    if prob.kind == "poisson":
        free = np.ones((prob.H, prob.W), bool) if prob.mask is None else prob.mask == 0
        x[:, free] += rng.uniform(-scale, scale, size=(4, int(free.sum())))
    else:
        x += rng.uniform(-scale, scale, size=x.shape)
    prob.x0 = x
    return prob


def direction(prob, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(prob.n_unknowns)
    if prob.kind == "poisson" and prob.mask is not None:
        p.reshape(4, -1)[:, prob.mask.reshape(-1) != 0] = 0.0
    return p


GRID_CASES = [("warp", 64, 64, 0.0), ("warp", 37, 29, 0.25), ("warp", 1, 1, 0.0), ("warp", 1, 45, 0.0),
              ("warp", 70, 1, 0.0), ("warp", 300, 41, 0.2),
              ("poisson", 64, 48, None), ("poisson", 45, 33, None), ("poisson", 1, 17, None),
              ("poisson", 301, 17, None), ("poisson", 40, 30, "nomask")]


def make_grid(kind, W, H, mf, seed=11):
    if kind == "warp":
        mask = synth.random_mask(W, H, mf, seed + 1) if mf else None
        prob = synth.warp_problem(W, H, max(1, (W * H) // 200), seed=seed, mask=mask)
        return perturbed(prob, 0.5, seed + 2)
    prob = synth.poisson_problem(W, H, seed=seed)
    if mf == "nomask":
        prob.mask = None
    return perturbed(prob, 0.2, seed + 2)


def make_mesh(level, noise, seed=31):
    return perturbed(synth.mesh_problem(level, seed=seed, handle_frac=0.05), noise, seed + 1)


def check_products(api, prob, seed):
    import torch
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.ProblemF64(prob)
    jtf, diag, E = gp.eval_jtf()
    rj, rd, rE = oracle.jtf_diag(e, x)
    assert rel(jtf.cpu().numpy(), rj) <= TOL_PRODUCT
    assert rel(diag.cpu().numpy(), rd) <= TOL_PRODUCT
    assert relE(E, rE) <= TOL_ENERGY
    assert relE(gp.energy(), rE) <= TOL_ENERGY
    p = direction(prob, seed)
    for lam in (0.0, 0.37):
        q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        qref = oracle.apply_jtj(e, x, p, lam, np.clip(rd, 1e-6, 1e32))
        assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT, lam
        assert relE(pq, float(p @ qref)) <= TOL_PRODUCT
    gp.close()


@pytest.mark.parametrize("kind,W,H,mf", GRID_CASES)
def test_grid_products_f64(api, kind, W, H, mf):
    check_products(api, make_grid(kind, W, H, mf), 5)


@pytest.mark.parametrize("level,noise", [(0, 0.3), (1, 0.2), (3, 0.1)])
def test_mesh_products_f64(api, level, noise):
    check_products(api, make_mesh(level, noise), 7)


def test_mesh_one_way_edges_f64(api):
    prob = make_mesh(2, 0.25, seed=61)
    rng = np.random.default_rng(5)
    sel = rng.random(prob.v0.size) < 0.6
    v0, v1 = prob.v0[sel], prob.v1[sel]
    dup = rng.choice(v0.size, size=7, replace=False)
    v0 = np.concatenate([v0, v0[dup]]).astype(np.int32)
    v1 = np.concatenate([v1, v1[dup]]).astype(np.int32)
    perm = rng.permutation(v0.size)                      # any order: the library sorts a copy
    prob = synth.MeshProblem(prob.V, prob.urshape, v0[perm], v1[perm], prob.x0, prob.handle_idx,
                             prob.handle_target)
    check_products(api, prob, 4)


def trajectory_close(rep, ref_hist, tol):
    for k, (a, b) in enumerate(zip(rep["E_history"], ref_hist)):
        assert relE(a, b) <= tol, (k, a, b)


def test_gn_warp_64_f64(api):
    prob = synth.warp_problem(64, 64, 8, seed=synth.BASE_SEED)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 10, 10)
    gp = api.ProblemF64(prob)
    rep = gp.solve_gn(10, 10)
    assert rep["outer_done"] == 10 and rep["pcg_done"] == ref.pcg_done
    trajectory_close(rep, ref.E_history, TOL_TRAJ)
    assert rel(gp.x.cpu().numpy(), ref.x) <= 1e-9


def test_gn_poisson_f64(api):
    prob = synth.poisson_problem(96, 80, seed=71)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 4, 20)
    gp = api.ProblemF64(prob)
    rep = gp.solve_gn(4, 20)
    trajectory_close(rep, ref.E_history, TOL_TRAJ)
    fixed = prob.mask != 0
    np.testing.assert_array_equal(gp.x.cpu().numpy()[:, fixed], prob.x0[:, fixed])
    assert rel(gp.x.cpu().numpy(), ref.x) <= 1e-9


def test_lm_mesh_f64(api):
    prob = synth.mesh_problem(3, seed=91, handle_frac=0.02)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 6, 15)
    gp = api.ProblemF64(prob)
    rep = gp.solve_lm(6, 15, lambda0=1e-3)
    assert rep["outer_done"] == ref.outer_done
    assert rep["accepted"] == int(sum(ref.accepted))
    trajectory_close(rep, ref.E_history, TOL_TRAJ)
    assert relE(rep["lambda_final"], ref.lambda_final) <= 1e-8
    assert rel(gp.x.cpu().numpy(), ref.x) <= 1e-8


def test_lm_warp_masked_rel_tol_f64(api):
    mask = synth.random_mask(48, 40, 0.1, 3)
    prob = synth.warp_problem(48, 40, 6, seed=93, mask=mask)
    e = oracle.make_energy(prob)
    prm = oracle.LMParams(rel_tol=1e-2)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 10, 10, prm)
    gp = api.ProblemF64(prob)
    rep = gp.solve_lm(10, 10, rel_tol=1e-2)
    assert rep["outer_done"] == ref.outer_done
    assert rep["converged"] == int(ref.outer_done < 10)
    trajectory_close(rep, ref.E_history, TOL_TRAJ)


def test_lm_rejections_f64(api):
    prob = synth.poisson_problem(30, 20, seed=92)
    gp = api.ProblemF64(prob)
    rep = gp.solve_lm(4, 10, lambda0=1e-3, eta=2.0)
    assert rep["accepted"] == 0 and rep["outer_done"] == 4
    assert rep["lambda_final"] == pytest.approx(1e-3 * 2 * 4 * 8 * 16, rel=1e-14)
    np.testing.assert_array_equal(gp.x.cpu().numpy(), prob.x0)


def test_gn_rounding_sensitive_warp_f64(api):
    """Undamped GN on a small warp with large handle pulls is not contractive:
    float32 rounding differences grow about tenfold per outer iteration and
    reach 1e-3 relative after 10 iterations.  In float64 the same trajectory
    stays on the oracle's to the bar of the energy checks."""
    prob = synth.warp_problem(34, 34, 8, seed=4)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 10, 10)
    gp = api.ProblemF64(prob)
    rep = gp.solve_gn(10, 10)
    trajectory_close(rep, ref.E_history, 1e-4)


def test_graph_replay_equals_direct_f64(api):
    import torch
    prob = synth.warp_problem(50, 40, 6, seed=81)
    a = api.ProblemF64(prob)
    b = api.ProblemF64(prob)
    ra = a.solve_gn(3, 8, use_graph=1)
    rb = b.solve_gn(3, 8, use_graph=0)
    assert ra["E_history"] == rb["E_history"]
    assert torch.equal(a.x, b.x)


def test_full_size_warp_f64(api):
    """ARAP warp 1024 x 1024 with 64 handles (the grid-at-scale configuration):
    J^T J p and J^T F over the whole grid, and the first GN iterations."""
    import torch
    prob = perturbed(synth.warp_problem(1024, 1024, 64, seed=synth.BASE_SEED), 0.3, 5)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.ProblemF64(prob)
    p = direction(prob, 9)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian(x)
    assert rel(q.cpu().numpy(), J.T @ (J @ p)) <= TOL_PRODUCT
    jtf, _, E = gp.eval_jtf()
    assert rel(jtf.cpu().numpy(), J.T @ e.residuals(x)) <= TOL_PRODUCT
    ref = oracle.gauss_newton(e, x, 2, 20)
    rep = gp.solve_gn(2, 20)
    trajectory_close(rep, ref.E_history, TOL_TRAJ)


def test_full_size_mesh_f64(api):
    """Icosphere level 7 (163,842 vertices, 983,040 directed edges)."""
    import torch
    prob = perturbed(synth.mesh_problem(7, seed=synth.BASE_SEED), 0.05, 6)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.ProblemF64(prob)
    p = direction(prob, 8)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian(x)
    assert rel(q.cpu().numpy(), J.T @ (J @ p)) <= TOL_PRODUCT
    jtf, _, E = gp.eval_jtf()
    assert rel(jtf.cpu().numpy(), J.T @ e.residuals(x)) <= TOL_PRODUCT


def test_invalid_arguments_f64(api):
    bad = synth.warp_problem(8, 8, 2, seed=1)
    bad.handle_idx = np.array([3, 3], np.int32)
    with pytest.raises(api.OptError) as ei:
        api.ProblemF64(bad)
    assert ei.value.status == 1
    m = synth.mesh_problem(0, seed=1)
    m.v1 = m.v1.copy()
    m.v1[0] = m.v0[0]                                      # a loop
    with pytest.raises(api.OptError):
        api.ProblemF64(m)
    gp = api.ProblemF64(synth.warp_problem(8, 8, 2, seed=1))
    with pytest.raises(api.OptError):
        gp.solve_gn(2, 2, materialized=1)                 # matrix-free only
    gp.close()


def test_fp64_fma_rate_is_measured(api):
    g = api.fp64_fma_rate()
    assert 10.0 < g < 1e6   # GFLOP/s


@pytest.mark.parametrize("kind", ["warp", "poisson", "mesh"])
def test_plain_cg_f64(api, kind):
    """use_precond = 0: unpreconditioned CG (M^-1 = 1), against the oracle's.
    Without the Jacobi scaling the warp's system is badly conditioned (the
    fit rows weigh 100 against rows of 4 .. 8), and CG carries the different
    summation orders of the two sides further: the bar is 1e-6, not 1e-9."""
    prob = {"warp": lambda: synth.warp_problem(40, 30, 5, seed=17),
            "poisson": lambda: synth.poisson_problem(48, 40, seed=18),
            "mesh": lambda: synth.mesh_problem(2, seed=19, handle_frac=0.05)}[kind]()
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 3, 10, use_precond=False)
    gp = api.ProblemF64(prob)
    rep = gp.solve_gn(3, 10, use_precond=0)
    assert rep["pcg_done"] == ref.pcg_done
    trajectory_close(rep, ref.E_history, 1e-6)
