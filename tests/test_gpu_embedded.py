"""Embedded deformation (Fig. 28) through the C ABI against the float64 oracle.

Tolerances as for the other energies: J^T J p and J^T F <= 1e-5 relative
(norm-wise, float32 arithmetic), energies <= 1e-4 relative, identical LM
iteration and acceptance counts.  Meshes from the icosahedron (12 vertices)
up to the 10,242-vertex icosphere (the size class of the paper's 12k-vertex
example), one-way / duplicated / unsorted edge lists, batches.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_PRODUCT = 1e-5
TOL_ENERGY = 1e-4


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


def make(level, noise, seed=31, w_rot=1.0, handle_frac=0.05):
    return synth.embedded_problem(level, seed=seed, handle_frac=handle_frac, x0_noise=noise, w_rot=w_rot)


def check_products(api, prob, seed):
    import torch
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    jtf, diag, E = gp.eval_jtf()
    rj, rd, rE = oracle.jtf_diag(e, x)
    assert rel(jtf.cpu().numpy(), rj) <= TOL_PRODUCT
    assert rel(diag.cpu().numpy(), rd) <= TOL_PRODUCT
    assert relE(E, rE) <= TOL_PRODUCT
    assert relE(gp.energy(), rE) <= TOL_PRODUCT
    p = np.random.default_rng(seed).standard_normal(prob.n_unknowns).astype(np.float32)
    for lam in (0.0, 0.37):
        q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(rd, 1e-6, 1e32))
        assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT, lam
        assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    gp.close()


@pytest.mark.parametrize("level,noise,w_rot", [(0, 0.3, 1.0), (1, 0.2, 4.0), (3, 0.1, 1.0), (3, 0.0, 0.5)])
def test_embedded_products(api, level, noise, w_rot):
    check_products(api, make(level, noise, w_rot=w_rot), 7)


def test_embedded_one_way_duplicated_unsorted_edges(api):
    prob = make(2, 0.25, seed=61)
    rng = np.random.default_rng(5)
    sel = rng.random(prob.v0.size) < 0.6
    v0, v1 = prob.v0[sel], prob.v1[sel]
    dup = rng.choice(v0.size, size=7, replace=False)
    v0 = np.concatenate([v0, v0[dup]]).astype(np.int32)
    v1 = np.concatenate([v1, v1[dup]]).astype(np.int32)
    perm = rng.permutation(v0.size)
    prob = synth.EmbeddedProblem(prob.V, prob.urshape, v0[perm], v1[perm], prob.x0, prob.handle_idx,
                                 prob.handle_target)
    check_products(api, prob, 4)


def test_embedded_pcg_iterates(api):
    prob = make(2, 0.2, seed=63)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    J = e.jacobian(x)
    b = -(J.T @ e.residuals(x))
    Minv = oracle.solver.jacobi_minv(np.asarray(J.multiply(J).sum(0)).ravel())
    for k in (1, 3, 6):
        gp.pcg_init(0.0)
        gp.pcg_step(k)
        dl, r, p, it = gp.pcg_state()
        d_ref, n_done, r_ref = oracle.jacobi_pcg(lambda v: J.T @ (J @ v), b, Minv, k)
        assert it == n_done == k
        assert rel(dl.cpu().numpy(), d_ref) <= 1e-4
        assert rel(r.cpu().numpy(), r_ref) <= 1e-4


def test_embedded_lm_matches_oracle(api):
    prob = synth.embedded_problem(3, seed=91, handle_frac=0.02)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 6, 15)
    gp = api.Problem(prob)
    rep = gp.solve_lm(6, 15, lambda0=1e-3)
    assert rep["outer_done"] == ref.outer_done
    assert rep["accepted"] == int(sum(ref.accepted))
    for k, (a, b) in enumerate(zip(rep["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    x = gp.x.cpu().numpy().reshape(-1)
    assert relE(e.energy(x), ref.E_history[-1]) <= TOL_ENERGY


def test_embedded_lm_rel_tol_stops_like_oracle(api):
    prob = synth.embedded_problem(2, seed=93, handle_frac=0.05)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 10, 10, oracle.LMParams(rel_tol=1e-2))
    gp = api.Problem(prob)
    rep = gp.solve_lm(10, 10, rel_tol=1e-2)
    assert rep["outer_done"] == ref.outer_done
    assert rep["converged"] == int(ref.outer_done < 10)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


def test_embedded_full_size_level5(api):
    """Icosphere level 5 (10,242 vertices, 61,440 directed edges, 122,904
    unknowns): products over the whole mesh and the first LM iterations."""
    import torch
    prob = make(5, 0.05, seed=synth.BASE_SEED, handle_frac=0.01)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = np.random.default_rng(8).standard_normal(prob.n_unknowns).astype(np.float32)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian(x)
    assert rel(q.cpu().numpy(), J.T @ (J @ p.astype(np.float64))) <= TOL_PRODUCT
    jtf, _, _ = gp.eval_jtf()
    assert rel(jtf.cpu().numpy(), J.T @ e.residuals(x)) <= TOL_PRODUCT
    ref = oracle.levenberg_marquardt(e, x, 3, 20)
    rep = gp.solve_lm(3, 20, lambda0=1e-3)
    assert rep["accepted"] == int(sum(ref.accepted))
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


def test_embedded_in_a_batch_equals_solo(api):
    probs = [synth.embedded_problem(2, seed=300, handle_frac=0.05), synth.embedded_problem(3, seed=301),
             synth.mesh_problem(2, seed=302, handle_frac=0.05)]
    solo = []
    for p in probs:
        g = api.Problem(p)
        solo.append(g.solve_lm(4, 8))
        g.close()
    members = [api.Problem(p) for p in probs]
    batch = api.Batch(members)
    reps, _ = batch.solve_lm(4, 8)
    for r, s in zip(reps, solo):
        assert r["outer_done"] == s["outer_done"] and r["accepted"] == s["accepted"]
        for a, b in zip(r["E_history"], s["E_history"]):
            assert relE(a, b) <= 1e-5
    batch.close()


def test_embedded_invalid_arguments(api):
    bad = synth.embedded_problem(0, seed=1)
    bad.w_rot = -1.0
    with pytest.raises(api.OptError) as ei:
        api.Problem(bad)
    assert ei.value.status == 1
    bad = synth.embedded_problem(0, seed=1)
    bad.v1 = bad.v1.copy()
    bad.v1[0] = bad.V
    with pytest.raises(api.OptError):
        api.Problem(bad)
    gp = api.Problem(synth.embedded_problem(0, seed=1))
    with pytest.raises(api.OptError):
        gp.solve_lm(2, 2, materialized=1)
    gp.close()


def test_embedded_plain_cg_lm(api):
    """use_precond = 0 (M^-1 = 1) under LM, against the oracle's."""
    prob = synth.embedded_problem(2, seed=95, handle_frac=0.05)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 4, 10, use_precond=False)
    gp = api.Problem(prob)
    rep = gp.solve_lm(4, 10, use_precond=0)
    assert rep["accepted"] == int(sum(ref.accepted))
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
