"""Volumetric ARAP deformation (Fig. 31) on its implicit voxel grid against
the FP64 oracle, against the same energy given as an explicit graph, in a
batch, and materialized."""
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
    return float(np.linalg.norm(np.asarray(a, np.float64).reshape(-1) - b) / max(np.linalg.norm(b), 1e-30))


def relE(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def as_graph(vp):
    v0, v1 = synth.volume_edges(vp.W, vp.H, vp.D)
    return synth.MeshProblem(vp.V, vp.urshape, v0, v1, vp.x0, vp.handle_idx, vp.handle_target,
                             vp.w_reg, vp.w_fit)


SIZES = [(1, 1, 1), (5, 4, 3), (13, 7, 9), (1, 6, 30)]


@pytest.mark.parametrize("W,H,D", SIZES)
@pytest.mark.parametrize("lam", [0.0, 0.35])
def test_volume_apply_and_jtf_match_oracle(api, W, H, D, lam):
    import torch
    vp = synth.volume_problem(W, H, D, max(1, W * H * D // 20), seed=401, x0_noise=0.3)
    e = oracle.make_energy(vp)
    x = vp.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(vp)
    p = np.random.default_rng(5).standard_normal(vp.n_unknowns).astype(np.float32)
    q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
    jtf, diag, E = oracle.jtf_diag(e, x)
    qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(diag, 1e-6, 1e32))
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    g, d, Eg = gp.eval_jtf()
    assert rel(g.cpu().numpy(), jtf) <= TOL_PRODUCT
    assert rel(d.cpu().numpy(), diag) <= TOL_PRODUCT
    assert relE(Eg, E) <= TOL_PRODUCT


def test_volume_implicit_grid_equals_explicit_graph(api):
    import torch
    vp = synth.volume_problem(17, 9, 11, 30, seed=402, x0_noise=0.2)
    a, b = api.Problem(vp), api.Problem(as_graph(vp))
    p = torch.as_tensor(np.random.default_rng(6).standard_normal(vp.n_unknowns).astype(np.float32), device="cuda")
    qa, _ = a.apply_jtj(p, 0.2)
    qb, _ = b.apply_jtj(p, 0.2)
    assert rel(qa.cpu().numpy(), qb.cpu().numpy().astype(np.float64)) <= 1e-6
    ra, rb = a.solve_lm(4, 15), b.solve_lm(4, 15)
    assert ra["accepted"] == rb["accepted"]
    for x, y in zip(ra["E_history"], rb["E_history"]):
        assert relE(x, y) <= 1e-5


@pytest.mark.parametrize("method", ["gn", "lm"])
def test_volume_solve_matches_oracle(api, method):
    # the paper's volumetric size: 4,961 voxels (here 11 x 11 x 41), 30 k unknowns
    vp = synth.volume_problem(11, 11, 41, 40, seed=synth.BASE_SEED)
    e = oracle.make_energy(vp)
    x0 = vp.x0.reshape(-1)
    ref = (oracle.gauss_newton(e, x0, 4, 20) if method == "gn" else oracle.levenberg_marquardt(e, x0, 6, 20))
    gp = api.Problem(vp)
    rep = gp.solve_gn(4, 20) if method == "gn" else gp.solve_lm(6, 20)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    if method == "lm":
        assert rep["accepted"] == int(sum(ref.accepted))


def test_volume_in_a_batch_equals_solo_and_materialized_agrees(api):
    probs = [synth.volume_problem(6, 5, 4, 8, seed=411), synth.volume_problem(9, 3, 7, 5, seed=412),
             synth.mesh_problem(1, seed=413, handle_frac=0.1)]
    solo = []
    for p in probs:
        g = api.Problem(p)
        solo.append(g.solve_lm(4, 10))
        g.close()
    members = [api.Problem(p) for p in probs]
    batch = api.Batch(members)
    reps, _ = batch.solve_lm(4, 10)
    for r, s_ in zip(reps, solo):
        assert r["E_history"] == s_["E_history"]
    batch.close()
    g = api.Problem(probs[0])
    rm = g.solve_lm(4, 10, materialized=1)
    for a, b in zip(rm["E_history"], solo[0]["E_history"]):
        assert relE(a, b) <= 1e-5
