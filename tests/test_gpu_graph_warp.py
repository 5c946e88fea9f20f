"""ARAP warping on an explicit graph (the explicit side of the implicit-grid
vs explicit-graph comparison, Fig. 18) against the FP64 oracle and against
the same warp solved on the implicit grid."""
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


def graph_warp(W, H, mask_frac, seed, noise=0.3, n_handles=None):
    mask = synth.random_mask(W, H, mask_frac, seed + 1) if mask_frac else None
    nh = max(1, (W * H) // 150) if n_handles is None else n_handles
    wp = synth.warp_problem(W, H, nh, seed=seed, mask=mask, x0_noise=noise)
    return wp, synth.warp_graph_from_grid(wp)


def random_graph(V, E, seed):
    """Not a grid: random positions, one-way and duplicated edges, isolated vertices."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, V - 3, E)
    b = (a + rng.integers(1, V - 3, E)) % (V - 3)
    keep = a != b
    a, b = a[keep], b[keep]
    order = np.lexsort((b, a))
    return synth.WarpGraphProblem(V=V, urshape=rng.uniform(-20, 20, (2, V)).astype(np.float32),
                                  v0=a[order].astype(np.int32), v1=b[order].astype(np.int32),
                                  x0=rng.uniform(-0.4, 0.4, (3, V)).astype(np.float32),
                                  handle_idx=rng.choice(V, 5, replace=False).astype(np.int32),
                                  handle_target=rng.uniform(-3, 3, (5, 2)).astype(np.float32))


CASES = [("grid", 37, 29, 0.0), ("grid", 64, 40, 0.2), ("random", 500, 2400, None)]


def make(case):
    kind, a, b, mf = case
    if kind == "grid":
        return graph_warp(a, b, mf, seed=311)[1]
    return random_graph(a, b, seed=312)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("lam", [0.0, 0.45])
def test_graph_warp_apply_and_jtf_match_oracle(api, case, lam):
    import torch
    prob = make(case)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = np.random.default_rng(3).standard_normal(prob.n_unknowns).astype(np.float32)
    q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
    jtf, diag, E = oracle.jtf_diag(e, x)
    qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(diag, 1e-6, 1e32))
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    g, d, Eg = gp.eval_jtf()
    assert rel(g.cpu().numpy(), jtf) <= TOL_PRODUCT
    assert rel(d.cpu().numpy(), diag) <= TOL_PRODUCT
    assert relE(Eg, E) <= TOL_PRODUCT


@pytest.mark.parametrize("method", ["gn", "lm"])
def test_graph_warp_solve_matches_oracle_and_grid(api, method):
    # the 64 x 64, 8-handle configuration (GN contracts there, so float32 and
    # float64 trajectories stay together)
    wp, gwp = graph_warp(64, 64, 0.0, seed=synth.BASE_SEED, noise=0.0, n_handles=8)
    e = oracle.make_energy(gwp)
    x0 = gwp.x0.reshape(-1)
    ref = oracle.gauss_newton(e, x0, 5, 20) if method == "gn" else oracle.levenberg_marquardt(e, x0, 5, 20)
    graph = api.Problem(gwp)
    grid = api.Problem(wp)
    rg = getattr(graph, f"solve_{method}")(5, 20)
    rw = getattr(grid, f"solve_{method}")(5, 20)
    for a, b in zip(rg["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    for a, b in zip(rg["E_history"], rw["E_history"]):
        assert relE(a, b) <= TOL_ENERGY
    # the unknowns come back in the caller's vertex order = pixel order
    xg = graph.x.cpu().numpy().reshape(3, -1)
    xw = grid.x.cpu().numpy().reshape(3, -1)
    assert np.linalg.norm(xg - xw) <= 1e-3 * max(np.linalg.norm(xw), 1.0)


def test_graph_warp_in_a_batch_equals_solo(api):
    probs = [make(CASES[0]), make(CASES[2]), synth.mesh_problem(1, seed=331, handle_frac=0.1),
             synth.warp_problem(40, 30, 6, seed=332)]
    solo = []
    for p in probs:
        g = api.Problem(p)
        solo.append(g.solve_gn(3, 8))
        g.close()
    members = [api.Problem(p) for p in probs]
    batch = api.Batch(members)
    reps, _ = batch.solve_gn(3, 8)
    for r, s_ in zip(reps, solo):
        assert r["E_history"] == s_["E_history"]
    batch.close()


def test_graph_warp_rejects_materialized(api):
    g = api.Problem(make(CASES[0]))
    with pytest.raises(api.OptError) as ei:
        g.solve_gn(2, 4, materialized=1)
    assert ei.value.status == 1
