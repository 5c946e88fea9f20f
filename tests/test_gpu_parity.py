"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: J^T J p and J^T F relative error <= 1e-5 (norm-wise, float32
arithmetic), energies and final energies <= 1e-4 relative, identical outer
iteration counts.  Sizes span several 32x8 tiles with ragged tails, plus the
degenerate 1x1 / 1xN / Nx1 grids and small meshes.
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


def perturbed(prob, scale, seed):
    """Random state near x0 (excluded Poisson pixels keep their values)."""
    rng = np.random.default_rng(seed)
    x = prob.x0.astype(np.float32).copy()
    if prob.kind == "poisson":
        free = np.ones((prob.H, prob.W), bool) if prob.mask is None else prob.mask == 0
        x[:, free] += rng.uniform(-scale, scale, size=(4, int(free.sum()))).astype(np.float32)
    else:
        x += rng.uniform(-scale, scale, size=x.shape).astype(np.float32)
    prob.x0 = x
    return prob


def random_direction(prob, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(prob.n_unknowns).astype(np.float32)
    if prob.kind == "poisson" and prob.mask is not None:
        p.reshape(4, -1)[:, prob.mask.reshape(-1) != 0] = 0.0
    return p


GRID_CASES = [
    ("warp", 64, 64, 0.0), ("warp", 37, 29, 0.0), ("warp", 37, 29, 0.25), ("warp", 1, 1, 0.0),
    ("warp", 1, 45, 0.0), ("warp", 70, 1, 0.0), ("warp", 100, 70, 0.1),
    # 128-pixel tiles (float4 rows): exact, ragged and masked widths
    ("warp", 256, 24, 0.0), ("warp", 300, 41, 0.0), ("warp", 301, 17, 0.2), ("warp", 520, 9, 0.0),
    ("poisson", 64, 48, None), ("poisson", 45, 33, None), ("poisson", 1, 17, None), ("poisson", 96, 80, None),
    # Poisson on 128-pixel tiles: exact, ragged widths, and no mask at all (every pixel free)
    ("poisson", 256, 24, None), ("poisson", 300, 41, None), ("poisson", 301, 17, None), ("poisson", 520, 9, None),
    ("poisson", 290, 20, "nomask"),
]


def make_grid(kind, W, H, mask_frac, seed=11):
    if kind == "warp":
        mask = synth.random_mask(W, H, mask_frac, seed + 1) if mask_frac else None
        prob = synth.warp_problem(W, H, max(1, (W * H) // 200), seed=seed, mask=mask)
        return perturbed(prob, 0.5, seed + 2)
    prob = synth.poisson_problem(W, H, seed=seed)
    if mask_frac == "nomask":
        prob.mask = None
    return perturbed(prob, 0.2, seed + 2)


@pytest.mark.parametrize("kind,W,H,mf", GRID_CASES)
@pytest.mark.parametrize("lam", [0.0, 0.37])
def test_grid_apply_jtj(api, kind, W, H, mf, lam):
    import torch
    prob = make_grid(kind, W, H, mf)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    p = random_direction(prob, 5)
    gp = api.Problem(prob)
    q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
    jtf, diag, E = oracle.jtf_diag(e, x)
    Dc = np.clip(diag, 1e-6, 1e32)
    qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, Dc)
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    gp.close()


@pytest.mark.parametrize("kind,W,H,mf", GRID_CASES)
def test_grid_eval_jtf(api, kind, W, H, mf):
    prob = make_grid(kind, W, H, mf, seed=21)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    jtf, diag, E = gp.eval_jtf()
    rj, rd, rE = oracle.jtf_diag(e, x)
    assert rel(jtf.cpu().numpy(), rj) <= TOL_PRODUCT
    np.testing.assert_allclose(diag.cpu().numpy().reshape(-1), rd, rtol=1e-5, atol=1e-6)
    assert relE(E, rE) <= TOL_PRODUCT
    assert relE(gp.energy(), rE) <= TOL_PRODUCT
    gp.close()


MESH_CASES = [(0, 0.3), (1, 0.2), (3, 0.1)]


def make_mesh(level, noise, seed=31):
    prob = synth.mesh_problem(level, seed=seed, handle_frac=0.05)
    return perturbed(prob, noise, seed + 1)


@pytest.mark.parametrize("level,noise", MESH_CASES)
@pytest.mark.parametrize("lam", [0.0, 0.5])
@pytest.mark.parametrize("form", [0, 1])
def test_mesh_apply_jtj(api, level, noise, lam, form):
    import torch
    prob = make_mesh(level, noise)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    p = random_direction(prob, 7)
    gp = api.Problem(prob)
    gp.set_apply_form(form)
    q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
    _, diag, _ = oracle.jtf_diag(e, x)
    qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(diag, 1e-6, 1e32))
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    gp.close()


@pytest.mark.parametrize("level,noise", MESH_CASES)
def test_mesh_eval_jtf(api, level, noise):
    prob = make_mesh(level, noise, seed=41)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    jtf, diag, E = gp.eval_jtf()
    rj, rd, rE = oracle.jtf_diag(e, x)
    assert rel(jtf.cpu().numpy(), rj) <= TOL_PRODUCT
    np.testing.assert_allclose(diag.cpu().numpy().reshape(-1), rd, rtol=1e-5, atol=1e-6)
    assert relE(E, rE) <= TOL_PRODUCT
    gp.close()


@pytest.mark.parametrize("keep", [0.6, 1.0])
def test_mesh_one_way_edges_and_isolated_vertices(api, keep):
    """Directed edge lists need not be symmetric: drop a random part of the
    directed edges (some vertices lose all in- or out-edges) and duplicate a
    few; J^T J p, J^T F, diag and E still match the oracle."""
    import torch
    prob = make_mesh(2, 0.25, seed=61)
    rng = np.random.default_rng(5)
    sel = rng.random(prob.v0.size) < keep
    v0, v1 = prob.v0[sel], prob.v1[sel]
    dup = rng.choice(v0.size, size=7, replace=False)
    v0 = np.concatenate([v0, v0[dup]]).astype(np.int32)
    v1 = np.concatenate([v1, v1[dup]]).astype(np.int32)
    order = np.lexsort((v1, v0))
    prob = synth.MeshProblem(prob.V, prob.urshape, v0[order], v1[order], prob.x0, prob.handle_idx,
                             prob.handle_target)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = random_direction(prob, 4)
    for lam, form in ((0.0, 0), (0.4, 0), (0.0, 1), (0.4, 1)):
        gp.set_apply_form(form)
        q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        jtf, diag, E = oracle.jtf_diag(e, x)
        qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(diag, 1e-6, 1e32))
        assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
        assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    g, d, Eg = gp.eval_jtf()
    assert rel(g.cpu().numpy(), jtf) <= TOL_PRODUCT
    assert rel(d.cpu().numpy(), diag) <= TOL_PRODUCT
    assert relE(Eg, E) <= TOL_PRODUCT


@pytest.mark.parametrize("hub_edges", [600, 2600])
def test_mesh_hub_vertex(api, hub_edges):
    """A hub vertex joined to many others (both directions): its tile's halo
    outgrows the tiled apply's 384 staged neighbours (600) or its edges
    outgrow the 2,304 shared-memory slots (2600), so the product runs on the
    general path; J^T J p, J^T F and the LM damping still match the oracle."""
    import torch
    base = synth.mesh_problem(5, seed=71, handle_frac=0.02)
    rng = np.random.default_rng(3)
    others = rng.choice(np.arange(1, base.V), size=hub_edges, replace=False).astype(np.int32)
    v0 = np.concatenate([base.v0, np.zeros(hub_edges, np.int32), others]).astype(np.int32)
    v1 = np.concatenate([base.v1, others, np.zeros(hub_edges, np.int32)]).astype(np.int32)
    order = np.lexsort((v1, v0))
    prob = synth.MeshProblem(base.V, base.urshape, v0[order], v1[order], base.x0, base.handle_idx,
                             base.handle_target)
    prob = perturbed(prob, 0.1, 4)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    with pytest.raises(api.OptError):
        gp.set_apply_form(1)                       # beyond the tiled apply's capacities
    assert gp.config()["apply_form"] == -1
    p = random_direction(prob, 6)
    jtf, diag, E = oracle.jtf_diag(e, x)
    for lam in (0.0, 0.3):
        q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        qref = oracle.apply_jtj(e, x, p.astype(np.float64), lam, np.clip(diag, 1e-6, 1e32))
        assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
        assert relE(pq, float(p.astype(np.float64) @ qref)) <= TOL_PRODUCT
    g, d, Eg = gp.eval_jtf()
    assert rel(g.cpu().numpy(), jtf) <= TOL_PRODUCT
    assert relE(Eg, E) <= TOL_PRODUCT
    gp.close()


def test_mesh_unsorted_edges_are_sorted_by_the_library(api):
    import torch
    prob = make_mesh(2, 0.2, seed=51)
    perm = np.random.default_rng(0).permutation(prob.v0.size)
    shuffled = synth.MeshProblem(prob.V, prob.urshape, prob.v0[perm], prob.v1[perm], prob.x0,
                                 prob.handle_idx, prob.handle_target)
    p = random_direction(prob, 3)
    a = api.Problem(prob)
    b = api.Problem(shuffled)
    qa, _ = a.apply_jtj(torch.as_tensor(p, device="cuda"))
    qb, _ = b.apply_jtj(torch.as_tensor(p, device="cuda"))
    assert rel(qb.cpu().numpy(), qa.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("case", ["warp", "poisson", "mesh"])
def test_pcg_iterates_match_oracle(api, case):
    prob = {"warp": lambda: make_grid("warp", 45, 21, 0.0, seed=61),
            "poisson": lambda: make_grid("poisson", 40, 30, None, seed=62),
            "mesh": lambda: make_mesh(2, 0.2, seed=63)}[case]()
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    gp.pcg_init(0.0)
    J = e.jacobian(x)
    F = e.residuals(x)
    b = -(J.T @ F)
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    Minv = oracle.solver.jacobi_minv(diag)
    for k in (1, 3, 6):
        gp.pcg_init(0.0)
        gp.pcg_step(k)
        dl, r, p, it = gp.pcg_state()
        d_ref, n_done, r_ref = oracle.jacobi_pcg(lambda v: J.T @ (J @ v), b, Minv, k)
        assert it == n_done == k
        assert rel(dl.cpu().numpy(), d_ref) <= 1e-4
        assert rel(r.cpu().numpy(), r_ref) <= 1e-4


def test_gn_config_warp_64(api):
    """ARAP warp 64x64, 8 handles, GN 10 x 10, Jacobi PCG (the small configuration)."""
    prob = synth.warp_problem(64, 64, 8, seed=synth.BASE_SEED)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 10, 10)
    gp = api.Problem(prob)
    rep = gp.solve_gn(10, 10)
    assert rep["outer_done"] == 10 and rep["pcg_done"] == ref.pcg_done
    for k, (a, b) in enumerate(zip(rep["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    x = gp.x.cpu().numpy().reshape(-1)
    assert rel(x, ref.x) <= 1e-3
    assert relE(e.energy(x), ref.E_history[-1]) <= TOL_ENERGY


def test_gn_poisson_small(api):
    prob = synth.poisson_problem(96, 80, seed=71)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 4, 20)
    gp = api.Problem(prob)
    rep = gp.solve_gn(4, 20)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    # fixed pixels never move
    fixed = prob.mask != 0
    np.testing.assert_array_equal(gp.x.cpu().numpy()[:, fixed], prob.x0[:, fixed])


@pytest.mark.parametrize("layout", ["rectangle", "scattered"])
@pytest.mark.parametrize("lm", [False, True])
def test_wide_poisson_solves_skip_quads_without_free_pixels(api, layout, lm):
    """128-pixel Poisson tiles read and write only quads that hold a free
    pixel (PCGInit: quads within one pixel of one).  A free rectangle whose
    edges cut through tiles and a scattered free set (70 % of the pixels
    fixed at random, so most quads are partly free) solve like the oracle and
    like 32-pixel tiles, which skip nothing, and fixed pixels never move."""
    W, H = 300, 41
    prob = synth.poisson_problem(W, H, seed=191)
    if layout == "scattered":
        prob.mask = (np.random.default_rng(192).random((H, W)) < 0.7).astype(np.uint8)
    e = oracle.make_energy(prob)
    outer, inner = (4, 15) if lm else (3, 20)
    x0 = prob.x0.reshape(-1)
    ref = oracle.levenberg_marquardt(e, x0, outer, inner) if lm else oracle.gauss_newton(e, x0, outer, inner)
    a = api.Problem(prob, tile_w=128)
    b = api.Problem(prob, tile_w=32)
    solve = (lambda g: g.solve_lm(outer, inner)) if lm else (lambda g: g.solve_gn(outer, inner))
    ra, rb = solve(a), solve(b)
    assert len(ra["E_history"]) == len(ref.E_history)
    for x, y, z in zip(ra["E_history"], rb["E_history"], ref.E_history):
        assert relE(x, z) <= TOL_ENERGY
        assert relE(x, y) <= 1e-5
    fixed = prob.mask != 0
    np.testing.assert_array_equal(a.x.cpu().numpy()[:, fixed], prob.x0[:, fixed])
    assert rel(a.x.cpu().numpy(), b.x.cpu().numpy()) <= 1e-4
    a.close()
    b.close()


def test_gn_graph_replay_equals_direct_launches(api):
    prob = synth.warp_problem(50, 40, 6, seed=81)
    a = api.Problem(prob)
    b = api.Problem(prob)
    ra = a.solve_gn(3, 8, use_graph=1)
    rb = b.solve_gn(3, 8, use_graph=0)
    assert ra["E_history"] == rb["E_history"]
    assert np.array_equal(a.x.cpu().numpy(), b.x.cpu().numpy())
    # replaying the cached graph from the same start reproduces the solve
    a.x.copy_(__import__("torch").as_tensor(prob.x0, device="cuda"))
    ra2 = a.solve_gn(3, 8, use_graph=1)
    assert ra2["E_history"] == ra["E_history"]


def check_lm_trajectory(rep, ref):
    """Same outer count and accept / reject sequence as the oracle (a
    rejected step leaves x, hence the next energy, bit for bit unchanged),
    every energy within 1e-4, lambda_final within the bound its gain ratios
    allow (tests/lm_tolerance.py)."""
    from lm_tolerance import lambda_tolerance
    E = rep["E_history"]
    assert rep["outer_done"] == ref.outer_done
    assert rep["accepted"] == sum(ref.accepted)
    assert [E[k + 1] != E[k] for k in range(ref.outer_done)] == list(ref.accepted)
    for k, (a, b) in enumerate(zip(E, ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    tol = lambda_tolerance(ref, E)
    assert relE(rep["lambda_final"], ref.lambda_final) <= tol, (rep["lambda_final"], ref.lambda_final, tol)


@pytest.mark.parametrize("form", [0, 1])
def test_lm_mesh_small(api, form):
    prob = synth.mesh_problem(3, seed=91, handle_frac=0.02)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 6, 15)
    gp = api.Problem(prob)
    gp.set_apply_form(form)
    rep = gp.solve_lm(6, 15, lambda0=1e-3)
    check_lm_trajectory(rep, ref)


def test_lm_mesh_level7_configuration(api):
    """The mesh configuration as specified: icosphere level 7 (163,842
    vertices, 983,040 directed edges), 1% seeded handles with offsets in
    [-0.1, 0.1]^3, LM from lambda0 = 1e-3, 15 outer x 30 PCG iterations, in
    the launch configuration the benchmark times (autotuned granularity),
    against the float64 oracle.

    This trajectory amplifies rounding: its gain ratios stay near 0.1-0.2, and
    the oracle's own run with float32 storage of x, the PCG vectors and J^T J p
    (oracle.solver round_to) leaves the plain float64 run by ~1e-8 up to outer
    iteration 8 and by up to ~5e-4 by iteration 15.  So the float32 solver is
    held to: the same decisions (outer count, accept / reject sequence, PCG
    iterations), every energy within 1e-4 where that float32-storage run stays
    within 1e-5 of the plain one, within 8x the float32-storage run's
    deviation (its running maximum) after that, and lambda_final within the
    bound of tests/lm_tolerance.py.  The float64 solver, which stores
    everything in float64, is held to 1e-9 on the whole trajectory."""
    import multiprocessing as mp
    from lm_tolerance import oracle_mesh_lm, lambda_tolerance
    prob = synth.mesh_problem(7, seed=synth.BASE_SEED)
    with mp.get_context("spawn").Pool(2) as pool:
        j_ref = pool.apply_async(oracle_mesh_lm, (7, synth.BASE_SEED, 15, 30))
        j_emu = pool.apply_async(oracle_mesh_lm, (7, synth.BASE_SEED, 15, 30, "float32"))
        gp = api.Problem(prob)
        gp.autotune()
        rep = gp.solve_lm(15, 30, lambda0=1e-3)
        gp.close()
        g64 = api.ProblemF64(prob)
        r64 = g64.solve_lm(15, 30, lambda0=1e-3)
        g64.close()
        ref, emu = j_ref.get(), j_emu.get()
    E, Er, Ee = rep["E_history"], ref["E_history"], emu["E_history"]
    n = ref["outer_done"]
    assert rep["outer_done"] == n == r64["outer_done"] and len(E) == len(Er) == n + 1
    assert rep["accepted"] == sum(ref["accepted"]) == r64["accepted"]
    assert [E[k + 1] != E[k] for k in range(n)] == ref["accepted"]
    assert rep["pcg_done"] == ref["pcg_done"]
    run_max = 0.0
    for k in range(n + 1):
        dev = relE(Ee[k], Er[k])
        run_max = max(run_max, dev)
        tol = TOL_ENERGY if run_max <= 1e-5 else max(TOL_ENERGY, 8.0 * run_max)
        assert relE(E[k], Er[k]) <= tol, (k, E[k], Er[k], tol)
        assert relE(r64["E_history"][k], Er[k]) <= 1e-9, (k, r64["E_history"][k], Er[k])

    class R:        # the oracle result in the shape lambda_tolerance reads
        accepted, E_history, rho, pred = ref["accepted"], Er, ref["rho"], ref["pred"]
    tol = lambda_tolerance(R, E)
    assert relE(rep["lambda_final"], ref["lambda_final"]) <= tol, (rep["lambda_final"], ref["lambda_final"], tol)


def test_lm_rejections_follow_nielsen(api):
    prob = synth.poisson_problem(30, 20, seed=92)
    gp = api.Problem(prob)
    rep = gp.solve_lm(4, 10, lambda0=1e-3, eta=2.0)
    assert rep["accepted"] == 0 and rep["outer_done"] == 4
    assert rep["lambda_final"] == pytest.approx(1e-3 * 2 * 4 * 8 * 16, rel=1e-12)
    np.testing.assert_array_equal(gp.x.cpu().numpy(), prob.x0)


def test_lm_relative_tolerance_stops_like_oracle(api):
    prob = synth.warp_problem(48, 40, 6, seed=93)
    e = oracle.make_energy(prob)
    prm = oracle.LMParams(rel_tol=1e-2)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 10, 10, prm)
    gp = api.Problem(prob)
    rep = gp.solve_lm(10, 10, rel_tol=1e-2)
    assert rep["outer_done"] == ref.outer_done
    assert rep["converged"] == int(ref.outer_done < 10)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


def test_invalid_arguments(api):
    import ctypes
    import torch
    lib = api.load_library()
    prob = synth.warp_problem(8, 8, 2, seed=1)
    bad = synth.warp_problem(8, 8, 2, seed=1)
    bad.handle_idx = np.array([3, 3], np.int32)           # duplicate handle
    with pytest.raises(api.OptError) as ei:
        api.Problem(bad)
    assert ei.value.status == 1
    bad.handle_idx = np.array([3, 64], np.int32)          # out of range
    with pytest.raises(api.OptError):
        api.Problem(bad)
    bad = synth.warp_problem(8, 8, 2, seed=1)
    bad.urshape = bad.urshape.copy()
    bad.urshape[0, 2, 2] = np.nan                          # non-finite constant
    with pytest.raises(api.OptError):
        api.Problem(bad)
    m = synth.mesh_problem(0, seed=1)
    m.v1 = m.v1.copy()
    m.v1[0] = m.V                                          # edge out of range
    with pytest.raises(api.OptError):
        api.Problem(m)
    gp = api.Problem(prob)
    p = api.default_params(outer=0, inner=5)
    assert lib.opt_solve_gn(gp.h, ctypes.byref(p), None) == 1
    gp.close()
    torch.cuda.synchronize()


def test_full_size_warp_apply_and_solve_start(api):
    """ARAP warp 1024x1024 with 64 handles (the grid-at-scale configuration):
    J^T J p over the whole grid and the first GN iterations against the oracle."""
    import torch
    prob = synth.warp_problem(1024, 1024, 64, seed=synth.BASE_SEED)
    prob = perturbed(prob, 0.3, 5)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = random_direction(prob, 9)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian(x)
    qref = J.T @ (J @ p.astype(np.float64))
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    jtf, _, E = gp.eval_jtf()
    assert rel(jtf.cpu().numpy(), J.T @ e.residuals(x)) <= TOL_PRODUCT
    ref = oracle.gauss_newton(e, x, 2, 20)
    rep = gp.solve_gn(2, 20)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    # the launch configuration the benchmark times: autotuned granularity
    # (the solve above wrote its result into the unknowns: start over from x0)
    gp.autotune()
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    assert rel(q.cpu().numpy(), qref) <= TOL_PRODUCT
    rep = gp.solve_gn(2, 20)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


def test_full_size_poisson_apply(api):
    import torch
    prob = synth.poisson_problem(1024, 1024, seed=synth.BASE_SEED)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = random_direction(prob, 4)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian()
    assert rel(q.cpu().numpy(), J.T @ (J @ p.astype(np.float64))) <= TOL_PRODUCT
    ref = oracle.gauss_newton(e, x, 2, 20)
    rep = gp.solve_gn(2, 20)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


def test_full_size_mesh_apply(api):
    """Icosphere level 7 (163,842 vertices, 983,040 directed edges)."""
    import torch
    prob = synth.mesh_problem(7, seed=synth.BASE_SEED)
    prob = perturbed(prob, 0.05, 6)
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    gp = api.Problem(prob)
    p = random_direction(prob, 8)
    q, _ = gp.apply_jtj(torch.as_tensor(p, device="cuda"))
    J = e.jacobian(x)
    assert rel(q.cpu().numpy(), J.T @ (J @ p.astype(np.float64))) <= TOL_PRODUCT
    jtf, _, E = gp.eval_jtf()
    assert rel(jtf.cpu().numpy(), J.T @ e.residuals(x)) <= TOL_PRODUCT


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", ["warp", "warp_masked", "poisson", "mesh", "volume"])
def test_materialized_solve_matches_oracle_and_matrix_free(api, case, mode):
    """Materialized forms (Sec. 7): CSR J with q = J^T (J p) (mode 1) and J^T J
    assembled once per outer iteration with q = A p (mode 2, Fig. 16),
    against the oracle and the matrix-free path on the same problem."""
    import torch
    if case == "warp":
        prob, lm, outer, inner = synth.warp_problem(70, 45, 6, seed=101), False, 4, 10
    elif case == "warp_masked":
        prob = synth.warp_problem(61, 37, 5, seed=102, mask=synth.random_mask(61, 37, 0.2, 3))
        lm, outer, inner = False, 3, 10
    elif case == "poisson":
        prob, lm, outer, inner = synth.poisson_problem(96, 80, seed=103), False, 3, 20
    elif case == "mesh":
        prob, lm, outer, inner = synth.mesh_problem(3, seed=104, handle_frac=0.02), True, 5, 15
    else:
        prob, lm, outer, inner = synth.volume_problem(7, 6, 8, 12, seed=105), True, 4, 15
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    ref = (oracle.levenberg_marquardt(e, x0, outer, inner) if lm else oracle.gauss_newton(e, x0, outer, inner))
    a, b = api.Problem(prob), api.Problem(prob)
    solve = (lambda g, **kw: g.solve_lm(outer, inner, **kw)) if lm else (lambda g, **kw: g.solve_gn(outer, inner, **kw))
    rm = solve(a, materialized=mode)
    rf = solve(b, materialized=0)
    assert rm["outer_done"] == rf["outer_done"] == (ref.outer_done if lm else outer)
    for x, y, z in zip(rm["E_history"], rf["E_history"], ref.E_history):
        assert relE(x, z) <= TOL_ENERGY
        assert relE(x, y) <= 1e-5
    assert rel(a.x.cpu().numpy(), b.x.cpu().numpy()) <= 1e-4
    # a second materialized solve from the same start replays the cached graph
    a.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    rm2 = solve(a, materialized=mode)
    assert rm2["E_history"] == rm["E_history"] or all(relE(x, y) <= 1e-6 for x, y in zip(rm2["E_history"], rm["E_history"]))


@pytest.mark.parametrize("W,H,mf", [(100, 30, 0.0), (33, 20, 0.3), (5, 7, 0.0)])
def test_wide_tiles_forced_on_narrow_grids(api, W, H, mf):
    """128-wide tiles on grids narrower than a tile (pitch padding, halo
    columns outside the image) give the same products as 32-wide tiles."""
    import torch
    for kind in ("warp", "poisson"):
        _forced_tiles_case(api, kind, W, H, mf)


def _forced_tiles_case(api, kind, W, H, mf):
    import torch
    prob = make_grid(kind, W, H, mf if kind == "warp" else None, seed=131)
    p = random_direction(prob, 2)
    a = api.Problem(prob, tile_w=128)
    b = api.Problem(prob, tile_w=32)
    for lam in (0.0, 0.3):
        qa, pqa = a.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        qb, pqb = b.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        assert rel(qa.cpu().numpy(), qb.cpu().numpy()) <= 1e-6
        assert relE(pqa, pqb) <= 1e-6
    ra = a.solve_gn(3, 6)
    rb = b.solve_gn(3, 6)
    for x, y in zip(ra["E_history"], rb["E_history"]):
        assert relE(x, y) <= 1e-5


def test_gn_wide_tiles_match_oracle(api):
    """A 320 x 64 warp (128-wide tiles, ragged last tile) through GN 4 x 10."""
    prob = synth.warp_problem(320, 64, 12, seed=141)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 4, 10)
    gp = api.Problem(prob)
    rep = gp.solve_gn(4, 10)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY


@pytest.mark.parametrize("kind", ["warp", "mesh"])
def test_chunking_and_autotune_keep_results(api, kind):
    prob = synth.warp_problem(300, 90, 9, seed=151) if kind == "warp" else synth.mesh_problem(3, seed=152)
    a = api.Problem(prob)
    ref = a.solve_gn(3, 8)
    for per in (1, 5, -3, 0):
        a.set_chunking(per)
        a.x.copy_(__import__("torch").as_tensor(prob.x0, device="cuda"))
        r = a.solve_gn(3, 8)
        for x, y in zip(r["E_history"], ref["E_history"]):
            assert relE(x, y) <= 1e-6
    chosen, ms = a.autotune()
    assert chosen in (-1, -2, -3, -4, -6, -8, 1, 4) and ms > 0
    a.x.copy_(__import__("torch").as_tensor(prob.x0, device="cuda"))
    r = a.solve_gn(3, 8)
    for x, y in zip(r["E_history"], ref["E_history"]):
        assert relE(x, y) <= 1e-6


@pytest.mark.parametrize("W,H,mf,method,graph", [(1024, 1024, 0.0, "gn", 1), (700, 300, 0.2, "lm", 1),
                                                 (260, 20, 0.0, "lm", 0)])
def test_persistent_pcg_equals_per_step_launches(api, W, H, mf, method, graph):
    """The persistent PCG loop (one cooperative launch per outer iteration,
    grid-wide barriers) runs the same arithmetic in the same order as one
    launch per PCG kernel: identical energies, PCG counts and unknowns."""
    mask = synth.random_mask(W, H, mf, 3) if mf else None
    prob = synth.warp_problem(W, H, synth.warp_handle_count(W, H), seed=161, mask=mask)
    a, b = api.Problem(prob), api.Problem(prob)
    ra = getattr(a, f"solve_{method}")(4, 12, persistent=1, use_graph=graph)
    rb = getattr(b, f"solve_{method}")(4, 12, persistent=0, use_graph=graph)
    assert ra["status"] == rb["status"] == "OPT_OK"
    assert ra["E_history"] == rb["E_history"]
    assert ra["pcg_done"] == rb["pcg_done"] and ra["accepted"] == rb["accepted"]
    assert np.array_equal(a.x.cpu().numpy(), b.x.cpu().numpy())
    # and against the oracle
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    ref = (oracle.gauss_newton(e, x0, 4, 12) if method == "gn" else oracle.levenberg_marquardt(e, x0, 4, 12))
    for x, y in zip(ra["E_history"], ref.E_history):
        assert relE(x, y) <= TOL_ENERGY


@pytest.mark.parametrize("kind,inner", [("poisson", 10), ("mesh", 10), ("warp", 3)])
def test_plain_cg_matches_oracle(api, kind, inner):
    """use_precond = 0 (M^-1 = 1).  Poisson and the mesh follow the oracle
    over 10 CG iterations; on the warp, whose fit rows weigh 100 against
    stencil rows of 4 .. 8, unpreconditioned CG amplifies rounding about
    100-fold per iteration (float32 vs float64: 7e-7 after 3 iterations, 5e-2
    after 8), so it is checked over 3 -- the Jacobi preconditioner removes
    this (float32 within 1e-7 at any count)."""
    prob = {"warp": lambda: synth.warp_problem(40, 30, 5, seed=17),
            "poisson": lambda: synth.poisson_problem(48, 40, seed=18),
            "mesh": lambda: synth.mesh_problem(2, seed=19, handle_frac=0.05)}[kind]()
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 2, inner, use_precond=False)
    gp = api.Problem(prob)
    rep = gp.solve_gn(2, inner, use_precond=0)
    assert rep["pcg_done"] == ref.pcg_done
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    gp.close()


def test_autotuned_configurations_keep_results(api):
    """The autotuner's choices -- granularity, a grid's tile width (re-planned
    from the creation descriptor), an ARAP mesh's apply form -- give the same
    results within 1e-6: every sum is compensated, so only the float32
    arithmetic of each element's own rows may differ."""
    import torch
    w = synth.warp_problem(300, 90, 9, seed=171)
    a = api.Problem(w)
    ref = a.solve_gn(3, 8)
    for tw in (32, 128):
        b = api.Problem(w, tile_w=tw)
        assert b.config()["tile_w"] == tw and b.config()["apply_form"] == -1
        r = b.solve_gn(3, 8)
        for x, y in zip(r["E_history"], ref["E_history"]):
            assert relE(x, y) <= 1e-6
        b.close()
    a.autotune()
    cfg = a.config()
    assert cfg["tile_w"] in (32, 128) and cfg["chunking"] in (-1, -2, -3, -4, -6, -8, 1, 4)
    a.x.copy_(torch.as_tensor(w.x0, device="cuda"))
    r = a.solve_gn(3, 8)
    for x, y in zip(r["E_history"], ref["E_history"]):
        assert relE(x, y) <= 1e-6
    a.close()
    m = synth.mesh_problem(3, seed=172, handle_frac=0.03)
    g = api.Problem(m)
    assert g.config()["apply_form"] == 0          # the two-pass gather by default
    g.set_apply_form(1)                            # tiled: tables built on first use
    assert g.config()["apply_form"] == 1
    p = random_direction(m, 3)
    q1, pq1 = g.apply_jtj(torch.as_tensor(p, device="cuda"), 0.2)
    r1 = g.solve_lm(4, 10)
    g.set_apply_form(0)
    g.x.copy_(torch.as_tensor(m.x0, device="cuda"))
    q0, pq0 = g.apply_jtj(torch.as_tensor(p, device="cuda"), 0.2)
    r0 = g.solve_lm(4, 10)
    assert rel(q1.cpu().numpy(), q0.cpu().numpy()) <= 1e-6 and relE(pq1, pq0) <= 1e-6
    assert r1["outer_done"] == r0["outer_done"]
    for x, y in zip(r1["E_history"], r0["E_history"]):
        assert relE(x, y) <= 1e-6
    g.autotune()
    assert g.config()["apply_form"] in (0, 1)
    with pytest.raises(api.OptError):
        g.set_apply_form(2)
    g.close()


@pytest.mark.parametrize("case", ["warp128", "warp32", "poisson", "mesh_gather", "mesh_tiled", "volume", "embedded"])
def test_dot_products_carry_float64_accuracy(api, case):
    """p.q from the applyJTJ pass (the scalar behind alpha) equals the float64
    dot product of the float32 vectors p and q the pass returns, to 1e-9
    relative: the compensated (Dot2) accumulation loses essentially nothing,
    where a float32 sum over ~1e6 terms would be off by ~1e-6."""
    import torch
    if case.startswith("warp"):
        prob = perturbed(synth.warp_problem(520, 300, 40, seed=181), 0.3, 2)
        gp = api.Problem(prob, tile_w=128 if case == "warp128" else 32)
    elif case == "poisson":
        prob = synth.poisson_problem(600, 400, seed=182)
        gp = api.Problem(prob)
    elif case == "volume":
        prob = synth.volume_problem(40, 30, 20, 50, seed=184)
        gp = api.Problem(prob)
    elif case == "embedded":
        prob = synth.embedded_problem(5, seed=185, x0_noise=0.05)
        gp = api.Problem(prob)
    else:
        prob = make_mesh(5, 0.1, seed=183)
        gp = api.Problem(prob)
        gp.set_apply_form(1 if case == "mesh_tiled" else 0)
    p = random_direction(prob, 11)
    for lam in (0.0, 0.25):
        q, pq = gp.apply_jtj(torch.as_tensor(p, device="cuda"), lam)
        exact = float(np.dot(p.astype(np.float64), q.cpu().numpy().reshape(-1).astype(np.float64)))
        assert relE(pq, exact) <= 1e-9, (case, lam, pq, exact)
    gp.close()


@pytest.mark.parametrize("method,mf,form", [("gn", 0.0, 0), ("gn", 0.2, 1), ("lm", 0.0, 1), ("lm", 0.2, 0)])
def test_wide_warp_init_reads_cos_sin_of_previous_update(api, method, mf, form):
    """From the second outer iteration on, the wide warp's PCGInit takes cos /
    sin of theta from the planes the previous outer update wrote instead of
    evaluating them: E(x_k) it reports must equal the energy evaluated
    independently (opt_eval_energy, its own cos / sin) at the same x_k, to
    the rounding of two differently ordered float32 residual evaluations
    (both sums compensated; about 1e-9 here, where cos / sin of the previous
    iterate would be off by the step's rotation, 1e-3 and more)."""
    import torch
    prob = make_grid("warp", 260, 24, mf, seed=171)
    gp = api.Problem(prob)
    x0 = torch.as_tensor(prob.x0, device="cuda")
    solve = getattr(gp, f"solve_{method}")
    rep = solve(3, 6, pcg_form=form)
    for k in (1, 2):
        gp.x.copy_(x0)
        rk = solve(k, 6, pcg_form=form)
        assert rk["E_history"][:k] == rep["E_history"][:k]
        Ek = gp.energy()
        assert relE(rep["E_history"][k], Ek) <= 1e-8, (k, rep["E_history"][k], Ek)
        assert relE(rk["E_history"][k], Ek) <= 1e-8
