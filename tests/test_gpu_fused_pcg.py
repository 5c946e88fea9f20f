"""The single-reduction PCG iteration (opt_solve_params.pcg_form = 1) of the
wide-tile ARAP warp against the FP64 oracle's textbook Jacobi-PCG (Saad,
Alg. 9.1; the paper's PCG of Sec. 4.1) and GN / LM (Sec. 4).

The form computes the same Krylov iterates as the two-pass PCG in exact
arithmetic, so the oracle is the same: the step delta after k iterations
(read back as x - x0 after one GN outer iteration of k PCG iterations, since
GN sets x = x0 + delta) within 1e-4 norm-wise, as the two-pass iterates are
held in test_gpu_parity.py, and energies within the stated 1e-4 with the
same outer-iteration count.  Grids are at least 128 pixels wide (the form
runs on 128-pixel tiles), with ragged widths and heights, masks, handles.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu

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


def warp(W, H, mask_frac, seed, perturb=0.5, n_handles=None):
    mask = synth.random_mask(W, H, mask_frac, seed + 1) if mask_frac else None
    prob = synth.warp_problem(W, H, n_handles or max(1, (W * H) // 200), seed=seed, mask=mask)
    if perturb:
        rng = np.random.default_rng(seed + 2)
        prob.x0 = (prob.x0 + rng.uniform(-perturb, perturb, size=prob.x0.shape)).astype(np.float32)
    return prob


CASES = [(128, 8, 0.0), (256, 24, 0.0), (300, 21, 0.0), (301, 17, 0.2), (520, 9, 0.0), (200, 37, 0.3)]


@pytest.mark.parametrize("W,H,mf", CASES)
def test_fused_iterates_match_oracle(api, W, H, mf):
    """delta after k = 1, 3, 6 single-reduction iterations equals the
    oracle's textbook PCG step from the same start."""
    import torch
    prob = warp(W, H, mf, seed=W + H)
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x0)
    b = -(J.T @ e.residuals(x0))
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    Minv = oracle.solver.jacobi_minv(diag)
    gp = api.Problem(prob)
    assert gp.config()["tile_w"] == 128
    for k in (1, 3, 6):
        gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
        rep = gp.solve_gn(1, k, pcg_form=1)
        d_ref, n_done, _ = oracle.jacobi_pcg(lambda v: J.T @ (J @ v), b, Minv, k)
        assert rep["pcg_done"] == n_done == k
        d = gp.x.cpu().numpy().reshape(-1).astype(np.float64) - prob.x0.reshape(-1)
        assert rel(d, d_ref) <= 1e-4, (k, rel(d, d_ref))


@pytest.mark.parametrize("W,H,mf", [(320, 64, 0.0), (300, 41, 0.2)])
def test_fused_gn_matches_oracle_and_two_pass(api, W, H, mf):
    """GN 4 x 10 from the unperturbed start: every outer energy within 1e-4
    of the oracle, the same PCG count, and within rounding of the two-pass
    form."""
    import torch
    prob = warp(W, H, mf, seed=141, perturb=0.0, n_handles=12)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 4, 10)
    gp = api.Problem(prob)
    rep1 = gp.solve_gn(4, 10, pcg_form=1)
    x1 = gp.x.cpu().numpy()
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    rep0 = gp.solve_gn(4, 10, pcg_form=0)
    assert rep1["outer_done"] == rep0["outer_done"] == 4
    assert rep1["pcg_done"] == ref.pcg_done
    for k, (a, b) in enumerate(zip(rep1["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    for a, b in zip(rep1["E_history"], rep0["E_history"]):
        assert relE(a, b) <= 1e-5
    assert relE(e.energy(x1.reshape(-1)), ref.E_history[-1]) <= TOL_ENERGY


def test_fused_lm_matches_oracle(api):
    """LM (damping in the product and in the preconditioner): the same
    accept / reject sequence and outer count as the oracle, energies within
    1e-4."""
    prob = warp(260, 40, 0.1, seed=77, perturb=0.3)
    e = oracle.make_energy(prob)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 6, 15)
    gp = api.Problem(prob)
    rep = gp.solve_lm(6, 15, pcg_form=1)
    assert rep["outer_done"] == ref.outer_done
    assert rep["accepted"] == sum(ref.accepted)
    for k, (a, b) in enumerate(zip(rep["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)


def test_fused_isolated_pixels_stop_after_exact_step(api):
    """Every free pixel isolated (no free neighbour): J^T J is diagonal, the
    Jacobi preconditioner inverts it and the first PCG step is exact.  The
    recurrence r.z then drops to rounding level (or below zero, which stops
    the loop with the known step still applied); the remaining iterations
    must leave delta at the exact step."""
    import torch
    W, H = 160, 9
    mask = np.ones((H, W), np.uint8)
    mask[::2, ::2] = 0
    prob = synth.warp_problem(W, H, 20, seed=5, mask=mask)
    rng = np.random.default_rng(8)
    prob.x0 = (prob.x0 + rng.uniform(-0.5, 0.5, size=prob.x0.shape)).astype(np.float32)
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x0)
    b = -(J.T @ e.residuals(x0))
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    d_exact = np.where(diag > 0, b / np.where(diag > 0, diag, 1.0), 0.0)
    gp = api.Problem(prob)
    for inner in (1, 2, 5):
        gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
        rep = gp.solve_gn(1, inner, pcg_form=1)
        assert rep["status"] == "OPT_OK"
        d = gp.x.cpu().numpy().reshape(-1).astype(np.float64) - x0
        assert rel(d, d_exact) <= 1e-5, (inner, rel(d, d_exact))


def test_fused_full_size_configuration(api):
    """ARAP warp 1024 x 1024, 64 handles, GN 20 x 20 (the grid-at-scale
    configuration) at the autotuned launch configuration: the first two outer
    iterations' energies against the oracle, the whole solve's energies
    within rounding of the two-pass form."""
    import torch
    prob = synth.warp_problem(1024, 1024, 64, seed=synth.BASE_SEED)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 2, 20)
    gp = api.Problem(prob)
    gp.autotune()
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    rep = gp.solve_gn(2, 20, pcg_form=1)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    r1 = gp.solve_gn(20, 20, pcg_form=1)
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    r0 = gp.solve_gn(20, 20, pcg_form=0)
    assert r1["pcg_done"] == r0["pcg_done"] == 400
    for a, b in zip(r1["E_history"], r0["E_history"]):
        assert relE(a, b) <= 1e-5


@pytest.mark.parametrize("kind,W,H", [("warp", 32767, 1), ("warp", 32767, 2), ("warp", 128, 1), ("warp", 133, 3),
                                      ("poisson", 4099, 2), ("poisson", 300, 3)])
def test_fused_extreme_extents(api, kind, W, H):
    """Grids of one row of 128-pixel tiles, below one tile's height (down to
    a single pixel row), up to the widest extent the planner accepts: GN
    2 x 5 with the single-reduction iteration, energies against the oracle
    and the same PCG iteration count."""
    prob = synth.warp_problem(W, H, 20, seed=5) if kind == "warp" else synth.poisson_problem(W, H, seed=4)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1).astype(np.float64), 2, 5)
    gp = api.Problem(prob)
    assert gp.config()["tile_w"] == 128
    rep = gp.solve_gn(2, 5, pcg_form=1)
    assert rep["status"] == "OPT_OK" and rep["pcg_done"] == ref.pcg_done
    for k, (a, b) in enumerate(zip(rep["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    gp.close()


def test_fused_all_pixels_excluded_or_fixed(api):
    """Every warp pixel masked or every Poisson pixel fixed, on 128-pixel
    tiles: r = 0, the first iteration breaks down (p.q = 0) with no step,
    E = 0 and nothing moves."""
    w = synth.warp_problem(130, 8, 0, seed=5, mask=np.ones((8, 130), np.uint8))
    p = synth.poisson_problem(140, 10, seed=4)
    p.mask = np.ones((10, 140), np.uint8)
    for prob in (w, p):
        gp = api.Problem(prob)
        assert gp.config()["tile_w"] == 128
        rep = gp.solve_gn(2, 5, pcg_form=1)
        assert rep["status"] == "OPT_OK"
        assert rep["E_history"] == [0.0, 0.0, 0.0] and rep["pcg_done"] == 0
        np.testing.assert_array_equal(gp.x.cpu().numpy(), prob.x0)
        gp.close()


def test_fused_form_on_other_problems_runs_two_pass(api):
    """pcg_form = 1 on problems the form does not cover (32-pixel tiles) runs
    the two-pass iteration: bit-identical results."""
    import torch
    for prob in (warp(100, 30, 0.0, seed=3), synth.poisson_problem(100, 40, seed=4)):
        gp = api.Problem(prob)
        r0 = gp.solve_gn(2, 5, pcg_form=0)
        gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
        r1 = gp.solve_gn(2, 5, pcg_form=1)
        assert r0["E_history"] == r1["E_history"]
    gp = api.Problem(warp(256, 8, 0.0, seed=9))
    with pytest.raises(Exception):
        gp.solve_gn(1, 1, pcg_form=2)


@pytest.mark.parametrize("method", ["gn", "lm"])
def test_fused_batch_matches_solo_and_oracle(api, method):
    """A batch with pcg_form = 1: its wide-tile warps (masked and not) take
    the single-reduction iteration, its narrow warps and Poisson members the
    two-pass one; every member equals its solo solve with the same parameter
    bit for bit (the batch keeps each member's chunks), and the wide warps
    match the oracle within 1e-4."""
    probs = [warp(260, 20, 0.0, seed=301, perturb=0.0, n_handles=6),
             warp(300, 16, 0.1, seed=302, perturb=0.0, n_handles=6),
             warp(129, 40, 0.0, seed=303, perturb=0.0, n_handles=4),
             warp(60, 33, 0.0, seed=304, perturb=0.0, n_handles=4),
             synth.poisson_problem(300, 24, seed=305)]
    outer, inner = (3, 8) if method == "gn" else (4, 8)
    solo = []
    for p in probs:
        g = api.Problem(p)
        solo.append(getattr(g, f"solve_{method}")(outer, inner, pcg_form=1))
        g.close()
    members = [api.Problem(p) for p in probs]
    batch = api.Batch(members)
    reps, _ = getattr(batch, f"solve_{method}")(outer, inner, pcg_form=1)
    for r, s in zip(reps, solo):
        assert r["outer_done"] == s["outer_done"] and r["accepted"] == s["accepted"]
        assert r["E_history"] == s["E_history"]
    for i in (0, 1, 2):
        e = oracle.make_energy(probs[i])
        x0 = probs[i].x0.reshape(-1)
        ref = (oracle.gauss_newton(e, x0, outer, inner) if method == "gn"
               else oracle.levenberg_marquardt(e, x0, outer, inner))
        for a, b in zip(reps[i]["E_history"], ref.E_history):
            assert relE(a, b) <= TOL_ENERGY
    batch.close()
    for m in members:
        m.close()


def test_fused_lm_relative_tolerance_stops_like_oracle(api):
    """LM with rel_tol: the loop stops at the oracle's outer iteration, the
    later launches of the solve graph (single-reduction iterations and last
    step included) leave the converged state alone."""
    prob = warp(256, 30, 0.0, seed=91, perturb=0.2)
    e = oracle.make_energy(prob)
    prm = oracle.solver.LMParams(rel_tol=1e-2)
    ref = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), 12, 10, prm)
    gp = api.Problem(prob)
    rep = gp.solve_lm(12, 10, rel_tol=1e-2, pcg_form=1)
    assert rep["outer_done"] == ref.outer_done < 12
    assert rep["converged"] == 1
    assert rep["accepted"] == sum(ref.accepted)
    for a, b in zip(rep["E_history"], ref.E_history):
        assert relE(a, b) <= TOL_ENERGY
    x = gp.x.cpu().numpy().reshape(-1)
    assert relE(e.energy(x), ref.E_history[-1]) <= TOL_ENERGY


def test_fused_server_requests_equal_solo(api):
    """The server with pcg_form = 1: wide warps (single-reduction), a narrow
    warp and a mesh (two-pass), some joining while others run; every result
    equals its solo LM solve with the same parameters, bit for bit on the
    grids (each member keeps its own chunks), and differs from the two-pass
    form's result (the server took the single-reduction iteration)."""
    probs = [warp(200, 24, 0.0, seed=501, perturb=0.0, n_handles=5),
             warp(300, 17, 0.1, seed=502, perturb=0.0, n_handles=5),
             warp(64, 40, 0.0, seed=503, perturb=0.0, n_handles=3),
             warp(140, 60, 0.0, seed=504, perturb=0.0, n_handles=6),
             synth.mesh_problem(1, seed=505, handle_frac=0.1)]
    refs = []
    for p in probs:
        g = api.Problem(p)
        r = g.solve_lm(8, 10, rel_tol=1e-6, pcg_form=1)
        refs.append((r, g.x.cpu().numpy().copy()))
        g.close()
    srv = api.Server(4 << 30, outer=8, inner=10, rel_tol=1e-6, pcg_form=1)
    tickets = [srv.submit(p) for p in probs[:3]]
    srv.step()
    tickets += [srv.submit(p) for p in probs[3:]]
    done = {}
    for _ in range(200):
        srv.step()
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        if len(done) == len(tickets):
            break
    assert len(done) == len(tickets)
    for k, (p, t, (ref, xref)) in enumerate(zip(probs, tickets, refs)):
        rep, x = done[t]
        assert rep["status"] == "OPT_OK"
        assert rep["outer_done"] == ref["outer_done"] and rep["accepted"] == ref["accepted"]
        if p.kind != "mesh":
            # the energies at the start of every outer iteration, bit for bit
            # (the last entry is the final energy, evaluated by another kernel)
            assert rep["E_history"][:-1] == ref["E_history"][:-1], k
        if k in (0, 1, 3):       # the wide warps: the two-pass form rounds differently
            g = api.Problem(p)
            r0 = g.solve_lm(8, 10, rel_tol=1e-6, pcg_form=0)
            g.close()
            assert r0["E_history"][:-1] != ref["E_history"][:-1]
        tol = 1e-5 if p.kind == "mesh" else 1e-6
        for a, b in zip(rep["E_history"][:-1], ref["E_history"][:-1]):
            assert relE(a, b) <= tol
        assert relE(rep["E_final"], ref["E_final"]) <= 1e-5
        d = np.linalg.norm(x.cpu().numpy().reshape(-1) - xref.reshape(-1)) / max(np.linalg.norm(xref), 1e-30)
        assert d <= (1e-4 if p.kind == "mesh" else 1e-6)
    srv.close()


POISSON_CASES = [(256, 24), (300, 41), (520, 9), (129, 33)]


@pytest.mark.parametrize("W,H", POISSON_CASES)
def test_fused_poisson_iterates_match_oracle(api, W, H):
    """Poisson editing on 128-pixel tiles: delta after k = 1, 3, 6
    single-reduction iterations equals the oracle's textbook PCG step; fixed
    pixels never move."""
    import torch
    prob = synth.poisson_problem(W, H, seed=W + 2 * H)
    rng = np.random.default_rng(W)
    free = prob.mask == 0
    prob.x0[:, free] += rng.uniform(-0.2, 0.2, size=(4, int(free.sum()))).astype(np.float32)
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x0)
    b = -(J.T @ e.residuals(x0))
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    Minv = oracle.solver.jacobi_minv(diag)
    gp = api.Problem(prob)
    assert gp.config()["tile_w"] == 128
    for k in (1, 3, 6):
        gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
        rep = gp.solve_gn(1, k, pcg_form=1)
        d_ref, n_done, _ = oracle.jacobi_pcg(lambda v: J.T @ (J @ v), b, Minv, k)
        assert rep["pcg_done"] == n_done == k
        x = gp.x.cpu().numpy()
        d = x.reshape(-1).astype(np.float64) - x0
        assert rel(d, d_ref) <= 1e-4, (k, rel(d, d_ref))
        np.testing.assert_array_equal(x[:, ~free], prob.x0[:, ~free])


@pytest.mark.parametrize("method", ["gn", "lm"])
def test_fused_poisson_solve_matches_oracle_and_two_pass(api, method):
    """Poisson 300 x 41 x 4 through GN 4 x 20 / LM 5 x 15 with the
    single-reduction iteration: energies within 1e-4 of the oracle (same
    outer count and accepted steps under LM) and within rounding of the
    two-pass form."""
    import torch
    prob = synth.poisson_problem(300, 41, seed=77)
    e = oracle.make_energy(prob)
    outer, inner = (4, 20) if method == "gn" else (5, 15)
    x0 = prob.x0.reshape(-1)
    ref = oracle.gauss_newton(e, x0, outer, inner) if method == "gn" else \
        oracle.levenberg_marquardt(e, x0, outer, inner)
    gp = api.Problem(prob)
    solve = getattr(gp, f"solve_{method}")
    r1 = solve(outer, inner, pcg_form=1)
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    r0 = solve(outer, inner, pcg_form=0)
    assert r1["outer_done"] == r0["outer_done"] == (outer if method == "gn" else ref.outer_done)
    if method == "lm":
        assert r1["accepted"] == sum(ref.accepted)
    for k, (a, b) in enumerate(zip(r1["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    for a, b in zip(r1["E_history"], r0["E_history"]):
        assert relE(a, b) <= 1e-5


@pytest.mark.parametrize("kind,inner", [("warp", 3), ("poisson", 10)])
def test_fused_plain_cg_matches_oracle(api, kind, inner):
    """Without the preconditioner (M^-1 = 1, so z = r and w = q) the
    single-reduction iteration is plain CG: GN energies within 1e-4 of the
    oracle's GN with unpreconditioned CG and within rounding of the two-pass
    form.  The warp is held over 3 CG iterations, as in test_gpu_parity.py:
    its fit rows weigh 100 against stencil rows of 4 .. 8, and unpreconditioned
    CG in float32 amplifies rounding about 100-fold per iteration (both forms
    alike: 3 % apart from the float64 oracle after one GN step of 15)."""
    import torch
    prob = warp(300, 24, 0.0, seed=61, perturb=0.0, n_handles=8) if kind == "warp" else \
        synth.poisson_problem(260, 30, seed=62)
    e = oracle.make_energy(prob)
    ref = oracle.gauss_newton(e, prob.x0.reshape(-1), 2, inner, use_precond=False)
    gp = api.Problem(prob)
    rep = gp.solve_gn(2, inner, use_precond=0, pcg_form=1)
    gp.x.copy_(torch.as_tensor(prob.x0, device="cuda"))
    rep0 = gp.solve_gn(2, inner, use_precond=0, pcg_form=0)
    assert rep["pcg_done"] == ref.pcg_done
    for k, (a, b) in enumerate(zip(rep["E_history"], ref.E_history)):
        assert relE(a, b) <= TOL_ENERGY, (k, a, b)
    for a, b in zip(rep["E_history"], rep0["E_history"]):
        assert relE(a, b) <= 1e-5

