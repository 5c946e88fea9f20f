"""Serving engine: continuous batching of LM solves under an HBM budget.  Each
request's result must equal its one-at-a-time solve (opt_solve_lm with the
same parameters) within the stated tolerances, whatever else is in the mix."""
import numpy as np
import pytest

from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu

OUTER, INNER, REL_TOL = 10, 10, 1e-3


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1604_06525_gb300 import build, api as api_mod
    build.build()
    api_mod.load_library()
    return api_mod


def relE(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def requests():
    rs = [synth.warp_problem(int(s), int(s), synth.warp_handle_count(int(s), int(s)), seed=400 + i)
          for i, s in enumerate(synth.batch_sides(6, 24, 96, seed=11))]
    rs += [synth.mesh_problem(1, seed=410, handle_frac=0.1), synth.mesh_problem(2, seed=411, handle_frac=0.05)]
    rs += [synth.poisson_problem(40, 30, seed=420), synth.poisson_problem(33, 51, seed=421)]
    return rs


def solo(api, prob):
    g = api.Problem(prob)
    r = g.solve_lm(OUTER, INNER, rel_tol=REL_TOL)
    x = g.x.cpu().numpy().copy()
    g.close()
    return r, x


def check_same(prob, rep, x, ref, xref):
    assert rep["status"] == "OPT_OK"
    assert rep["outer_done"] == ref["outer_done"]
    assert rep["accepted"] == ref["accepted"]
    assert rep["converged"] == ref["converged"]
    tol = 1e-5 if prob.kind == "mesh" else 1e-6
    for a, b in zip(rep["E_history"][:-1], ref["E_history"][:-1]):
        assert relE(a, b) <= tol
    assert relE(rep["E_final"], ref["E_final"]) <= 1e-5
    xs = x.cpu().numpy().reshape(-1)
    d = np.linalg.norm(xs - xref.reshape(-1)) / max(np.linalg.norm(xref), 1e-30)
    assert d <= (1e-4 if prob.kind == "mesh" else 1e-6)


@pytest.mark.parametrize("max_rounds", [1, 16])
def test_serve_alone_equals_mix(api, max_rounds):
    """Requests joining while others run equal their solo solves, with one
    LM outer iteration per step and with up to 16 per step when nothing
    waits (the energy history then comes from the per-round records)."""
    probs = requests()
    refs = [solo(api, p) for p in probs]
    srv = api.Server(4 << 30, outer=OUTER, inner=INNER, rel_tol=REL_TOL, max_rounds=max_rounds)
    tickets = [srv.submit(p) for p in probs[:5]]
    srv.step()
    srv.step()
    tickets += [srv.submit(p) for p in probs[5:]]     # join while others are mid-solve
    done = {}
    for _ in range(200):
        active, queued = srv.step()
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        if len(done) == len(tickets):
            break
    assert len(done) == len(tickets)
    for p, t, (ref, xref) in zip(probs, tickets, refs):
        rep, x = done[t]
        check_same(p, rep, x, ref, xref)
    srv.close()


def server_estimate_warp(W, H, n_handles):
    """The server's footprint estimate of a planned warp (24 pitched planes,
    tiles, handles, fixed overhead)."""
    P = (W + 31) // 32 * 32
    tiles = ((W + 31) // 32) * ((H + 7) // 8)
    return 24 * P * H * 4 + tiles * 64 + n_handles * 16 + (1 << 16)


def test_serve_budget_limits_admission(api):
    probs = [synth.warp_problem(64, 48, 8, seed=500 + i) for i in range(6)]
    refs = [solo(api, p) for p in probs]
    est = server_estimate_warp(64, 48, 8)
    srv = api.Server(2 * est + 100, outer=OUTER, inner=INNER, rel_tol=REL_TOL)   # room for exactly two
    tickets = [srv.submit(p) for p in probs]
    done, max_active = {}, 0
    for _ in range(400):
        active, queued = srv.step()
        max_active = max(max_active, active)
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        if len(done) == len(tickets):
            break
    assert len(done) == len(tickets)
    assert max_active == 2
    for p, t, (ref, xref) in zip(probs, tickets, refs):
        rep, x = done[t]
        check_same(p, rep, x, ref, xref)
    srv.close()


def test_serve_max_active_caps_admission_in_arrival_order(api):
    """max_active = 3 under an ample budget: never more than three requests
    admitted, admission in arrival order (the requests admitted so far, done
    or active, are always the first ones submitted), every result equal to
    its solo solve."""
    probs = requests()
    refs = [solo(api, p) for p in probs]
    srv = api.Server(4 << 30, outer=OUTER, inner=INNER, rel_tol=REL_TOL, max_active=3)
    tickets = [srv.submit(p) for p in probs]
    done, max_active = {}, 0
    for _ in range(400):
        active, queued = srv.step()
        max_active = max(max_active, active)
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        admitted = len(tickets) - queued
        assert len(done) + active == admitted
        assert all(tickets.index(t) < admitted for t in done)
        if len(done) == len(tickets):
            break
    assert len(done) == len(tickets)
    assert max_active == 3
    for p, t, (ref, xref) in zip(probs, tickets, refs):
        rep, x = done[t]
        check_same(p, rep, x, ref, xref)
    with pytest.raises(api.OptError) as ei:
        srv.set_max_active(-1)
    assert ei.value.status == 1
    for bad in (0, 65):
        with pytest.raises(api.OptError) as ei:
            srv.set_max_rounds(bad)
        assert ei.value.status == 1
    srv.close()


def test_serve_rejects_oversize_and_reports_planning_errors(api):
    srv = api.Server(1 << 20, outer=OUTER, inner=INNER)
    with pytest.raises(api.OptError) as ei:
        srv.submit(synth.warp_problem(512, 512, 8, seed=1))
    assert ei.value.status == 6
    srv.close()
    srv = api.Server(1 << 30, outer=OUTER, inner=INNER)
    bad = synth.warp_problem(16, 16, 2, seed=2)
    bad.handle_idx = np.array([5, 5], np.int32)           # duplicate handle: planning fails
    t = srv.submit(bad)
    srv.step()
    with pytest.raises(api.OptError) as ei:
        srv.poll(t)
    assert ei.value.status == 1
    srv.close()


def test_serve_failed_rebuild_ends_active_requests_and_keeps_serving(api):
    """A batch rebuild that fails (an out-of-memory made on the host through
    the server's test hook, no device fault) ends every request active at
    that moment with the error; their budget is returned, and requests queued
    afterwards are served normally, equal to their solo solves."""
    probs = requests()
    srv = api.Server(4 << 30, outer=OUTER, inner=INNER, rel_tol=REL_TOL)
    first = [srv.submit(p) for p in probs[:3]]
    srv.step()                                        # admitted, one outer iteration done
    srv.inject_rebuild_failure(2)                     # OPT_ERR_OOM at the next rebuild
    late = srv.submit(probs[3])                       # its admission forces the rebuild
    st, active, queued = srv.step_status()
    assert st == 2 and active == 0 and queued == 0
    for t in first + [late]:
        with pytest.raises(api.OptError) as ei:
            srv.poll(t)
        assert ei.value.status == 2
    # the server goes on with new requests
    refs = [solo(api, p) for p in probs[4:7]]
    tickets = [srv.submit(p) for p in probs[4:7]]
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
    for p, t, (ref, xref) in zip(probs[4:7], tickets, refs):
        rep, x = done[t]
        check_same(p, rep, x, ref, xref)
    with pytest.raises(api.OptError):
        srv.inject_rebuild_failure(0)
    srv.close()


def test_problem_from_template_equals_plain_problem(api):
    """Planning from a device-resident template (the input path both serving
    arms take) gives the same solve as planning from host arrays."""
    for prob in (synth.warp_problem(70, 50, 6, seed=430), synth.mesh_problem(2, seed=431, handle_frac=0.05)):
        tpl = api.make_descriptor(prob, "cuda") + (prob.kind,)
        a = api.Problem(prob)
        b = api.Problem.from_template(tpl)
        ra = a.solve_lm(OUTER, INNER, rel_tol=REL_TOL)
        rb = b.solve_lm(OUTER, INNER, rel_tol=REL_TOL)
        assert ra["E_history"] == rb["E_history"] and ra["outer_done"] == rb["outer_done"]
        assert np.array_equal(a.x.cpu().numpy(), b.x.cpu().numpy())
        # the template's own unknowns are untouched
        assert np.array_equal(tpl[1].cpu().numpy().reshape(-1), prob.x0.reshape(-1).astype(np.float32))
        a.close()
        b.close()
