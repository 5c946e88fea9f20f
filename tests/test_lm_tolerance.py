"""CPU pins of the tolerances tests/lm_tolerance.py derives for the GPU parity
tests (the energy at a float32 state, and lambda_final after Nielsen's damping
update, Sec. 4 of the paper).

A derived tolerance is only as good as its derivation, so each is checked here
against something other than itself: the slope of ln f against central finite
differences of Nielsen's factor, and both bounds against the oracle's own
float32 storage emulation (oracle.solver `round_to`), which rounds exactly the
values a float32 solver stores and keeps everything else in float64.  A bound
must cover the deviation that emulation shows and must not be vacuous."""
import numpy as np
import pytest

import oracle
from oracle import solver as so
from paper_1604_06525_gb300 import synth
from lm_tolerance import U32, U64, _dlnf, energy_rounding_bound, lambda_tolerance


def nielsen_factor(rho):
    """Nielsen's damping factor for an accepted step (Madsen, Nielsen &
    Tingleff 2004, Sec. 3.2)."""
    return max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("rho", [0.02, 0.1, 0.3, 0.5, 0.7, 0.9, 0.93, 0.95, 1.2])
def test_nielsen_slope_matches_finite_differences(rho):
    """|d ln f / d rho| by central differences, on both sides of rho = 1/2
    (where it vanishes) and on the flat part beyond (2 rho - 1)^3 = 2/3."""
    h = 1e-6
    fd = abs(np.log(nielsen_factor(rho + h)) - np.log(nielsen_factor(rho - h))) / (2.0 * h)
    assert _dlnf(rho) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def near_minimum_states(prob):
    """Two GN outer iterations into the solve, then one more: the previous
    and the next state of an outer update that the energy is evaluated at."""
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    x_prev = so.gauss_newton(e, x0, 2, 10).x
    x_next = so.gauss_newton(e, x_prev, 1, 10).x
    return e, x_prev, x_next


@pytest.mark.parametrize("kind", ["warp", "mesh"])
def test_energy_rounding_bound_covers_float32_state(kind):
    """E at the state rounded to float32 (and reached by a step carrying two
    ulps of its own rounding) stays within the float32 bound; the float64
    bound of the same state lies below that deviation, so the bound scales
    with the unit roundoff and is not vacuous."""
    prob = (synth.warp_problem(40, 24, 4, seed=7) if kind == "warp"
            else synth.mesh_problem(2, seed=5, handle_frac=0.05))
    e, x_prev, x_next = near_minimum_states(prob)
    E = e.energy(x_next)
    rng = np.random.default_rng(3)
    step = (x_next - x_prev) * (1.0 + 2.0 * U32 * rng.choice([-1.0, 1.0], x_next.size))
    for x32 in (x_next.astype(np.float32), (x_prev + step).astype(np.float32)):
        dev = rel(e.energy(x32.astype(np.float64)), E)
        assert dev <= energy_rounding_bound(e, x_prev, x_next, u=U32)
        assert energy_rounding_bound(e, x_prev, x_next, u=U64) < dev


LM_CASES = [
    # (kind, size, seed, outer, inner): gain ratios from ~1 (the mesh at level
    # 3) down to 0.02-0.3 (the level-4 mesh and the warps), where the slope of
    # ln f is largest
    ("mesh", 3, 91, 6, 15),
    ("mesh", 4, 3, 12, 20),
    ("warp", (48, 32, 6), 11, 8, 10),
    ("warp", (64, 40, 8), 12, 8, 10),
]


@pytest.mark.parametrize("kind,size,seed,outer,inner", LM_CASES)
def test_lambda_tolerance_covers_float32_storage_trajectory(kind, size, seed, outer, inner):
    """The float32-storage run takes the same decisions as the float64 run,
    and its lambda_final lies within the tolerance derived from its own
    energies; that tolerance stays below 1e-4 (first order in the energy
    deviations, not a blanket allowance)."""
    prob = (synth.mesh_problem(size, seed=seed) if kind == "mesh"
            else synth.warp_problem(*size, seed=seed))
    e = oracle.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    ref = so.levenberg_marquardt(e, x0, outer, inner)
    emu = so.levenberg_marquardt(e, x0, outer, inner, round_to=np.float32)
    assert emu.outer_done == ref.outer_done and emu.accepted == ref.accepted
    tol = lambda_tolerance(ref, emu.E_history)
    assert rel(emu.lambda_final, ref.lambda_final) <= tol
    assert tol <= 1e-4
    if kind == "mesh" and size == 4:
        assert min(ref.rho) < 0.1          # the case reaches the steep part of f


def test_lambda_tolerance_vanishes_where_nothing_moves():
    """Energies equal to the oracle's give no allowance; a linear problem
    (Poisson: the model is exact, rho = 1, f on its flat part) gives none
    either, and its float32-storage run ends with the same lambda bit for
    bit: lambda0 / 3^k."""
    m = synth.mesh_problem(3, seed=91, handle_frac=0.02)
    em = oracle.make_energy(m)
    ref = so.levenberg_marquardt(em, m.x0.reshape(-1), 6, 15)
    assert lambda_tolerance(ref, ref.E_history) == pytest.approx(1e-12, abs=1e-15)
    p = synth.poisson_problem(24, 20, seed=23)
    ep = oracle.make_energy(p)
    ref = so.levenberg_marquardt(ep, p.x0.reshape(-1), 4, 20)
    emu = so.levenberg_marquardt(ep, p.x0.reshape(-1), 4, 20, round_to=np.float32)
    assert all(r == pytest.approx(1.0, abs=1e-6) for r in ref.rho + emu.rho)
    assert lambda_tolerance(ref, emu.E_history) == pytest.approx(1e-12, abs=1e-15)
    assert emu.lambda_final == ref.lambda_final == pytest.approx(1e-3 / 3 ** 4, rel=1e-12)
