"""Tolerances derived from the arithmetic for two LM quantities that float32
cannot pin at the stated 1e-4 (helpers of the GPU parity tests).

energy_rounding_bound: an energy evaluated at a state the GPU holds in
    float32.  The unknowns x_k = x_{k-1} + delta are rounded to float32 (half
    an ulp, u |x_k|) and delta carries the rounding of the PCG recurrences
    (a few ulps of |delta|).  To first order the energy moves by
    grad E . dx = 2 (J^T F) . dx, so
        |dE| / E <= 2 sum_i |(J^T F)_i| c u (|x_i| + |delta_i|) / E,   c = 4.
    Near a minimum E is small while |x| is not (the residual cancels), so the
    bound can exceed 1e-4 although every operation is correctly rounded.

lambda_tolerance: the LM damping after Nielsen's update (Madsen, Nielsen &
    Tingleff 2004, Sec. 3.2; Sec. 4 of the paper) is lambda_0 times a product
    of factors f(rho_k) = max(1/3, 1 - (2 rho_k - 1)^3) for accepted steps and
    of exact powers of 2 for rejected ones.  The gain ratio rho_k =
    (E_k - E'_k) / pred_k divides a difference of nearby energies, so an error
    e_k in that difference moves rho_k by about e_k (1 + |rho_k|) / pred_k
    (the predicted decrease is taken to carry an error of the same size), and
    ln lambda_final by sum_k |d ln f / d rho| * that.  e_k is measured: the
    difference between the GPU's and the oracle's energy decrease of step k.
"""
import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def energy_rounding_bound(energy, x_prev, x_next, u=U32, c=4.0):
    """First-order bound on the relative error of E(x_next) when x_next is
    held in a precision of unit roundoff u (module docstring)."""
    import oracle
    x_prev = np.asarray(x_prev, np.float64).reshape(-1)
    x_next = np.asarray(x_next, np.float64).reshape(-1)
    g, _, E = oracle.jtf_diag(energy, x_next)
    if E == 0.0:
        return 0.0
    dx = c * u * (np.abs(x_next) + np.abs(x_next - x_prev))
    return float(2.0 * np.sum(np.abs(g) * dx) / E)


def _dlnf(rho):
    """|d ln f / d rho| for f(rho) = max(1/3, 1 - (2 rho - 1)^3)."""
    t = 2.0 * rho - 1.0
    f = 1.0 - t ** 3
    return 0.0 if f <= 1.0 / 3.0 else 6.0 * t * t / f


def lambda_tolerance(ref, E_gpu, safety=2.0):
    """Relative tolerance of lambda_final for an LM solve whose oracle run is
    `ref` (oracle.LMResult) and whose GPU energies per outer iteration are
    E_gpu (module docstring)."""
    tot = 0.0
    for k, acc in enumerate(ref.accepted):
        if not acc:
            continue
        e_k = abs((E_gpu[k] - E_gpu[k + 1]) - (ref.E_history[k] - ref.E_history[k + 1]))
        rho, pred = ref.rho[k], ref.pred[k]
        drho = safety * e_k * (1.0 + abs(rho)) / pred
        # largest slope of ln f over [rho - drho, rho + drho]
        grid = np.linspace(rho - drho, rho + drho, 65)
        slope = max(_dlnf(r) for r in grid)
        tot += slope * drho
    return float(np.expm1(tot)) + 1e-12


def oracle_mesh_lm(level, seed, outer, inner, round_to=None):
    """The oracle's LM on a seeded icosphere mesh problem, as a plain dict
    (a spawned worker's job in the GPU tests).  round_to: None or "float32"
    (oracle.solver's reduced-precision storage emulation)."""
    import oracle
    from paper_1604_06525_gb300 import synth
    prob = synth.mesh_problem(level, seed=seed)
    e = oracle.make_energy(prob)
    r = oracle.levenberg_marquardt(e, prob.x0.reshape(-1), outer, inner,
                                   round_to=None if round_to is None else np.dtype(round_to))
    return {"E_history": list(r.E_history), "accepted": list(r.accepted), "outer_done": r.outer_done,
            "pcg_done": r.pcg_done, "lambda_final": r.lambda_final, "E_trial": list(r.E_trial),
            "pred": list(r.pred), "rho": list(r.rho)}
