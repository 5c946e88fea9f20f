"""The single-reduction PCG iteration (opt_solve_params.pcg_form = 1) is a
rearrangement of the textbook Jacobi-PCG of the oracle (Saad, Alg. 9.1; the
paper's PCG of Sec. 4.1): carrying z = M^-1 r and w = M^-1 q, it takes alpha
= r.z / p.q from the r.z of the stored vectors and the next r.z, which only
sets beta, from the recurrence r.z' = r.z - 2 alpha q.z + alpha^2 q.M^-1 q.
These CPU tests restate that iteration in float64 numpy, step by step as the
GPU kernels order it (the vector update of iteration i inside iteration i + 1,
the last step after the loop), and check that it reproduces the oracle's
iterates on the normal equations of the paper's energies, and that its
breakdown rule leaves the exact step of a diagonal system alone."""
import numpy as np
import pytest

import oracle
from paper_1604_06525_gb300 import synth


def single_reduction_pcg(apply_A, b, Minv, iters):
    """The GPU form's arithmetic order in float64: returns (delta, iterations
    completed)."""
    d = np.zeros_like(b)
    z = Minv * b                 # iteration 0 starts from r_0 = b and M^-1
    p_prev = np.zeros_like(b)
    w_prev = np.zeros_like(b)
    alpha_prev, beta, n_done, active = 0.0, 0.0, 0, True
    for it in range(iters):
        if not active:
            break
        if it > 0:
            z = z - alpha_prev * w_prev          # z_i = z_{i-1} - alpha w_{i-1}
            d = d + alpha_prev * p_prev          # the pending step
        p = z + beta * p_prev
        q = apply_A(p)
        w = Minv * q
        pq, qz, qw = p @ q, q @ z, q @ w
        rz = z @ (z / Minv)                      # r = z / M^-1
        if not (pq > 0 and rz > 0):
            alpha_prev, active = 0.0, False
            break
        alpha = rz / pq
        rz_next = rz - 2 * alpha * qz + alpha * alpha * qw
        n_done += 1
        alpha_prev, p_prev, w_prev = alpha, p, w
        if not rz_next > 0:
            active = False
            break
        beta = rz_next / rz
    return d + alpha_prev * p_prev, n_done      # the last step


def normal_equations(prob):
    e = oracle.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x)
    b = -(J.T @ e.residuals(x))
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    return (lambda v: J.T @ (J @ v)), b, oracle.solver.jacobi_minv(diag)


@pytest.mark.parametrize("case", ["warp", "poisson", "mesh"])
@pytest.mark.parametrize("iters", [1, 3, 8])
def test_single_reduction_reproduces_textbook_pcg(case, iters):
    prob = {"warp": lambda: synth.warp_problem(20, 12, 4, seed=3),
            "poisson": lambda: synth.poisson_problem(24, 16, seed=4),
            "mesh": lambda: synth.mesh_problem(1, seed=5, handle_frac=0.1)}[case]()
    rng = np.random.default_rng(1)
    if case != "poisson":
        prob.x0 = (prob.x0 + rng.uniform(-0.3, 0.3, size=prob.x0.shape)).astype(np.float32)
    A, b, Minv = normal_equations(prob)
    d_ref, n_ref, _ = oracle.jacobi_pcg(A, b, Minv, iters)
    d, n = single_reduction_pcg(A, b, Minv, iters)
    assert n == n_ref == iters
    assert np.linalg.norm(d - d_ref) <= 1e-9 * np.linalg.norm(d_ref)


def test_single_reduction_stops_after_the_exact_step_of_a_diagonal_system():
    """J^T J diagonal and M^-1 its inverse: the first step is exact; the
    recurrence's next r.z is rounding-level (or not positive, which ends the
    loop with the step applied), and delta stays the exact step."""
    rng = np.random.default_rng(2)
    diag = rng.uniform(1.0, 100.0, 50)
    b = rng.standard_normal(50)
    Minv = 1.0 / diag
    for iters in (1, 2, 5):
        d, _ = single_reduction_pcg(lambda v: diag * v, b, Minv, iters)
        assert np.allclose(d, b / diag, rtol=1e-12, atol=0)


def test_recurrence_matches_the_stored_residual():
    """In exact arithmetic the recurrence equals r_{i+1}.z_{i+1}: checked on
    one PCG step of a random SPD system in float64."""
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    r = rng.standard_normal(30)
    Minv = 1.0 / np.diag(A)
    z = Minv * r
    p = z.copy()
    q = A @ p
    alpha = (r @ z) / (p @ q)
    r1 = r - alpha * q
    rz_next = r @ z - 2 * alpha * (q @ z) + alpha ** 2 * (q @ (Minv * q))
    assert abs(rz_next - r1 @ (Minv * r1)) <= 1e-12 * (r @ z)
