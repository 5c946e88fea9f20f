"""Textbook Jacobi-PCG, Gauss-Newton and Levenberg-Marquardt in float64
(test infrastructure; see the package docstring).

Gauss-Newton (Sec. 4): linearize F(x+d) ~ F(x) + J d and solve the normal
equations 2 J^T J d = -2 J^T F; the factors 2 cancel, so the inner system is
J^T J d = b with b = -J^T F.  Then x <- x + d, repeated K times.

Levenberg-Marquardt (Sec. 4): the same with J^T J + lambda * D, D the clamped
diagonal of J^T J; lambda is the inverse trust-region radius.  The paper says
its strategy is adapted from Ceres and names initial / min / max radius and
min / max diagonal clamps without values; the damping update used here is the
published one of Madsen, Nielsen & Tingleff (Methods for Non-Linear Least
Squares Problems, 2004, Sec. 3.2): gain ratio rho = (E - E') / (E - L(d)),
accept if rho > eta, lambda *= max(1/3, 1 - (2 rho - 1)^3) and nu = 2 on
acceptance, lambda *= nu and nu *= 2 on rejection.

PCG (Sec. 4.1; the algorithm box of Fig. 6 is an image): textbook
Hestenes-Stiefel CG with the Jacobi preconditioner M = diag(J^T J) (+ the LM
damping), starting from d0 = 0, for exactly `iters` iterations (Saad,
Iterative Methods for Sparse Linear Systems, Alg. 9.1).  It stops early only
on breakdown: r.z == 0 (the residual vanished) or p.q <= 0.  Rows whose
diagonal is zero get M^-1 = 1 (their right-hand side is zero, so this only
avoids a division by zero).

round_to (jacobi_pcg, gauss_newton, levenberg_marquardt): None for plain
float64.  A numpy dtype (np.float32) makes the runs store what a reduced-
precision solver stores in that precision -- the unknowns x (after every
update and at the LM trial point), the PCG vectors d, r, z, p, the product
q = A p and the scalars alpha, beta -- while every product, dot product and
energy is still formed in float64.  It measures how far a trajectory carries
the rounding of that storage (some LM trajectories amplify a 1e-8 rounding to
1e-4 within a few outer iterations); it is not a model of any kernel.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def jtf_diag(energy, x):
    """(J^T F, diag(J^T J), E) at x (Sec. 4.2 evalJTF + preconditioner rows;
    evalF).  Note the library's r0 is b = -J^T F."""
    F = energy.residuals(x)
    J = energy.jacobian(x)
    return J.T @ F, np.asarray(J.multiply(J).sum(axis=0)).ravel(), float(F @ F)


def apply_jtj(energy, x, p, lam: float = 0.0, Dc=None):
    """q = (J^T J + lam * diag(Dc)) p at x (Sec. 4.2 applyJTJ, without the
    factor 2 that cancels against the right-hand side)."""
    J = energy.jacobian(x)
    q = J.T @ (J @ np.asarray(p, np.float64))
    if lam != 0.0:
        q = q + lam * Dc * p
    return q


def jacobi_minv(diag):
    """Inverse Jacobi preconditioner with the zero-diagonal rule."""
    out = np.ones_like(diag)
    nz = diag != 0
    out[nz] = 1.0 / diag[nz]
    return out


def _rounder(round_to):
    if round_to is None:
        return lambda v: v
    return lambda v: np.asarray(v, round_to).astype(np.float64)


def jacobi_pcg(apply_A, b, Minv, iters: int, round_to=None):
    """Textbook Jacobi-PCG for A d = b from d0 = 0.

    Returns (d, n_done, r) where n_done counts completed iterations and r is
    the recurrence residual.  round_to: see the module docstring."""
    rd = _rounder(round_to)
    d = np.zeros_like(b)
    r = rd(b.copy())
    z = rd(Minv * r)
    p = z.copy()
    rho = float(r @ z)
    n_done = 0
    for _ in range(iters):
        if rho == 0.0:
            break
        q = rd(apply_A(p))
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = float(rd(rho / pq))
        d = rd(d + alpha * p)
        r = rd(r - alpha * q)
        z = rd(Minv * r)
        rho_new = float(r @ z)
        beta = float(rd(rho_new / rho))
        p = rd(z + beta * p)
        rho = rho_new
        n_done += 1
    return d, n_done, r


@dataclass
class GNResult:
    x: np.ndarray
    E_history: list          # E(x_k) for k = 0..outer
    pcg_done: int


def gauss_newton(energy, x0, outer: int, inner: int, use_precond: bool = True, round_to=None) -> GNResult:
    """Gauss-Newton with a fixed number of outer and PCG iterations
    (round_to: see the module docstring)."""
    rd = _rounder(round_to)
    x = rd(np.asarray(x0, np.float64).reshape(-1).copy())
    hist = []
    total = 0
    for _ in range(outer):
        F = energy.residuals(x)
        J = energy.jacobian(x)
        hist.append(float(F @ F))
        b = -(J.T @ F)
        diag = np.asarray(J.multiply(J).sum(axis=0)).ravel()
        Minv = jacobi_minv(diag) if use_precond else np.ones_like(diag)
        d, n_done, _ = jacobi_pcg(lambda p: J.T @ (J @ p), b, Minv, inner, round_to)
        total += n_done
        x = rd(x + d)
    hist.append(energy.energy(x))
    return GNResult(x, hist, total)


@dataclass
class LMParams:
    lambda0: float = 1e-3
    lambda_min: float = 1e-16
    lambda_max: float = 1e32
    diag_min: float = 1e-6
    diag_max: float = 1e32
    eta: float = 1e-3
    rel_tol: float = 0.0          # > 0: stop after an accepted step with |dE|/E < rel_tol


@dataclass
class LMResult:
    x: np.ndarray
    E_history: list              # E(x_k) at the start of each outer iteration, then final
    accepted: list               # per outer iteration
    lambdas: list                # lambda used by each outer iteration
    outer_done: int
    pcg_done: int
    lambda_final: float = 0.0    # damping after the last update
    E_trial: list = None         # per outer iteration: E(x + d)
    pred: list = None            # per outer iteration: predicted decrease E - |F + J d|^2
    rho: list = None             # per outer iteration: gain ratio


def levenberg_marquardt(energy, x0, outer: int, inner: int, prm: LMParams = LMParams(),
                        use_precond: bool = True, round_to=None) -> LMResult:
    """Levenberg-Marquardt with Nielsen's damping update (module docstring).

    A rejected step counts as an outer iteration.  With prm.rel_tol > 0 the
    loop stops after an accepted step whose relative energy change is below
    rel_tol (or whose new energy is exactly zero).  round_to: see the module
    docstring."""
    rd = _rounder(round_to)
    x = rd(np.asarray(x0, np.float64).reshape(-1).copy())
    lam, nu = prm.lambda0, 2.0
    hist, acc, lams = [], [], []
    trials, preds, rhos = [], [], []
    total = 0
    k = 0
    while k < outer:
        F = energy.residuals(x)
        J = energy.jacobian(x)
        E = float(F @ F)
        hist.append(E)
        lams.append(lam)
        b = -(J.T @ F)
        diag = np.asarray(J.multiply(J).sum(axis=0)).ravel()
        Dc = np.clip(diag, prm.diag_min, prm.diag_max)
        Minv = jacobi_minv(diag + lam * Dc) if use_precond else np.ones_like(diag)
        d, n_done, _ = jacobi_pcg(lambda p: J.T @ (J @ p) + lam * Dc * p, b, Minv, inner, round_to)
        total += n_done
        x_trial = rd(x + d)
        if round_to is not None:
            d = x_trial - x                     # the step the rounded state actually takes
        E_new = energy.energy(x_trial)
        Fl = F + J @ d                          # linear model of the residuals
        pred = E - float(Fl @ Fl)
        rho = (E - E_new) / pred if pred > 0.0 else -np.inf
        trials.append(E_new)
        preds.append(pred)
        rhos.append(rho)
        k += 1
        if rho > prm.eta:
            x = x_trial
            lam = lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
            nu = 2.0
            acc.append(True)
            lam = min(max(lam, prm.lambda_min), prm.lambda_max)
            if prm.rel_tol > 0.0 and (E_new == 0.0 or abs(E - E_new) / E < prm.rel_tol):
                break
        else:
            lam = lam * nu
            nu = 2.0 * nu
            acc.append(False)
            lam = min(max(lam, prm.lambda_min), prm.lambda_max)
    hist.append(energy.energy(x))
    return LMResult(x, hist, acc, lams, k, total, lam, trials, preds, rhos)
