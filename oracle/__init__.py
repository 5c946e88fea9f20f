"""FP64 CPU oracle for the Gauss-Newton / Levenberg-Marquardt PCG hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never calls it, and the
two share no code: the only common module is the seeded input generator
``paper_1604_06525_gb300.synth``, which holds no solver arithmetic.

Contents
--------
energies.py   residual vectors F(x) and explicitly assembled sparse Jacobians
              J(x) for the three energy templates of the paper
              (ARAP image warping, Fig. 24; ARAP mesh deformation, Fig. 25;
              Poisson image editing, Fig. 27), the warp written on a graph
              (Fig. 18), volumetric ARAP (Fig. 31) and embedded deformation
              (Fig. 28), in float64.
solver.py     textbook Jacobi-preconditioned CG, Gauss-Newton (Sec. 4) and
              Levenberg-Marquardt (Sec. 4, Nielsen's damping update), run step
              by step on the assembled J, in float64.

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
(finite differences, closed forms, invariants, dense solves, LM monotonicity).
Parity of the whole GN/LM trajectory against the paper itself is unpinned: the
paper prints no convergence values (its convergence plots are images).
"""
from .energies import WarpEnergy, PoissonEnergy, MeshEnergy, make_energy  # noqa: F401
from .solver import (jacobi_pcg, gauss_newton, levenberg_marquardt,  # noqa: F401
                     LMParams, jtf_diag, apply_jtj)
