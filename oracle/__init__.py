"""FP64 CPU oracle of the LOSS method (Guo, Li, Xiong, "Distributed local spline simulator for wave
propagation", arXiv 2301.05127).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2301_05127_gb300``) and neither imports the other; both receive their inputs from ``synth``.

The oracle is plain and slow on purpose: every 1-D derivative assembles the paper's local system and
solves it with a generic pivoted banded solver (LAPACK ``gbsv`` through ``scipy.linalg.solve_banded``), the
boundary closure weights come from explicit rows of the inverse of the global collocation matrix, and the
time integrator is the literal Strang sequence "half A, full B, half A".  Everything is float64.

Modules
-------
spline   1-D cubic-B-spline collocation, PMBC weights and closures, local solves, derivatives (Sec. 3.1-3.2)
wave     acoustic and elastic velocity-stress steppers, Ricker source, receivers, energy (Sec. 2, 3.3, 4)
adjoint  discrete adjoint of the stepper and the misfit gradient with respect to vp, vs, rho
exact    closed-form solutions of the Gaussian-pulse experiment (Sec. 4.1), in continuous time and for the
         Strang-split time stepping with exact spatial derivatives
"""
from . import adjoint, exact, spline, wave  # noqa: F401
