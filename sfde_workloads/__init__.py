"""Seeded, synthetic inputs for the 2-D Riesz space-fractional diffusion problem.

This module is shared by the FP64 CPU oracle and by the CUDA library's tests and
benchmark.  It holds no arithmetic of the solution method (no stiffness or mass
matrices, no time stepping, no MGRIT): only problem definitions and the data a
caller hands to a solver, i.e.

* time grids (uniform, graded, piecewise uniform), Sec. 2 / Sec. 4.1;
* nodal initial values psi_0^I (defined below Eq. (2.4): u^0_i = psi_0(x_i, y_i));
* the separable load vectors F_n = sum_r w_{n,r} (f^r_y, phi_j)(f^r_x, phi_i)
  (defined below Eq. (2.4): f^n_j = int_{I_n} (f, phi_j) dt) for the manufactured solution of
  Example 4.1 and for the Gaussian-bump source, and dense (non-separable) load vectors of a moving
  bump;
* load vectors of the manufactured solution against the P1-triangle hats of Sec. 2;
* the benchmark workloads (sizes, orders, diffusivities, seeds).

Every random draw comes from ``numpy.random.default_rng(seed)`` on the host and
is passed to both solvers as data.
"""
from .generate import (  # noqa: F401
    Workload, workload, WORKLOADS, time_grid, sine_mode_amplitudes, sine_mode_nodal,
    manufactured_initial, manufactured_forcing, manufactured_exact, gaussian_bump_forcing,
    interior_nodes, Forcing, DenseForcing, moving_bump_dense_forcing, LowRankDenseForcing,
    p1_manufactured_forcing,
)
