"""FP64 CPU oracle for the MGRIT solver of the 2-D Riesz space-fractional diffusion equation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The CUDA library never imports, links or executes anything here, and this package
never imports the CUDA library: the two share only the seeded inputs of
``sfde_workloads``.

Contents (all plain NumPy/SciPy in float64, written from the paper):

* ``sfde``      -- 1-D Riesz stiffness/mass matrices (Sec. 2), the fully discrete
                   Crank-Nicolson-type step (Eq. (2.6)), sequential time stepping;
* ``mgrit``     -- Algorithm 1 (multilevel V-cycle, FCF relaxation, injection,
                   C-point correction), in nodal and in modal coordinates;
* ``analysis``  -- Lemma 3.1's two-level C-point error propagator, the
                   eigenvalue relations (Eq. (3.6)) and Theorem 3.1's bound;
* ``p1``        -- the paper's block-Toeplitz P1-triangle matrices (Sec. 2).

Parity status per function is recorded in each module's header.
"""
from . import sfde, mgrit, analysis  # noqa: F401
