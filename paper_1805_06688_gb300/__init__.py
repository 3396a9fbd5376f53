"""GB300 (sm_103a) MGRIT solver for the 2-D Riesz space-fractional diffusion equation.

A thin ctypes binding of the C ABI declared in ``include/sfde.h``: every function here only
marshals arguments (NumPy arrays or torch tensors, host or device) into the library, whose
CUDA kernels do all the work.  There is no fallback: if ``libsfde.so`` has not been built,
importing the binding works but the first call raises ``RuntimeError``.
"""
from ._binding import (  # noqa: F401
    SFDE_OK, SFDE_EINVAL, SFDE_ENOMEM, SFDE_ECUDA, SFDE_ENOCONV, SFDE_ETIMEOUT, SFDE_EUNSUPPORTED,
    SFDE_ESCRATCH, NOALLOC_SCRATCH_DOUBLES, sfde_step_batch_noalloc,
    PREC_FP64, PREC_MIXED_BF16, PREC_MIXED_TF32, PREC_MIXED_FP32, PREC_MIXED_AUTO, RELAX_FCF, RELAX_F, COARSE_CN, COARSE_BE,
    COARSE_AUTO, OP_TENSOR, OP_P1, SfdeError, MgritOpts, MgritStats, SfdeOpts, lib, library_path, exported_symbols,
    sfde_setup, sfde_set_initial, sfde_set_forcing, mgrit_solve, seq_timestep, sfde_step_batch,
    sfde_get_operator, sfde_profile_enable, sfde_profile_read, SfdeProfile, sfde_destroy,
    sfde_strerror, make_opts, Problem, sfde_batch_solve, batch_solve, SfdeTuning, sfde_set_tuning,
    sfde_autotune, sfde_get_tuning, STOP_NATIVE, STOP_SFORM, sfde_set_forcing_dense, sfde_propagate_batch,
)
