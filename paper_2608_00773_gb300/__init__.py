"""GB300-native Q4C real-space integration (arxiv 2608.00773, Section III A).

The compute path lives in libq4c.so (CUDA for sm_103a, C ABI in
include/q4c.h); this package only marshals arguments to it.
"""
from .binding import (  # noqa: F401
    EXPORTS, Q4CError, Tables, Grid, nao_tabulate, nao_tabulate_knots, grid_partition, q4c_integrate, q4c_density, q4c_density_full, q4c_kfold, q4c_spinor_basis, q4c_spinor_transform,
    q4c_spinor_density_matrices, q4c_tables_set_columns, q4c_integrate_columns, q4c_tables_set_kappa,
    q4c_spinor_nnz,
    q4c_integrate_backward, q4c_scf_pass, q4c_autotune, q4c_grid_tiling, q4c_grid_set_tiling,
    q4c_basis_eval, q4c_set_wait_limit_ns, integrate, profile, profile_read, load, LIB_PATH, Q4C_FP64, Q4C_SPLIT,
)
from .setup_workload import setup  # noqa: F401
