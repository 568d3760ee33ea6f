"""FP64 CPU oracle for proximal message passing (test infrastructure only).

This package is the plain, slow reference that the CUDA path is checked
against.  It is test infrastructure: only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product library never
does.  It shares no code with the CUDA path.

Parity status of each function is recorded in its docstring; every function
here is pinned by ``-m "not gpu"`` tests against closed forms, brute force,
analytic small grids or identities that the paper states.
"""
from .mp import (  # noqa: F401
    Oracle, OracleOptions, Network, Shard,
    prox_gen, prox_line, prox_fixed_load, prox_hvdc,
    ramp_rows, storage_rows, inner_admm, inner_matrix,
    node_mean, average, residual,
)
