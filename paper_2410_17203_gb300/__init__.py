"""GB300 proximal message passing for contingency-constrained DC OPF.

The compute path is the CUDA library ``lib/libopfmp.so`` behind the C ABI in
``include/opf.h``; :mod:`.binding` exposes the same entry points to Python.
"""
from .binding import (  # noqa: F401
    BATCH_LAYOUTS, OpfError, Solver, UnrolledCost, WarmStartNet, load_library, opf_abi_version,
    opf_batch_autotune, opf_batch_compact, opf_batch_converged, opf_batch_create,
    opf_batch_destroy, opf_batch_iterate, opf_batch_stopped, opf_create, opf_create_slice, opf_default_options,
    opf_destroy, opf_get_info, opf_get_state, opf_history, opf_iterate, opf_last_error, opf_reset,
    opf_price_noalloc, opf_residuals, opf_set_state, opf_set_state_from_nodes, opf_solution, opf_status_str, state_shapes,
    opf_slice_begin, opf_slice_exchange, opf_slice_finish, opf_slice_local, opf_slice_prime, unrolled_cost,
)
