"""Shared helpers for the parity tests (GPU path vs the FP64 oracle)."""
import numpy as np

# Tolerances (derived in the design notes from FP32 iterates vs FP64):
#   state arrays: normwise relative 1e-5 after up to 100 iterations;
#   residuals: relative 1e-3 (differences of FP32 iterates) plus an absolute
#   floor tied to the FP32 rounding of the state.
STATE_RTOL = 1e-5
RES_RTOL = 1e-3


def oracle_arrays(o):
    L = o.net.L
    return dict(p_line=o.line_p(), th1=o.th[:, :L], th2=o.th[:, L:], v1=o.v[:, :L],
                v2=o.v[:, L:], p_dev=o.dev_p(), u=o.u)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def compare_states(gpu_state, o, rtol=STATE_RTOL, keys=None):
    ref = oracle_arrays(o)
    errs = {}
    for k, r in ref.items():
        if keys and k not in keys:
            continue
        g = gpu_state[k]
        assert g.shape == r.shape, (k, g.shape, r.shape)
        errs[k] = rel_err(g, r)
    bad = {k: e for k, e in errs.items() if not e <= rtol}
    assert not bad, f"normwise relative error above {rtol}: {bad} (all: {errs})"
    return errs


def compare_residuals(res_gpu, res_ora, state_scale, rtol=RES_RTOL):
    # absolute floor: FP32 rounding of iterates of size state_scale over the vector
    floor = 1e-6 * state_scale
    for j in range(6):
        assert abs(res_gpu[j] - res_ora[j]) <= rtol * abs(res_ora[j]) + floor, (
            j, res_gpu, res_ora)
