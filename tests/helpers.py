"""Shared helpers for the parity tests (GPU path vs the FP64 oracle)."""
import numpy as np

# Tolerances of FP32 iterates against the FP64 oracle:
#   state arrays: normwise relative 1e-5 after up to 100 iterations -- the
#   stated bar; FP32 rounds each stored value to 6e-8 relative, and the
#   iteration is nonexpansive, so rounding adds up over the iterations
#   without being amplified (100 iterations of a few roundings each stay
#   near 1e-6);
#   residuals: relative 1e-3 plus an absolute floor of 1e-6 times the state's
#   norm -- a residual is a difference of FP32 iterates (p - p_prev, theta -
#   theta_bar), so near convergence it cancels most of their digits and keeps
#   the FP32 rounding of the state as an absolute error.
STATE_RTOL = 1e-5
RES_RTOL = 1e-3


def hang_triangle(case, node=0):
    """The case with two device-free nodes X, Y joined to ``node`` and to each
    other (lines node-X, X-Y, Y-node, appended last): no power flows in the
    triangle at any fixed point, and outaging X-Y (line index L - 2) leaves a
    node whose only active terminal is one line."""
    n0 = case["n_nodes"]
    ext = dict(case)
    ext["n_nodes"] = n0 + 2
    ext["line_from"] = np.concatenate([case["line_from"], np.array([node, n0, n0 + 1], np.int32)])
    ext["line_to"] = np.concatenate([case["line_to"], np.array([n0, n0 + 1, node], np.int32)])
    ext["line_b"] = np.concatenate([case["line_b"], [8.0, 12.0, 10.0]])
    ext["line_u"] = np.concatenate([case["line_u"], [0.7, 0.9, 1.1]])
    return ext


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
