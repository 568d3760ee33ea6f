"""ctypes binding of the C ABI in ``include/opf.h`` (argument marshalling only).

Every function keeps the C name.  Errors raise :class:`OpfError` carrying the
``opf_status`` code.  Host arrays are NumPy; device buffers are anything with a
``data_ptr()`` (PyTorch tensors) and are passed with ``on_device=True``.
There is no fallback: if the CUDA library is not built, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libopfmp.so")

OPF_OK, OPF_EINVAL, OPF_ENOMEM, OPF_ECUDA, OPF_ETIMEOUT, OPF_ENONFINITE, OPF_ESTATE, OPF_ESTALLED = range(8)
OPF_HISTORY_COLS = 10  # doubles per residual-history row (opf_history)
# capacity of the fixed device array behind opf_price_noalloc (N * T floats)
OPF_PRICE_SCRATCH_FLOATS = 1 << 20
OPF_WSNET_OUT = 2      # outputs per row of the warm-start network (price, angle)

F32P = C.POINTER(C.c_float)
F64P = C.POINTER(C.c_double)
I32P = C.POINTER(C.c_int32)


class OpfError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = int(status)
        super().__init__(f"{where}: {_status_str(status)} ({status}) {msg}".rstrip())


class opf_network(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int32),
        ("n_lines", C.c_int32), ("line_from", I32P), ("line_to", I32P),
        ("line_b", F64P), ("line_u", F64P),
        ("n_gens", C.c_int32), ("gen_node", I32P), ("gen_a", F64P), ("gen_b", F64P),
        ("gen_pmin", F64P), ("gen_pmax", F64P), ("gen_ramp", F64P),
        ("n_loads", C.c_int32), ("load_node", I32P), ("load_p", F64P), ("load_voll", F64P),
        ("n_stor", C.c_int32), ("stor_node", I32P), ("stor_P", F64P), ("stor_dur", F64P),
        ("stor_eff", F64P), ("stor_cost", F64P),
        ("n_hvdc", C.c_int32), ("hvdc_from", I32P), ("hvdc_to", I32P), ("hvdc_u", F64P),
    ]


class opf_contingencies(C.Structure):
    _fields_ = [("K", C.c_int32), ("outaged_line", I32P)]


class opf_options(C.Structure):
    _fields_ = [
        ("rho_p", C.c_double), ("rho_theta", C.c_double), ("eps", C.c_double),
        ("mu", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
        ("adapt_every", C.c_int32), ("inner_iters", C.c_int32), ("check_every", C.c_int32),
        ("stall_window", C.c_int32),
        ("sync_timeout_ms", C.c_int64),
        ("cuda_stream", C.c_void_p),
        ("adapt_until", C.c_int64), ("history_len", C.c_int32), ("reserved0", C.c_int32),
    ]


class opf_state(C.Structure):
    _fields_ = [("p_line", C.c_void_p), ("th1", C.c_void_p), ("th2", C.c_void_p),
                ("v1", C.c_void_p), ("v2", C.c_void_p), ("p_dev", C.c_void_p),
                ("u", C.c_void_p), ("inner", C.c_void_p)]


class opf_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int64), ("converged", C.c_int32), ("status", C.c_int32),
        ("rho_p", C.c_double), ("rho_theta", C.c_double), ("tolerance", C.c_double),
        ("N", C.c_int32), ("L", C.c_int32), ("S", C.c_int32), ("T", C.c_int32),
        ("K", C.c_int32), ("J", C.c_int32), ("n_ramp", C.c_int32), ("n_stor", C.c_int32),
        ("inner_len", C.c_int64), ("device_bytes", C.c_int64),
        ("kernels_per_iteration", C.c_int32), ("stalled", C.c_int32),
        ("frozen_at", C.c_int64), ("history_rows", C.c_int64),
        ("k_begin", C.c_int32), ("k_count", C.c_int32),
    ]


ABI_VERSION = 5     # OPF_ABI_VERSION of include/opf.h

EXPORTS = ["opf_default_options", "opf_create", "opf_create_slice", "opf_slice_exchange", "opf_slice_prime",
           "opf_slice_begin", "opf_slice_local", "opf_slice_finish", "opf_iterate", "opf_residuals", "opf_solution",
           "opf_price_noalloc", "opf_history", "opf_set_state_from_nodes", "opf_get_state", "opf_set_state", "opf_reset", "opf_get_info",
           "opf_destroy", "opf_status_str", "opf_last_error", "opf_abi_version",
           "opf_batch_create", "opf_batch_iterate", "opf_batch_converged", "opf_batch_stopped",
           "opf_batch_destroy",
           "opf_batch_autotune", "opf_batch_compact",
           "opf_wsnet_param_count", "opf_wsnet_create", "opf_wsnet_get_params", "opf_wsnet_set_params",
           "opf_wsnet_forward", "opf_wsnet_gradient", "opf_wsnet_train_step", "opf_wsnet_destroy",
           "opf_diff_create", "opf_diff_cost_grad", "opf_diff_cost_grad_on", "opf_diff_set_record_limit",
           "opf_diff_destroy"]

_lib = None


def load_library(path=None):
    """Load the CUDA library (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"CUDA library not built: {p} (run __graft_entry__.build())")
    lib = C.CDLL(p)
    lib.opf_abi_version.restype = C.c_int32
    if lib.opf_abi_version() != ABI_VERSION:
        raise OSError(f"{p} has ABI version {lib.opf_abi_version()}, this binding expects {ABI_VERSION} "
                      "(rebuild the library)")
    lib.opf_default_options.argtypes = [C.POINTER(opf_options)]
    lib.opf_default_options.restype = None
    lib.opf_create.argtypes = [C.POINTER(opf_network), C.c_int32, C.POINTER(opf_contingencies),
                               C.POINTER(opf_options), C.POINTER(C.c_void_p)]
    lib.opf_iterate.argtypes = [C.c_void_p, C.c_int32, C.c_double]
    lib.opf_create_slice.argtypes = [C.POINTER(opf_network), C.c_int32, C.POINTER(opf_contingencies), C.c_int32,
                                     C.c_int32, C.POINTER(opf_options), C.POINTER(C.c_void_p)]
    lib.opf_slice_exchange.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]
    lib.opf_slice_prime.argtypes = [C.c_void_p]
    lib.opf_slice_begin.argtypes = [C.c_void_p, C.c_int32, C.c_double]
    lib.opf_slice_local.argtypes = [C.c_void_p]
    lib.opf_slice_finish.argtypes = [C.c_void_p]
    lib.opf_residuals.argtypes = [C.c_void_p, F64P]
    lib.opf_solution.argtypes = [C.c_void_p, C.c_int32, F64P, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    lib.opf_price_noalloc.argtypes = [C.c_void_p, C.c_void_p]
    lib.opf_history.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]
    lib.opf_set_state_from_nodes.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_double]
    lib.opf_get_state.argtypes = [C.c_void_p, C.c_int32, C.POINTER(opf_state)]
    lib.opf_set_state.argtypes = [C.c_void_p, C.c_int32, C.POINTER(opf_state)]
    lib.opf_reset.argtypes = [C.c_void_p]
    lib.opf_get_info.argtypes = [C.c_void_p, C.POINTER(opf_info)]
    lib.opf_destroy.argtypes = [C.c_void_p]
    lib.opf_destroy.restype = None
    lib.opf_status_str.argtypes = [C.c_int]
    lib.opf_status_str.restype = C.c_char_p
    lib.opf_last_error.argtypes = []
    lib.opf_last_error.restype = C.c_char_p
    lib.opf_abi_version.argtypes = []
    lib.opf_abi_version.restype = C.c_int32
    lib.opf_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]
    lib.opf_batch_iterate.argtypes = [C.c_void_p, C.c_int32]
    lib.opf_batch_converged.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    lib.opf_batch_stopped.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32)]
    lib.opf_batch_destroy.argtypes = [C.c_void_p]
    lib.opf_batch_destroy.restype = None
    lib.opf_batch_autotune.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), F64P]
    lib.opf_batch_compact.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    for name in ("opf_batch_create", "opf_batch_iterate", "opf_batch_converged", "opf_batch_stopped",
                 "opf_batch_autotune", "opf_batch_compact"):
        getattr(lib, name).restype = C.c_int
    lib.opf_wsnet_param_count.argtypes = [C.c_int32]
    lib.opf_wsnet_param_count.restype = C.c_int64
    lib.opf_wsnet_create.argtypes = [C.c_int32, C.c_int32, I32P, I32P, F64P, C.c_int32, C.c_int32,
                                     C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.opf_wsnet_get_params.argtypes = [C.c_void_p, C.c_void_p]
    lib.opf_wsnet_set_params.argtypes = [C.c_void_p, C.c_void_p]
    lib.opf_wsnet_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.opf_wsnet_gradient.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                                       C.POINTER(C.c_double), C.c_void_p]
    lib.opf_wsnet_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                                         C.c_float, C.POINTER(C.c_double)]
    lib.opf_wsnet_destroy.argtypes = [C.c_void_p]
    lib.opf_wsnet_destroy.restype = None
    for name in ("opf_wsnet_create", "opf_wsnet_get_params", "opf_wsnet_set_params", "opf_wsnet_forward",
                 "opf_wsnet_gradient", "opf_wsnet_train_step"):
        getattr(lib, name).restype = C.c_int
    F32P = C.POINTER(C.c_float)
    lib.opf_diff_create.argtypes = [C.POINTER(opf_network), C.c_int32, C.POINTER(opf_contingencies),
                                    C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                    C.POINTER(C.c_void_p)]
    lib.opf_diff_cost_grad.argtypes = [C.c_void_p, C.c_int32, F32P, F32P, F32P, F64P, F32P, F32P, F32P]
    lib.opf_diff_cost_grad_on.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                          F64P, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.opf_diff_set_record_limit.argtypes = [C.c_void_p, C.c_int64]
    lib.opf_diff_destroy.argtypes = [C.c_void_p]
    lib.opf_diff_destroy.restype = None
    for name in ("opf_diff_create", "opf_diff_cost_grad", "opf_diff_cost_grad_on", "opf_diff_set_record_limit"):
        getattr(lib, name).restype = C.c_int
    for name in ("opf_create_slice", "opf_slice_exchange", "opf_slice_prime", "opf_slice_begin", "opf_slice_local",
                 "opf_slice_finish"):
        getattr(lib, name).restype = C.c_int
    for name in ("opf_create", "opf_iterate", "opf_residuals", "opf_solution", "opf_price_noalloc", "opf_history",
                 "opf_set_state_from_nodes",
                 "opf_get_state", "opf_set_state", "opf_reset", "opf_get_info"):
        getattr(lib, name).restype = C.c_int
    if path is None:
        _lib = lib
    return lib


def _status_str(s):
    try:
        return load_library().opf_status_str(int(s)).decode()
    except OSError:
        return "status"


def _check(status, where):
    if status != OPF_OK:
        raise OpfError(status, where, opf_last_error())


def opf_status_str(status):
    return load_library().opf_status_str(int(status)).decode()


def opf_last_error():
    return load_library().opf_last_error().decode()


def opf_abi_version():
    return int(load_library().opf_abi_version())


def opf_default_options(**overrides):
    o = opf_options()
    load_library().opf_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None and a.size else C.POINTER(ctype)()


# array lengths of a case: (count key, per time step) for every array field
_SIZES = {
    "line_to": ("line_from", False), "line_b": ("line_from", False), "line_u": ("line_from", False),
    "gen_a": ("gen_node", False), "gen_b": ("gen_node", False), "gen_ramp": ("gen_node", False),
    "gen_pmin": ("gen_node", True), "gen_pmax": ("gen_node", True),
    "load_p": ("load_node", True), "load_voll": ("load_node", False),
    "stor_P": ("stor_node", False), "stor_dur": ("stor_node", False), "stor_eff": ("stor_node", False),
    "stor_cost": ("stor_node", False),
    "hvdc_to": ("hvdc_from", False), "hvdc_u": ("hvdc_from", False),
}


def _check_sizes(case, where):
    """The C entry points take plain pointers and read n (or n x T) values
    behind each; an array of another length would be read past its end, so
    the lengths are checked here, against the declared horizon T."""
    T = int(case["T"])
    for name, (count_key, per_t) in _SIZES.items():
        n = len(case.get(count_key, ()))
        a = np.asarray(case.get(name, ()))
        if per_t:
            if a.size != n * T or (a.ndim == 2 and a.shape != (n, T)):
                raise OpfError(OPF_EINVAL, where, f"{name} has shape {a.shape}; expected ({n}, horizon T = {T})")
        elif a.size != n:
            raise OpfError(OPF_EINVAL, where, f"{name} has {a.size} values; expected {n}")


def _network(case, where="opf_create"):
    """The opf_network and opf_contingencies of a case dict, plus the arrays
    they point into (keep them alive while the structs are used)."""
    _check_sizes(case, where)
    keep = {}

    def f64(name, shape=None):
        a = np.ascontiguousarray(np.asarray(case.get(name, ()), dtype=np.float64))
        keep[name] = a
        return _ptr(a, C.c_double)

    def i32(name):
        a = np.ascontiguousarray(np.asarray(case.get(name, ()), dtype=np.int32))
        keep[name] = a
        return _ptr(a, C.c_int32)

    net = opf_network(
        n_nodes=int(case["n_nodes"]),
        n_lines=len(case["line_from"]), line_from=i32("line_from"), line_to=i32("line_to"),
        line_b=f64("line_b"), line_u=f64("line_u"),
        n_gens=len(case["gen_node"]), gen_node=i32("gen_node"), gen_a=f64("gen_a"),
        gen_b=f64("gen_b"), gen_pmin=f64("gen_pmin"), gen_pmax=f64("gen_pmax"),
        gen_ramp=f64("gen_ramp"),
        n_loads=len(case["load_node"]), load_node=i32("load_node"), load_p=f64("load_p"),
        load_voll=f64("load_voll"),
        n_stor=len(case["stor_node"]), stor_node=i32("stor_node"), stor_P=f64("stor_P"),
        stor_dur=f64("stor_dur"), stor_eff=f64("stor_eff"), stor_cost=f64("stor_cost"),
        n_hvdc=len(case.get("hvdc_from", ())), hvdc_from=i32("hvdc_from"), hvdc_to=i32("hvdc_to"),
        hvdc_u=f64("hvdc_u"),
    )
    out = np.ascontiguousarray(np.asarray(case["outaged"], dtype=np.int32))
    keep["outaged"] = out
    ctg = opf_contingencies(K=len(out), outaged_line=_ptr(out, C.c_int32))
    return net, ctg, keep


def opf_create(case, options=None, stream=None):
    """Create a solver context from a case dict (see ``gridgen``).  Returns the handle."""
    lib = load_library()
    T = int(case["T"])
    net, ctg, keep = _network(case)
    if options is None:
        options = opf_default_options()
    elif isinstance(options, dict):
        options = opf_default_options(**options)
    if stream is not None:
        options.cuda_stream = C.c_void_p(int(stream))
    h = C.c_void_p()
    _check(lib.opf_create(C.byref(net), T, C.byref(ctg), C.byref(options), C.byref(h)),
           "opf_create")
    try:
        _CTX_INFO[h.value] = opf_get_info(h)
    except OpfError:
        lib.opf_destroy(h)
        raise
    return h


def opf_create_slice(case, k_begin, k_end, options=None, stream=None):
    """A context for contingencies k_begin .. k_end - 1 of the case (0 is the
    base case); see include/opf.h for the iteration protocol."""
    lib = load_library()
    T = int(case["T"])
    net, ctg, keep = _network(case, "opf_create_slice")
    if options is None:
        options = opf_default_options()
    elif isinstance(options, dict):
        options = opf_default_options(**options)
    if stream is not None:
        options.cuda_stream = C.c_void_p(int(stream))
    h = C.c_void_p()
    _check(lib.opf_create_slice(C.byref(net), T, C.byref(ctg), int(k_begin), int(k_end), C.byref(options),
                                C.byref(h)), "opf_create_slice")
    try:
        _CTX_INFO[h.value] = opf_get_info(h)
    except OpfError:
        lib.opf_destroy(h)
        raise
    return h


class _DeviceBuffer:
    """A device array the library owns, exposed to torch without a copy."""

    def __init__(self, ptr, n, device):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}
        self.device = device


def opf_slice_exchange(h):
    """The slice's exchange buffer as a float64 CUDA tensor sharing the
    library's memory (sum it over the slices between local and finish)."""
    import torch
    ptr, n = C.c_void_p(), C.c_int64()
    _check(load_library().opf_slice_exchange(h, C.byref(ptr), C.byref(n)), "opf_slice_exchange")
    return torch.as_tensor(_DeviceBuffer(ptr.value, n.value, None), device="cuda")


def opf_slice_prime(h):
    _check(load_library().opf_slice_prime(h), "opf_slice_prime")


def opf_slice_begin(h, n_iters, rho=0.0):
    _check(load_library().opf_slice_begin(h, int(n_iters), float(rho)), "opf_slice_begin")


def opf_slice_local(h):
    _check(load_library().opf_slice_local(h), "opf_slice_local")


def opf_slice_finish(h):
    _check(load_library().opf_slice_finish(h), "opf_slice_finish")


def opf_destroy(h):
    if h:
        _CTX_INFO.pop(getattr(h, "value", h), None)
        load_library().opf_destroy(h)


def opf_iterate(h, n_iters, rho=0.0):
    _check(load_library().opf_iterate(h, int(n_iters), float(rho)), "opf_iterate")


def opf_residuals(h, raise_on_status=True):
    """Residuals of the last iteration (6 FP64 values) and the device status."""
    out = np.zeros(6)
    st = load_library().opf_residuals(h, out.ctypes.data_as(F64P))
    if raise_on_status:
        _check(st, "opf_residuals")
        return out
    return out, st


def opf_get_info(h):
    info = opf_info()
    _check(load_library().opf_get_info(h, C.byref(info)), "opf_get_info")
    return {name: getattr(info, name) for name, _ in opf_info._fields_}


def _addr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _buf(x, n, on_device, name, where):
    """Address of a float32 buffer of exactly n elements: a contiguous CUDA
    tensor when on_device, else a C-contiguous NumPy array.  The library
    reads or writes n elements behind the pointer, so anything else is
    refused here rather than touched out of bounds there."""
    if x is None:
        return None
    if on_device:
        ok = (hasattr(x, "data_ptr") and getattr(x, "is_cuda", False) and str(x.dtype) == "torch.float32"
              and x.is_contiguous() and x.numel() == n)
        if not ok:
            raise OpfError(OPF_EINVAL, where, f"{name} must be a contiguous float32 CUDA tensor of {n} elements")
        return x.data_ptr()
    ok = (isinstance(x, np.ndarray) and x.dtype == np.float32 and x.flags.c_contiguous and x.size == n)
    if not ok:
        raise OpfError(OPF_EINVAL, where, f"{name} must be a C-contiguous float32 NumPy array of {n} elements")
    return x.ctypes.data


# sizes of each context (fixed for its lifetime), filled by opf_create
_CTX_INFO = {}


def _ctx_info(h):
    info = _CTX_INFO.get(getattr(h, "value", h))
    return info if info is not None else opf_get_info(h)


def opf_solution(h, on_device=False, objective=True, p_dev=None, p_line=None, theta_node=None,
                 price=None):
    """Fill the given output buffers (NumPy float32 on host, tensors on device).

    Returns the objective (float) or None."""
    i = _ctx_info(h)
    Kp, L, N, S, T = i["k_count"], i["L"], i["N"], i["S"], i["T"]
    dv = bool(on_device)
    ptrs = [_buf(p_dev, S * T, dv, "p_dev", "opf_solution"), _buf(p_line, Kp * L * T, dv, "p_line", "opf_solution"),
            _buf(theta_node, Kp * N * T, dv, "theta_node", "opf_solution"),
            _buf(price, N * T, dv, "price", "opf_solution")]
    obj = C.c_double(0.0)
    st = load_library().opf_solution(h, int(dv), C.byref(obj) if objective else F64P(), *ptrs)
    _check(st, "opf_solution")
    return obj.value if objective else None


def opf_price_noalloc(h, out=None):
    """Nodal prices [N][T] into the host float32 array ``out`` (or a new one),
    staged through the library's fixed device array (no allocation)."""
    info = _ctx_info(h)
    if out is None:
        out = np.zeros((info["N"], info["T"]), np.float32)
    ptr = _buf(out, info["N"] * info["T"], False, "out", "opf_price_noalloc")
    _check(load_library().opf_price_noalloc(h, ptr), "opf_price_noalloc")
    return out


def opf_history(h, max_rows=None):
    """The residual history kept on the device (include/opf.h, opf_history):
    an array [rows, OPF_HISTORY_COLS], oldest row first, of the most recent
    ``max_rows`` rows (default: all that are kept)."""
    if max_rows is None:
        max_rows = int(opf_get_info(h)["history_rows"])
    max_rows = max(0, int(max_rows))
    out = np.zeros((max_rows, OPF_HISTORY_COLS), np.float64)
    n = C.c_int32(0)
    _check(load_library().opf_history(h, max_rows, out.ctypes.data if max_rows else None, C.byref(n)),
           "opf_history")
    return out[:n.value]


def opf_batch_create(handles):
    """A batch over existing context handles (they must outlive it)."""
    arr = (C.c_void_p * len(handles))(*handles)
    out = C.c_void_p()
    _check(load_library().opf_batch_create(arr, len(handles), C.byref(out)), "opf_batch_create")
    return out


def opf_batch_iterate(b, n_iters):
    _check(load_library().opf_batch_iterate(b, int(n_iters)), "opf_batch_iterate")


BATCH_LAYOUTS = ("as given, contiguous, 1x", "longest first, contiguous, 1x", "longest first, round-robin, 1x",
                 "as given, contiguous, 1/4", "longest first, contiguous, 1/4", "longest first, round-robin, 1/4")


def opf_batch_autotune(b, steps=20):
    """Time the candidate schedules and keep the fastest; returns (index into
    BATCH_LAYOUTS, ms per batch iteration of every layout).  Leaves the
    iterates unchanged."""
    choice = C.c_int32(-1)
    ms = (C.c_double * len(BATCH_LAYOUTS))()
    _check(load_library().opf_batch_autotune(b, int(steps), C.byref(choice), ms), "opf_batch_autotune")
    return choice.value, list(ms)


def opf_batch_compact(b):
    """Drop the stopped instances from the batch's schedule (the iterates do
    not change); returns how many instances it still schedules."""
    n = C.c_int32(0)
    _check(load_library().opf_batch_compact(b, C.byref(n)), "opf_batch_compact")
    return n.value


def opf_batch_converged(b):
    n = C.c_int32(0)
    _check(load_library().opf_batch_converged(b, C.byref(n)), "opf_batch_converged")
    return n.value


def opf_batch_stopped(b):
    """(converged, stalled, with an error status) instance counts of a batch."""
    n = [C.c_int32(0) for _ in range(3)]
    _check(load_library().opf_batch_stopped(b, *(C.byref(x) for x in n)), "opf_batch_stopped")
    return tuple(x.value for x in n)


def opf_batch_destroy(b):
    if b:
        load_library().opf_batch_destroy(b)


def opf_wsnet_param_count(n_features):
    return int(load_library().opf_wsnet_param_count(int(n_features)))


class WarmStartNet:
    """The learned warm-start network of include/opf_wsnet.h (device tensors
    in, device tensors out; host NumPy for parameters and gradients)."""

    def __init__(self, n_nodes, line_from, line_to, line_b, T, n_features, params=None, seed=0,
                 stream=None):
        lf = np.ascontiguousarray(line_from, np.int32)
        lt = np.ascontiguousarray(line_to, np.int32)
        lb = np.ascontiguousarray(line_b, np.float64)
        if not (lt.size == lf.size and lb.size == lf.size):
            raise OpfError(OPF_EINVAL, "opf_wsnet_create", "line_from, line_to and line_b differ in length")
        self.R = int(n_nodes) * int(T)
        self.F = int(n_features)
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        if p is not None and p.size != opf_wsnet_param_count(self.F):
            raise OpfError(OPF_EINVAL, "opf_wsnet_create",
                           f"params has {p.size} values; expected {opf_wsnet_param_count(self.F)}")
        self._keep = (lf, lt, lb, p)
        out = C.c_void_p()
        _check(load_library().opf_wsnet_create(
            int(n_nodes), len(lf), lf.ctypes.data_as(I32P), lt.ctypes.data_as(I32P),
            lb.ctypes.data_as(F64P), int(T), self.F, None if p is None else p.ctypes.data,
            int(seed), stream, C.byref(out)), "opf_wsnet_create")
        self.h = out

    def params(self):
        out = np.zeros(opf_wsnet_param_count(self.F), np.float32)
        _check(load_library().opf_wsnet_get_params(self.h, out.ctypes.data), "opf_wsnet_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        ptr = _buf(p, opf_wsnet_param_count(self.F), False, "params", "opf_wsnet_set_params")
        _check(load_library().opf_wsnet_set_params(self.h, ptr), "opf_wsnet_set_params")

    def _xy(self, x, y, where):
        return (_buf(x, self.R * self.F, True, "x", where),
                _buf(y, self.R * OPF_WSNET_OUT, True, "y", where))

    def forward(self, x, y):
        _check(load_library().opf_wsnet_forward(self.h, *self._xy(x, y, "opf_wsnet_forward")),
               "opf_wsnet_forward")
        return y

    def gradient(self, x, y_target, scale):
        sc = (C.c_float * 2)(*[float(v) for v in scale])
        loss = C.c_double(0.0)
        g = np.zeros(opf_wsnet_param_count(self.F), np.float32)
        _check(load_library().opf_wsnet_gradient(self.h, *self._xy(x, y_target, "opf_wsnet_gradient"), sc,
                                                 C.byref(loss), g.ctypes.data), "opf_wsnet_gradient")
        return loss.value, g

    def train_step(self, x, y_target, scale, lr):
        sc = (C.c_float * 2)(*[float(v) for v in scale])
        loss = C.c_double(0.0)
        _check(load_library().opf_wsnet_train_step(self.h, *self._xy(x, y_target, "opf_wsnet_train_step"), sc,
                                                   float(lr), C.byref(loss)), "opf_wsnet_train_step")
        return loss.value

    def close(self):
        if self.h:
            load_library().opf_wsnet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UnrolledCost:
    """The cost after K unrolled iterations and its gradients (include/opf_diff.h).

    ``cost_grad(K, load_p, gen_pmax, line_u)`` takes host arrays ([D][T],
    [G][T], [L]; None = the case's own) and returns (f, dict of gradients
    with the same keys and shapes)."""

    def __init__(self, case, rho_p=1.0, rho_theta=1.0, checkpoint_every=16, stream=None):
        net, ctg, keep = _network(case, "opf_diff_create")
        self.T = int(case["T"])
        self.D, self.G, self.L = len(case["load_node"]), len(case["gen_node"]), len(case["line_from"])
        out = C.c_void_p()
        _check(load_library().opf_diff_create(C.byref(net), self.T, C.byref(ctg), float(rho_p),
                                              float(rho_theta), int(checkpoint_every), stream,
                                              C.byref(out)), "opf_diff_create")
        del keep
        self.h = out

    def set_record_limit(self, nbytes):
        """Device memory a gradient call may keep for its record of the
        forward pass (opf_diff_set_record_limit); 0 recomputes instead."""
        _check(load_library().opf_diff_set_record_limit(self.h, int(nbytes)), "opf_diff_set_record_limit")

    def cost_grad(self, K, load_p=None, gen_pmax=None, line_u=None, grads=True):
        F32P = C.POINTER(C.c_float)

        def arr(x, shape):
            if x is None:
                return None, F32P()
            a = np.ascontiguousarray(np.asarray(x, np.float32).reshape(shape))
            return a, a.ctypes.data_as(F32P)

        a1, p1 = arr(load_p, (self.D, self.T))
        a2, p2 = arr(gen_pmax, (self.G, self.T))
        a3, p3 = arr(line_u, (self.L,))
        g = dict(load_p=np.zeros((self.D, self.T), np.float32), gen_pmax=np.zeros((self.G, self.T), np.float32),
                 line_u=np.zeros(self.L, np.float32))
        gp = [_ptr(g[k], C.c_float) if grads else F32P() for k in ("load_p", "gen_pmax", "line_u")]
        f = C.c_double(0.0)
        _check(load_library().opf_diff_cost_grad(self.h, int(K), p1, p2, p3, C.byref(f), *gp),
               "opf_diff_cost_grad")
        return f.value, (g if grads else None)

    def cost_grad_device(self, K, load_p, gen_pmax, line_u, grads=True):
        """The same with CUDA tensors (float32, contiguous; None = the case's
        own data): returns (f, dict of gradient tensors on the same device)."""
        import torch
        shapes = dict(load_p=(self.D, self.T), gen_pmax=(self.G, self.T), line_u=(self.L,))
        ins = dict(load_p=load_p, gen_pmax=gen_pmax, line_u=line_u)
        dev = next((x.device for x in ins.values() if x is not None), torch.device("cuda"))
        ptr = {k: (None if x is None else _buf(x, int(np.prod(shapes[k])), True, k, "opf_diff_cost_grad_on"))
               for k, x in ins.items()}
        g = {k: torch.zeros(s, dtype=torch.float32, device=dev) for k, s in shapes.items()} if grads else None
        gp = [g[k].data_ptr() if grads else None for k in ("load_p", "gen_pmax", "line_u")]
        f = C.c_double(0.0)
        _check(load_library().opf_diff_cost_grad_on(self.h, int(K), 1, ptr["load_p"], ptr["gen_pmax"],
                                                    ptr["line_u"], C.byref(f), *gp), "opf_diff_cost_grad_on")
        return f.value, g

    def close(self):
        if self.h:
            load_library().opf_diff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_UNROLLED_FN = None


def _unrolled_fn():
    global _UNROLLED_FN
    if _UNROLLED_FN is None:
        import torch

        class UnrolledCostFn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, diff, K, load_p, gen_pmax, line_u):
                want = any(ctx.needs_input_grad[2:])
                xs = (load_p, gen_pmax, line_u)
                if all(x.is_cuda for x in xs):
                    # device tensors go to the library as they are
                    dv = [x.detach().to(torch.float32).contiguous() for x in xs]
                    f, g = diff.cost_grad_device(K, *dv, grads=want)
                    if want:
                        ctx.save_for_backward(*[g[k].to(x.dtype) for k, x in zip(("load_p", "gen_pmax", "line_u"), xs)])
                else:
                    host = [x.detach().to("cpu", torch.float32).numpy() for x in xs]
                    f, g = diff.cost_grad(K, *host, grads=want)
                    if want:
                        ctx.save_for_backward(*[torch.from_numpy(g[k]).to(x.device, x.dtype) for k, x in
                                                zip(("load_p", "gen_pmax", "line_u"), xs)])
                return torch.tensor(f, dtype=load_p.dtype, device=load_p.device)

            @staticmethod
            def backward(ctx, go):
                gl, gp, gu = ctx.saved_tensors
                return None, None, go * gl, go * gp, go * gu

        _UNROLLED_FN = UnrolledCostFn
    return _UNROLLED_FN


def unrolled_cost(diff, K, load_p, gen_pmax, line_u):
    """f(p^K) of an :class:`UnrolledCost` as a torch scalar differentiable with
    respect to the tensors load_p [D][T], gen_pmax [G][T] and line_u [L]; the
    forward and the reverse pass both run in ``opf_diff_cost_grad``."""
    return _unrolled_fn().apply(diff, int(K), load_p, gen_pmax, line_u)


STATE_FIELDS = ("p_line", "th1", "th2", "v1", "v2", "p_dev", "u", "inner")


def state_shapes(info):
    Kp, L, N, S, T = info["k_count"], info["L"], info["N"], info["S"], info["T"]
    return dict(p_line=(Kp, L, T), th1=(Kp, L, T), th2=(Kp, L, T), v1=(Kp, L, T),
                v2=(Kp, L, T), p_dev=(S, T), u=(Kp, N, T), inner=(info["inner_len"],))


def opf_get_state(h, on_device=False, out=None):
    """Export the state into ``out`` (dict of buffers) or new host arrays."""
    info = _ctx_info(h)
    if out is None:
        if on_device:
            raise ValueError("pass device buffers in `out` for on_device=True")
        out = {k: np.zeros(s, np.float32) for k, s in state_shapes(info).items()}
    n = {k: int(np.prod(s)) for k, s in state_shapes(info).items()}
    st = opf_state(**{k: _buf(out.get(k), n[k], bool(on_device), k, "opf_get_state") for k in STATE_FIELDS})
    _check(load_library().opf_get_state(h, int(bool(on_device)), C.byref(st)), "opf_get_state")
    return out


def opf_set_state(h, state, on_device=False):
    """Import a state dict (missing keys are zeroed on the device)."""
    n = {k: int(np.prod(s)) for k, s in state_shapes(_ctx_info(h)).items()}
    keep = {}
    ptrs = {}
    for k in STATE_FIELDS:
        x = state.get(k)
        if x is None:
            ptrs[k] = None
            continue
        if not on_device:
            x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
            keep[k] = x
        ptrs[k] = _buf(x, n[k], bool(on_device), k, "opf_set_state")
    st = opf_state(**ptrs)
    _check(load_library().opf_set_state(h, int(bool(on_device)), C.byref(st)), "opf_set_state")


def opf_set_state_from_nodes(h, rows, price_scale, on_device=False):
    """Starting state from node rows [T * N, stride] (price / price_scale,
    angle, ...): a float32 CUDA tensor with on_device, else a NumPy array."""
    info = _ctx_info(h)
    R = info["N"] * info["T"]
    if on_device:
        if not (hasattr(rows, "data_ptr") and rows.dim() == 2 and rows.shape[0] == R):
            raise OpfError(OPF_EINVAL, "opf_set_state_from_nodes", f"rows must be a [{R}, stride] CUDA tensor")
        stride = int(rows.shape[1])
    else:
        rows = np.ascontiguousarray(np.asarray(rows, np.float32))
        if rows.ndim != 2 or rows.shape[0] != R:
            raise OpfError(OPF_EINVAL, "opf_set_state_from_nodes", f"rows must have shape [{R}, stride]")
        stride = int(rows.shape[1])
    ptr = _buf(rows, R * stride, bool(on_device), "rows", "opf_set_state_from_nodes")
    _check(load_library().opf_set_state_from_nodes(h, int(bool(on_device)), ptr, stride, float(price_scale)),
           "opf_set_state_from_nodes")


def opf_reset(h):
    _check(load_library().opf_reset(h), "opf_reset")


class Solver:
    """Owner of one context (calls opf_destroy when collected)."""

    def __init__(self, case, options=None, stream=None):
        self.h = opf_create(case, options, stream)
        self.info = opf_get_info(self.h)

    def iterate(self, n, rho=0.0):
        opf_iterate(self.h, n, rho)

    def residuals(self):
        return opf_residuals(self.h)

    def history(self, max_rows=None):
        return opf_history(self.h, max_rows)

    def get_info(self):
        return opf_get_info(self.h)

    def state(self):
        return opf_get_state(self.h)

    def set_state(self, st):
        opf_set_state(self.h, st)

    def solution(self):
        i = self.info
        Kp, L, N, S, T = i["k_count"], i["L"], i["N"], i["S"], i["T"]
        out = dict(p_dev=np.zeros((S, T), np.float32), p_line=np.zeros((Kp, L, T), np.float32),
                   theta_node=np.zeros((Kp, N, T), np.float32), price=np.zeros((N, T), np.float32))
        out["objective"] = opf_solution(self.h, False, True, **out)
        return out

    def close(self):
        if self.h:
            opf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
