"""The C ABI without a GPU: the library loads, exports every function that
include/opf.h declares, the ctypes structures match the C layout, and the host
side rejects invalid networks before touching the device."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "opf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2410_17203_gb300 import build, binding
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.load_library()


def declared_functions():
    """Every function declared in the headers under include/."""
    names = set()
    inc = os.path.dirname(HEADER)
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(opf_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_2410_17203_gb300 import binding
    assert set(names) == set(binding.EXPORTS)


def test_history_columns_and_status_codes_match_header():
    from paper_2410_17203_gb300 import binding
    h = open(HEADER).read()
    m = re.search(r"#define OPF_HISTORY_COLS (\d+)", h)
    assert m and binding.OPF_HISTORY_COLS == int(m.group(1))
    for name in ("OPF_ESTATE", "OPF_ESTALLED", "OPF_ENONFINITE"):
        m = re.search(name + r" = (\d+)", h)
        assert m and getattr(binding, name) == int(m.group(1)), name


def test_price_scratch_capacity_matches_header():
    from paper_2410_17203_gb300 import binding
    m = re.search(r"#define OPF_PRICE_SCRATCH_FLOATS \(1 << (\d+)\)", open(HEADER).read())
    assert m and binding.OPF_PRICE_SCRATCH_FLOATS == 1 << int(m.group(1))


def test_abi_version_and_status_strings(lib):
    from paper_2410_17203_gb300 import binding as b
    assert b.opf_abi_version() == 5
    for s in range(8):
        assert b.opf_status_str(s) not in ("", "unknown status")
    assert b.opf_status_str(99) == "unknown status"


def test_default_options_are_the_papers(lib):
    from paper_2410_17203_gb300 import opf_default_options
    o = opf_default_options()
    assert (o.rho_p, o.rho_theta, o.mu, o.gamma) == (1.0, 1.0, 2.0, 1.1)
    assert (o.adapt_every, o.inner_iters, o.check_every, o.eps) == (10, 10, 10, 1e-4)
    # no limit on the adaptation and no stall rule (Section 3.5 adapts for the whole run)
    assert (o.adapt_until, o.stall_window, o.history_len) == (0, 0, 4096)


def test_ctypes_layout_matches_c(lib, tmp_path):
    """Compile a probe against opf.h with gcc and compare sizes and offsets."""
    from paper_2410_17203_gb300 import binding as b
    structs = {"opf_network": b.opf_network, "opf_contingencies": b.opf_contingencies,
               "opf_options": b.opf_options, "opf_state": b.opf_state, "opf_info": b.opf_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "opf.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "probe.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if l)
    for sname, cls in structs.items():
        assert int(got[sname]) == __import__("ctypes").sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[f"{sname}.{f}"]) == getattr(cls, f).offset, f"{sname}.{f}"


def _bad(case, **changes):
    c = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in case.items()}
    for k, v in changes.items():
        if callable(v):
            v(c)
        else:
            c[k] = v
    return c


@pytest.mark.parametrize("mutate, what", [
    (lambda c: c["line_from"].__setitem__(0, 30), "line node id out of range"),
    (lambda c: c["line_to"].__setitem__(2, c["line_from"][2]), "itself"),
    (lambda c: c["line_b"].__setitem__(1, 0.0), "susceptance"),
    (lambda c: c["line_u"].__setitem__(1, -1.0), "line limit"),
    (lambda c: c["gen_pmin"].__setitem__((0, 0), 9.0), "pmin > pmax"),
    (lambda c: c["gen_a"].__setitem__(0, -0.1), "quadratic cost"),
    (lambda c: c["load_p"].__setitem__((3, 0), np.nan), "non-finite load"),
    (lambda c: c["gen_node"].__setitem__(0, -1), "generator node id"),
    (lambda c: c.__setitem__("outaged", np.array([40], np.int32)), "outaged line"),
    (lambda c: c.__setitem__("T", 0), "horizon"),
    (lambda c: c.__setitem__("T", 4096), "horizon"),
    (lambda c: c.update(hvdc_from=np.array([3], np.int32), hvdc_to=np.array([3], np.int32),
                        hvdc_u=np.array([1.0])), "HVDC link connects a node to itself"),
    (lambda c: c.update(hvdc_from=np.array([3], np.int32), hvdc_to=np.array([30], np.int32),
                        hvdc_u=np.array([1.0])), "HVDC node id"),
    (lambda c: c.update(hvdc_from=np.array([3], np.int32), hvdc_to=np.array([4], np.int32),
                        hvdc_u=np.array([-1.0])), "HVDC limit"),
])
def test_invalid_networks_are_rejected_on_the_host(lib, mutate, what):
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, opf_create
    case = make_case("tiny")
    if what == "horizon":
        bad = _bad(case)
        mutate(bad)
        T = bad["T"]
        bad.update(T=max(T, 1))
        # the arrays stay T=1; only the declared horizon is wrong
        bad["T"] = T
    else:
        bad = _bad(case)
        mutate(bad)
    with pytest.raises(OpfError) as e:
        opf_create(bad)
    assert e.value.status == 1
    assert what.split()[0].lower() in str(e.value).lower()


@pytest.mark.parametrize("T", [0, -3, 2049])
def test_horizon_is_checked_by_the_library(lib, T):
    """The C entry point itself rejects a horizon outside [1, 2048] before
    reading any array (called here without the binding's size checks)."""
    import ctypes as C
    from gridgen import make_case
    from paper_2410_17203_gb300 import binding as b
    net, ctg, keep = b._network(make_case("tiny"))
    h = C.c_void_p()
    assert lib.opf_create(C.byref(net), T, C.byref(ctg), None, C.byref(h)) == b.OPF_EINVAL
    assert "horizon" in b.opf_last_error().lower() and not h


@pytest.mark.parametrize("mutate, what", [
    (lambda c: c.__setitem__("line_u", c["line_u"][:-1]), "line_u has 39 values; expected 40"),
    (lambda c: c.__setitem__("gen_pmax", c["gen_pmax"][:, [0, 0]]), "gen_pmax has shape (6, 2)"),
    (lambda c: c.__setitem__("load_p", np.zeros((1, 20))), "load_p has shape (1, 20)"),
    (lambda c: c.__setitem__("stor_eff", np.ones(2)), "stor_eff has 2 values; expected 0"),
    (lambda c: c.update(hvdc_from=np.array([1], np.int32), hvdc_to=np.array([2, 3], np.int32),
                        hvdc_u=np.ones(1)), "hvdc_to has 2 values; expected 1"),
])
def test_array_lengths_are_checked_by_the_binding(lib, mutate, what):
    """Plain pointers carry no length: the binding checks every array against
    the counts and the horizon before the library reads them."""
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, UnrolledCost, opf_create
    bad = _bad(make_case("tiny"))
    mutate(bad)
    for make in (opf_create, UnrolledCost):
        with pytest.raises(OpfError) as e:
            make(bad)
        assert e.value.status == 1 and what in str(e.value)


def test_isolated_node_is_rejected(lib):
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, opf_create
    case = make_case("tiny")
    case["n_nodes"] = 31          # node 30 has no terminal
    with pytest.raises(OpfError, match="no terminal"):
        opf_create(case)


@pytest.mark.parametrize("opt", [dict(rho_p=0.0), dict(rho_theta=-1.0), dict(inner_iters=0),
                                 dict(gamma=0.5), dict(adapt_every=-1)])
def test_invalid_options_are_rejected(lib, opt):
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, opf_create
    with pytest.raises(OpfError) as e:
        opf_create(make_case("tiny"), opt)
    assert e.value.status == 1


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2410_17203_gb300 import binding
    with pytest.raises(OSError):
        binding.load_library(str(tmp_path / "missing.so"))


def test_valid_network_without_a_gpu_fails_loudly(lib):
    """With no CUDA device the library reports the failed CUDA call; it has
    no host fallback that would iterate on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the context is created there")
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, opf_create
    with pytest.raises(OpfError) as e:
        opf_create(make_case("tiny"))
    assert e.value.status in (2, 3)            # OPF_ENOMEM / OPF_ECUDA, never OPF_OK


def test_buffers_are_checked_before_the_library_touches_them(lib):
    """Output and input buffers travel as plain pointers: the binding accepts
    only float32 buffers of the exact element count (C-contiguous NumPy on the
    host, contiguous CUDA tensors on the device)."""
    import torch
    from paper_2410_17203_gb300 import OpfError, binding as b
    ok = np.zeros((3, 4), np.float32)
    assert b._buf(ok, 12, False, "x", "f") == ok.ctypes.data
    assert b._buf(None, 12, False, "x", "f") is None
    for bad in (np.zeros((3, 5), np.float32), np.zeros((3, 4)), np.zeros((4, 3), np.float32).T,
                torch.zeros(12)):
        with pytest.raises(OpfError) as e:
            b._buf(bad, 12, False, "x", "f")
        assert e.value.status == 1 and "12 elements" in str(e.value)
    # a host tensor is not a device buffer
    with pytest.raises(OpfError, match="CUDA tensor"):
        b._buf(torch.zeros(12), 12, True, "x", "f")


def test_warm_start_network_arguments_are_checked(lib):
    from paper_2410_17203_gb300 import OpfError, WarmStartNet, binding as b
    with pytest.raises(OpfError, match="differ in length"):
        WarmStartNet(4, [0, 1, 2], [1, 2], [1.0, 1.0, 1.0], 2, 3)
    with pytest.raises(OpfError, match="params has 5 values"):
        WarmStartNet(4, [0, 1, 2], [1, 2, 3], [1.0, 1.0, 1.0], 2, 3, params=np.zeros(5, np.float32))
    assert b.opf_wsnet_param_count(3) == 64 * 3 + 64 + 3 * (2 * 64 * 64 + 64) + 64 * 2 + 2


def test_slice_range_is_checked_on_the_host(lib):
    """opf_create_slice refuses an empty or out-of-range block of
    contingencies, and over-relaxation, before touching the device."""
    from gridgen import make_case
    from paper_2410_17203_gb300 import OpfError, opf_create_slice
    case = make_case("tiny")                     # K = 5: contingencies 0 .. 5
    for a, b in [(0, 0), (3, 2), (-1, 2), (0, 7), (6, 7)]:
        with pytest.raises(OpfError) as e:
            opf_create_slice(case, a, b)
        assert e.value.status == 1, (a, b)
    with pytest.raises(OpfError) as e:
        opf_create_slice(case, 0, 3, dict(alpha=1.5))
    assert e.value.status == 1
