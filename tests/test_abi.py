"""The C-ABI library loads and exports every entry point of include/polyprec.h,
the binding's struct layouts match the C compiler's, and the host-only logic
(coefficients, option defaults, argument checks) is right.  No GPU needed:
nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2208_01339_gb300 import build as B
from paper_2208_01339_gb300 import polyprec as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polyprec.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
    bound = {s[0] for s in P.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sizes.c"
    fields = {
        "pp_csr": [f for f, _ in P.Csr._fields_],
        "pp_options": [f for f, _ in P.Options._fields_],
        "pp_stats": [f for f, _ in P.Stats._fields_],
        "pp_info": [f for f, _ in P.Info._fields_],
        "pp_dfn": [f for f, _ in P.Dfn._fields_],
        "pp_batch_item": [f for f, _ in P.BatchItem._fields_],
        "pp_tune_entry": [f for f, _ in P.TuneEntry._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {k: int(v) for k, v in (ln.split() for ln in out if ln.strip())}
    for st, cls in (("pp_csr", P.Csr), ("pp_options", P.Options), ("pp_stats", P.Stats), ("pp_info", P.Info),
                    ("pp_dfn", P.Dfn), ("pp_batch_item", P.BatchItem), ("pp_tune_entry", P.TuneEntry)):
        assert c[st] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert c[f"{st}.{f}"] == getattr(cls, f).offset, f"{st}.{f}"


def test_options_default(lib):
    o = P.make_options()
    assert (o.k, o.xi, o.interval, o.lanczos_steps, o.seed_scaling, o.apply_prec, o.maxit) == (20, -1.0, 0, 10, 1, 0,
                                                                                              10000)
    assert o.rtol == 1e-8 and o.zero_guess == 1 and o.check_every == 4


@pytest.mark.parametrize("alpha,beta,xi,k", [(1.0, 1e5, 0.0, 63), (1.0, 1e5, 1e-4, 63), (0.0272, 11.97, 1e-3, 20),
                                             (0.3, 2.0, 1e-2, 0), (0.5, 0.6, 0.0, 200)])
def test_coeffs_match_oracle(lib, alpha, beta, xi, k):
    tb, d, sb, rho = P.polyprec_coeffs(alpha, beta, xi, k)
    c = O.cheb_coeffs(alpha, beta, xi, k)
    assert tb == pytest.approx(c.theta_bar, rel=1e-15)
    assert d == pytest.approx(c.delta, rel=1e-15)
    assert sb == pytest.approx(c.sigma_bar, rel=1e-15)
    np.testing.assert_allclose(rho, c.rho, rtol=1e-13)


@pytest.mark.parametrize("args", [(2.0, 1.0, 0.0, 3), (0.0, 1.0, 0.0, 3), (1.0, 2.0, -1e-3, 3), (1.0, 2.0, 0.0, -1),
                                  (1.0, float("inf"), 0.0, 3)])
def test_coeffs_reject_invalid(lib, args):
    with pytest.raises(P.PolyPrecError) as ei:
        P.polyprec_coeffs(*args)
    assert ei.value.status == P.PP_EINVAL


def test_null_arguments_rejected_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    o = P.make_options()
    nbytes = ctypes.c_size_t()
    assert lib.pp_workspace_size(None, ctypes.byref(o), ctypes.byref(nbytes)) == P.PP_EINVAL
    csr = P.Csr(0, 0, None, None, None)
    assert lib.pp_workspace_size(ctypes.byref(csr), ctypes.byref(o), ctypes.byref(nbytes)) == P.PP_EINVAL
    bad = P.make_options(k=-2)
    csr = P.Csr(10, 10, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16))
    assert lib.pp_workspace_size(ctypes.byref(csr), ctypes.byref(bad), ctypes.byref(nbytes)) == P.PP_EINVAL
    assert lib.pcg_solve(None, None, None, None, None) == P.PP_EINVAL
    assert lib.polyprec_apply(None, None, None, 1, None) == P.PP_EINVAL
    assert lib.pp_destroy(None) == P.PP_OK
    assert lib.pp_autotune(None, None, None, 0, None, 0, None, None) == P.PP_EINVAL
    assert lib.pp_autotune(ctypes.byref(csr), ctypes.byref(o), ctypes.c_void_p(8), 1 << 20, None, 0, None,
                           None) == P.PP_EINVAL  # unaligned workspace
    assert lib.pp_set_lowrank(None, None, 0, 0, None) == P.PP_EINVAL
    assert lib.pp_fracture_bands(0, None, None, None, None, None, None) == P.PP_EINVAL
    off = np.array([0, 2], dtype=np.int64)
    assert lib.pp_fracture_bands(1, ctypes.c_void_p(off.ctypes.data), None, None, None, None, None) == P.PP_EINVAL
    assert b"NULL" in lib.pp_last_error(None)


def test_static_apply_argument_checks_without_gpu(lib):
    """polyprec_apply_csr_static checks its arguments before any CUDA call:
    too many rows, z overlapping r, and a negative degree."""
    one = ctypes.c_void_p(256)
    f = lib.polyprec_apply_csr_static
    assert f(262145, 262145, one, one, one, 1.0, 2.0, 0.0, 3, one, ctypes.c_void_p(1 << 24), None) == P.PP_EINVAL
    assert b"262144" in lib.pp_last_error(None)
    r, z = ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 8 * 99)  # z starts inside r[0:100]
    assert f(100, 300, one, one, one, 1.0, 2.0, 0.0, 4, r, z, None) == P.PP_EINVAL
    assert b"overlap" in lib.pp_last_error(None)
    assert f(100, 300, one, one, one, 1.0, 2.0, 0.0, 4, r, r, None) == P.PP_EINVAL
    assert f(100, 300, one, one, one, 1.0, 2.0, 0.0, -1, r, ctypes.c_void_p(1 << 24), None) == P.PP_EINVAL


def test_max_blocks_option_checked(lib):
    bad = P.make_options(max_blocks=-1)
    csr = P.Csr(10, 10, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16))
    nbytes = ctypes.c_size_t()
    assert lib.pp_workspace_size(ctypes.byref(csr), ctypes.byref(bad), ctypes.byref(nbytes)) == P.PP_EINVAL
    assert b"max_blocks" in lib.pp_last_error(None)


def test_fma_rate_argument_checks_without_gpu(lib):
    out = ctypes.c_double()
    assert lib.pp_fp64_fma_rate(None, 3, ctypes.byref(out), None) == P.PP_EINVAL
    assert lib.pp_fp64_fma_rate(ctypes.c_void_p(256), 0, ctypes.byref(out), None) == P.PP_EINVAL
    assert lib.pp_fp64_fma_rate(ctypes.c_void_p(256), 3, None, None) == P.PP_EINVAL


def test_batch_tuning_argument_checks_without_gpu(lib):
    o = P.make_options()
    us = ctypes.c_double()
    assert lib.pp_batch_time_step(None, 3, ctypes.byref(us), None) == P.PP_EINVAL
    nbytes = ctypes.c_size_t()
    assert lib.pp_batch_autotune_workspace_size(None, 1, None, ctypes.byref(nbytes)) == P.PP_EINVAL
    assert lib.pp_batch_autotune(None, 1, ctypes.byref(o), ctypes.c_void_p(256), 1 << 20, None, 0, None,
                                 None) == P.PP_EINVAL
    assert lib.pp_batch_autotune(None, 1, ctypes.byref(o), ctypes.c_void_p(8), 1 << 20, None, 0, None,
                                 None) == P.PP_EINVAL  # unaligned workspace
