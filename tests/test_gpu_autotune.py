"""The autotuner of the step storage (pp_autotune): every candidate layout
is built and timed, the fastest is returned, and solving with it gives the
oracle's answer (the layout does not change the method)."""
import ctypes

import numpy as np
import pytest

import oracle as O
from helpers import assert_close, rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_autotune_picks_fastest_and_solves(prec):
    A = I.diffusion3d(24, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    rp, ci, va = P.to_device_csr(A)
    base = dict(k=6, rtol=1e-10, apply_prec=prec, flexible=1 if prec != "f64" else 0)
    chosen, table = P.autotune(rp, ci, va, A.n, **base)
    # CSR, DIA (FP32/BF16: direct, TMA-staged, plane marching) and 12 SELL layouts
    assert len(table) == (14 if prec == "f64" else 16)
    assert all(t["status"] == 0 and t["us_per_step"] > 0 for t in table)
    best = min(t["us_per_step"] for t in table)
    pick = next(t for t in table if t["us_per_step"] <= 1.03 * best)  # ties within 3%: first in order
    assert (P.FORMAT_NAME[pick["format"]], pick["sell_C"], pick["sell_sigma"], pick["sell_variant"]) == (
        chosen["format"], chosen["sell_C"], chosen["sell_sigma"], chosen["sell_variant"])
    assert table[0]["format"] == 3 and table[-1]["format"] == 1  # DIA first, CSR last
    S = P.Solver(rp, ci, va, A.n, **chosen)
    x, st = S.solve(torch.as_tensor(b, device="cuda"))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=6, rtol=1e-10, flexible=prec != "f64")
    assert st["status"] == 0
    if prec == "f64":
        assert st["iterations"] == so["iterations"]
        assert_close(to_np(x), xo, 1e-10)
    else:
        assert_close(to_np(x), xo, 1e-7)


def test_autotune_skips_layouts_that_do_not_fit():
    A = I.diffusion3d(20, 1.0, seed=2)
    rp, ci, va = P.to_device_csr(A)
    lib = P.lib()
    o = P.make_options(k=4)
    csr = P.Csr(A.n, A.nnz, P._ptr(rp), P._ptr(ci), P._ptr(va))
    need = {}
    for fmt, C, sig in (("csr", 0, 0), ("sell", 128, 1024)):
        oc = P.make_options(k=4, format=fmt, sell_C=C, sell_sigma=sig, interval="given", alpha=1e-2, beta=2.0)
        nb = ctypes.c_size_t()
        assert lib.pp_workspace_size(ctypes.byref(csr), ctypes.byref(oc), ctypes.byref(nb)) == 0
        need[fmt] = nb.value
    small = min(need.values())
    ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    ent = (P.TuneEntry * 16)()
    cnt = ctypes.c_int()
    rc = lib.pp_autotune(ctypes.byref(csr), ctypes.byref(o), P._ptr(ws), small, ent, 16, ctypes.byref(cnt), None)
    assert rc == 0
    st = [ent[i].status for i in range(cnt.value)]
    assert 0 in st and P.PP_EINVAL in st
    ok = [ent[i] for i in range(cnt.value) if ent[i].status == 0]
    fastest = min(e.us_per_step for e in ok)
    best = next(e for e in ok if e.us_per_step <= 1.03 * fastest)
    assert (o.format, o.sell_C, o.sell_variant) == (best.format, best.sell_C, best.sell_variant)
