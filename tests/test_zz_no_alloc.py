"""The workspace-free apply, for callers that cannot allocate device memory.

polyprec_apply_csr_static serves code that may not call cudaMalloc (a
component inside a host application that owns all device allocation, or a
loop where an allocation's device synchronization is not allowed): it
takes only inputs and outputs and keeps its recurrence vectors in a static
device array.  This file is collected last on purpose, so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from helpers import assert_close, oracle_apply, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

APPLY_TOL = 1e-12  # the FP64 apply tolerance of tests/test_gpu_apply.py


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 25])
def test_static_apply_matches_workspace_apply_on_two_calls(k):
    """k = 0 (scaling only), 1 and 2 (first steps) and k mod 3 = 0, 1, 2
    (the three rotations of the recurrence buffers over z and the static
    array), each on two calls in a row, against the workspace apply and the
    oracle's Algorithm 2."""
    A = I.diffusion3d(20, 1.5, seed=3)
    alpha, beta, xi = 0.2, 450.0, 1e-3  # beta above the Gershgorin bound 433
    S = P.Solver.from_host(A, k=k, interval="given", alpha=alpha, beta=beta, xi=xi, seed_scaling=False,
                           format="csr")
    rp, ci, va = P.to_device_csr(A)
    for seed in (1, 2):  # two calls in a row share the static array
        rh = I.rhs_normal(A.n, seed)
        r = torch.as_tensor(rh, device="cuda")
        z_ref = to_np(S.apply(r))
        z = to_np(P.apply_csr_static(rp, ci, va, A.n, alpha, beta, xi, k, r))
        torch.cuda.synchronize()
        assert_close(z, z_ref, APPLY_TOL)
        assert_close(z, oracle_apply(A, rh, alpha, beta, xi, k, seed_scaling=False), APPLY_TOL)


def test_static_apply_at_the_row_limit():
    """n = 64^3 = 262,144 rows, exactly the size of the static array."""
    A = I.diffusion3d(64, 1.0, seed=5)
    assert A.n == 262144
    alpha, beta, xi, k = 0.5, 110.0, 1e-3, 5  # beta above the Gershgorin bound 108
    rp, ci, va = P.to_device_csr(A)
    rh = I.rhs_normal(A.n, 3)
    z = to_np(P.apply_csr_static(rp, ci, va, A.n, alpha, beta, xi, k, torch.as_tensor(rh, device="cuda")))
    torch.cuda.synchronize()
    assert_close(z, oracle_apply(A, rh, alpha, beta, xi, k, seed_scaling=False), APPLY_TOL)


def test_static_apply_rejects_overlapping_output():
    A = I.diffusion3d(6, 1.0, seed=1)
    rp, ci, va = P.to_device_csr(A)
    r = torch.as_tensor(I.rhs_normal(A.n, 1), device="cuda")
    with pytest.raises(P.PolyPrecError) as ei:
        P.apply_csr_static(rp, ci, va, A.n, 0.5, 50.0, 0.0, 4, r, r)
    assert ei.value.status == P.PP_EINVAL


def test_static_apply_rejects_too_many_rows():
    one = ctypes.c_void_p(256)
    z = ctypes.c_void_p(1 << 30)  # apart from r: the size check is the one that fails
    rc = P.lib().polyprec_apply_csr_static(262145, 262145, one, one, one, 1.0, 2.0, 0.0, 3, one, z, None)
    assert rc == P.PP_EINVAL
    assert b"262144" in P.lib().pp_last_error(None)
