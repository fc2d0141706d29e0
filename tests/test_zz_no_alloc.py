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

from helpers import rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

APPLY_TOL = 1e-12  # the FP64 apply tolerance of tests/test_gpu_apply.py


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_static_apply_matches_workspace_apply_on_two_calls():
    A = I.diffusion3d(20, 1.5, seed=3)
    alpha, beta, xi, k = 0.2, 40.0, 1e-3, 25
    S = P.Solver.from_host(A, k=k, interval="given", alpha=alpha, beta=beta, xi=xi, seed_scaling=False,
                           format="csr")
    rp, ci, va = P.to_device_csr(A)
    for seed in (1, 2):  # two calls in a row share the static array
        r = torch.as_tensor(I.rhs_normal(A.n, seed), device="cuda")
        z_ref = to_np(S.apply(r))
        z = to_np(P.apply_csr_static(rp, ci, va, A.n, alpha, beta, xi, k, r))
        torch.cuda.synchronize()
        assert rel(z, z_ref) <= APPLY_TOL


def test_static_apply_rejects_too_many_rows():
    one = ctypes.c_void_p(256)
    rc = P.lib().polyprec_apply_csr_static(262145, 262145, one, one, one, 1.0, 2.0, 0.0, 3, one, one, None)
    assert rc == P.PP_EINVAL
    assert b"262144" in P.lib().pp_last_error(None)
