"""GPU parity of pcg_solve against the FP64 oracle (Section 1 PCG with the
Chebyshev preconditioner), through the C ABI.

Tolerances (spec: relative solution error 1e-10 in FP64):
  * same options, same stopping test -> same iteration count and
    ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-10;
  * fixed iteration count (maxit) -> iterates within 1e-11;
  * rtol 1e-12 -> within 1e-10 of a dense direct solve.
"""
import os

import numpy as np
import pytest

import oracle as O
from helpers import assert_close, rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gpu_solve(A, b, x0=None, **opts):
    S = P.Solver.from_host(A, **opts)
    bt = torch.as_tensor(b, device="cuda")
    xt = None if x0 is None else torch.as_tensor(x0, device="cuda").clone()
    x, st = S.solve(bt, xt, allow=(0, 1, -2, -3))
    torch.cuda.synchronize()
    return to_np(x), st, S


def oracle_solve(A, b, x0=None, seed=0, **opts):
    return O.pcg_csr(A, b, x0=x0, v0=I.lanczos_start(A.n, seed), **opts)


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_poisson32_k20_matches_oracle(fmt):
    """The 32^3 Poisson workload: k = 20, 10 Lanczos steps, xi by the
    10/kappa rule, rtol 1e-8."""
    A = I.poisson3d(32)
    b = I.rhs_ones_plus_noise(A, 0)
    xg, sg, S = gpu_solve(A, b, k=20, lanczos_steps=10, format=fmt, rtol=1e-8)
    xo, so = oracle_solve(A, b, k=20, lanczos_steps=10, rtol=1e-8)
    assert sg["status"] == 0 and so["status"] == 0
    assert sg["iterations"] == so["iterations"]
    assert sg["alpha_hat"] == pytest.approx(so["alpha_hat"], rel=1e-9)
    assert sg["beta_hat"] == pytest.approx(so["beta_hat"], rel=1e-9)
    assert_close(xg, xo, 1e-10)
    assert sg["mvp"] == sg["iterations"] * 21 and sg["dots"] == 3 * sg["iterations"]
    assert np.linalg.norm(b - A.matvec(xg)) / np.linalg.norm(b) <= 1e-7


def test_tight_solve_matches_dense():
    A = I.diffusion3d(12, 1.5, seed=1)
    b = I.rhs_normal(A.n, 2)
    xg, sg, _ = gpu_solve(A, b, k=10, rtol=1e-13, lanczos_steps=20)
    assert sg["status"] == 0
    assert_close(xg, np.linalg.solve(A.to_dense(), b), 1e-10)


@pytest.mark.parametrize("fmt,C,sigma,var", [("csr", 0, 0, 0), ("sell", 32, 0, 1), ("sell", 64, 0, 1),
                                             ("sell", 32, 0, 2), ("sell", 64, 0, 2), ("sell", 64, 512, 2),
                                             ("dia", 0, 0, 0)])
def test_fixed_iterations_iterates(fmt, C, sigma, var):
    A = I.diffusion3d(20, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    opts = dict(k=12, lanczos_steps=10, rtol=0.0, maxit=3)
    xg, sg, _ = gpu_solve(A, b, format=fmt, sell_C=C, sell_sigma=sigma, sell_variant=var, **opts)
    xo, so = oracle_solve(A, b, **opts)
    assert sg["status"] == P.PP_MAXIT and so["status"] == 1
    assert sg["iterations"] == 3
    assert_close(xg, xo, 1e-11)


def test_results_independent_of_check_interval_and_graphs():
    A = I.diffusion3d(16, 2.0, seed=2)
    b = I.rhs_normal(A.n, 3)
    ref = None
    for ce in (1, 3, 8):
        for g in (0, 1):
            x, st, _ = gpu_solve(A, b, k=7, check_every=ce, use_graphs=g, rtol=1e-9)
            assert st["status"] == 0
            if ref is None:
                ref = (x, st["iterations"])
            assert st["iterations"] == ref[1]
            assert np.array_equal(x, ref[0])  # deterministic reductions: bit-identical


def test_repeat_solves_bit_identical():
    A = I.diffusion3d(14, 1.0, seed=5)
    b = I.rhs_normal(A.n, 4)
    S = P.Solver.from_host(A, k=9, rtol=1e-9)
    bt = torch.as_tensor(b, device="cuda")
    x1, s1 = S.solve(bt)
    x2, s2 = S.solve(bt)
    assert s1["iterations"] == s2["iterations"]
    assert torch.equal(x1, x2)


def test_nonzero_initial_guess():
    A = I.diffusion3d(12, 1.0, seed=3)
    b = I.rhs_normal(A.n, 5)
    x0 = I.rhs_normal(A.n, 6)
    xg, sg, _ = gpu_solve(A, b, x0=x0, k=6, rtol=1e-10, zero_guess=0)
    xo, so = oracle_solve(A, b, x0=x0, k=6, rtol=1e-10)
    assert sg["status"] == 0 and sg["iterations"] == so["iterations"]
    assert_close(xg, xo, 1e-10)
    assert sg["mvp"] == sg["iterations"] * 7 + 1


def test_flexible_cg():
    A = I.diffusion3d(14, 2.0, seed=4)
    b = I.rhs_normal(A.n, 7)
    x1, s1, _ = gpu_solve(A, b, k=8, rtol=1e-10)
    x2, s2, _ = gpu_solve(A, b, k=8, rtol=1e-10, flexible=1)
    xo, so = oracle_solve(A, b, k=8, rtol=1e-10, flexible=True)
    assert s2["status"] == 0 and abs(s1["iterations"] - s2["iterations"]) <= 1
    assert s2["iterations"] == so["iterations"]
    assert_close(x2, xo, 1e-10)
    assert_close(x1, x2, 1e-8)


def test_zero_rhs_and_degree_zero():
    A = I.poisson3d(6)
    x, st, _ = gpu_solve(A, np.zeros(A.n), k=5)
    assert st["status"] == 0 and st["iterations"] == 0 and not x.any()
    b = I.rhs_normal(A.n, 1)
    xg, sg, _ = gpu_solve(A, b, k=0, rtol=1e-10)
    xo, so = oracle_solve(A, b, k=0, rtol=1e-10)
    assert sg["iterations"] == so["iterations"] and rel(xg, xo) <= 1e-10


def test_breakdown_is_reported_not_faulted():
    """An interval far below lambda_max makes p_k(A) A indefinite (odd k)."""
    A = I.diagonal(300)
    b = I.rhs_uniform(300, 0)
    x, st, _ = gpu_solve(A, b, k=3, interval="given", alpha=1.0, beta=20.0, xi=0.0, seed_scaling=False,
                         rtol=1e-10, maxit=60)
    _, so = O.pcg_csr(A, b, k=3, interval="given", alpha=1.0, beta=20.0, xi=0.0, seed_scaling=False, rtol=1e-10,
                      maxit=60)
    assert st["status"] == so["status"] and st["status"] in (P.PP_EBREAKDOWN, P.PP_MAXIT)
    assert st["iterations"] == so["iterations"]


def test_nan_rhs_reports_nonfinite():
    A = I.poisson3d(5)
    b = I.rhs_normal(A.n, 1)
    b[3] = np.nan
    _, st, _ = gpu_solve(A, b, k=3)
    assert st["status"] == P.PP_ENONFINITE


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_table1_iterations_on_gpu(fmt):
    """Table 1: the PCG iteration counts of the diagonal test on the GPU."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1.txt"))
    n = 100000
    A = I.diagonal(n)
    b = I.rhs_uniform(n, 0)
    for row in rows:
        xi, iters = float(row[0]), int(row[1])
        _, st, _ = gpu_solve(A, b, k=63, interval="given", alpha=1.0, beta=float(n), xi=xi, seed_scaling=False,
                             rtol=1e-10, format=fmt)
        assert st["status"] == 0
        assert st["iterations"] == iters


@pytest.mark.slow
def test_full_size_192_apply_and_iterations():
    """The 192^3 lognormal(sigma=2) diffusion workload in the configuration the
    benchmark times (SELL-C-sigma, FP64): one p_20 apply compared with the
    oracle over all 7,077,888 rows, and three PCG iterations compared."""
    from helpers import oracle_apply

    A = I.diffusion3d(192, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    S = P.Solver.from_host(A, k=20, lanczos_steps=10, rtol=0.0, maxit=3, format="sell")
    info = S.info()
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    ref = oracle_apply(A, b, info["alpha_hat"], info["beta_hat"], info["xi"], 20)
    assert_close(z, ref, 1e-12)
    x, st = S.solve(torch.as_tensor(b, device="cuda"), allow=(0, 1))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=20, lanczos_steps=10, rtol=0.0, maxit=3)
    assert so["alpha_hat"] == pytest.approx(info["alpha_hat"], rel=1e-9)
    assert st["iterations"] == 3
    assert_close(to_np(x), xo, 1e-11)
