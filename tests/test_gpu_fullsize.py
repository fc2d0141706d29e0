"""GPU parity at the sizes the benchmark runs, in the storage it times.

The 192^3 lognormal(sigma=2) diffusion matrix (7,077,888 rows) goes through
the symmetric DIA kernels the autotuner picks for it: one p_5 apply
(Algorithm 2) in FP64, FP32 and BF16 values, and three PCG iterations
(Section 1) in FP64, each compared with the FP64 oracle on every row.  The
128^3 matrix (2,097,152 rows) is larger than one round of every DIA
variant's grid (two resident waves of 256-thread blocks with 4 or 2 rows
per thread cover at most about 1.6M rows), so the grid-stride loops take a
second, partial round in every mode: the plain product, the residual, the
three recurrence steps, the Lanczos step and the fused inner products of
PCG and flexible CG.

Tolerances (the same as the small-case tests): FP64 apply 1e-12, three FP64
PCG iterations 1e-11, FP32/BF16 applies 2e-5 against the oracle run on the
same rounded matrix values, all relative 2-norm and per element.
"""
import numpy as np
import pytest

import oracle as O
from helpers import assert_close, oracle_apply, oracle_interval, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

ALPHA, BETA, XI = 0.0015, 2.0, 7.5e-3  # near the Lanczos interval of the 192^3 matrix


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def diff192():
    A = I.diffusion3d(192, 2.0, seed=1)
    return A, I.rhs_normal(A.n, 1)


@pytest.fixture(scope="module")
def diff128():
    A = I.diffusion3d(128, 2.0, seed=1)
    return A, I.rhs_normal(A.n, 1)


def round_bf16(x: np.ndarray) -> np.ndarray:
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def oracle_apply_rounded(A, r, alpha, beta, xi, k, prec):
    vh, w = O.jacobi_scale(A)
    vr = vh.astype(np.float32).astype(np.float64) if prec == "f32" else round_bf16(vh)
    return w * O.cheb_apply(A, alpha, beta, xi, k, w * r, val=vr)


def test_dia_192_f64_apply(diff192):
    A, b = diff192
    S = P.Solver.from_host(A, k=5, interval="given", alpha=ALPHA, beta=BETA, xi=XI, format="dia")
    assert S.info()["format"] == 3 and S.info()["ndiag"] == 3
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    assert_close(z, oracle_apply(A, b, ALPHA, BETA, XI, 5), 1e-12)
    S.close()


def test_dia_192_f64_three_pcg_iterations(diff192):
    A, b = diff192
    S = P.Solver.from_host(A, k=5, lanczos_steps=10, rtol=0.0, maxit=3, format="dia")
    info = S.info()
    x, st = S.solve(torch.as_tensor(b, device="cuda"), allow=(0, 1))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=5, lanczos_steps=10, rtol=0.0, maxit=3)
    assert so["alpha_hat"] == pytest.approx(info["alpha_hat"], rel=1e-9)
    assert so["beta_hat"] == pytest.approx(info["beta_hat"], rel=1e-9)
    assert st["iterations"] == 3 and st["status"] == P.PP_MAXIT
    assert_close(to_np(x), xo, 1e-11)
    S.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_dia_192_low_precision_apply(diff192, prec, variant):
    A, b = diff192
    S = P.Solver.from_host(A, k=5, interval="given", alpha=ALPHA, beta=BETA, xi=XI, format="dia", apply_prec=prec,
                           sell_variant=variant)
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, b, ALPHA, BETA, XI, 5, prec), 2e-5)
    S.close()


def test_dia_128_lanczos_interval(diff128):
    """kLanczos with its fused (y, x) product over two grid rounds."""
    A, _ = diff128
    S = P.Solver.from_host(A, k=2, lanczos_steps=10, seed=3, format="dia")
    lo, hi = oracle_interval(A, 3, 10)
    info = S.info()
    assert info["lanczos_steps_done"] == 10
    assert info["alpha_hat"] == pytest.approx(lo, rel=1e-9)
    assert info["beta_hat"] == pytest.approx(hi, rel=1e-9)
    S.close()


@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_dia_128_apply_and_product(diff128, k):
    """kCheb1 (k = 1), kCheb2 (k >= 2), kChebK (k >= 3) and kSpmv."""
    A, b = diff128
    S = P.Solver.from_host(A, k=k, interval="given", alpha=0.004, beta=2.0, xi=1e-3, format="dia")
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    assert_close(z, oracle_apply(A, b, 0.004, 2.0, 1e-3, k), 1e-12)
    x = I.rhs_normal(A.n, 5)
    assert_close(to_np(S.operator(torch.as_tensor(x, device="cuda"))), A.matvec(x), 1e-13)
    S.close()


@pytest.mark.parametrize("flexible", [0, 1])
def test_dia_128_pcg_fused_dots(diff128, flexible):
    """A nonzero initial guess runs the residual kernel (kResid with ||r||^2
    fused); PCG fuses (p, Ap) into the product and (r, z) into the last
    recurrence step; FCG(1) fuses (q, z) as well (two products)."""
    A, b = diff128
    x0 = I.rhs_normal(A.n, 6)
    S = P.Solver.from_host(A, k=4, lanczos_steps=10, rtol=0.0, maxit=3, format="dia", zero_guess=0,
                           flexible=flexible)
    x, st = S.solve(torch.as_tensor(b, device="cuda"), torch.as_tensor(x0, device="cuda").clone(), allow=(0, 1))
    xo, so = O.pcg_csr(A, b, x0=x0, v0=I.lanczos_start(A.n, 0), k=4, lanczos_steps=10, rtol=0.0, maxit=3,
                       flexible=bool(flexible))
    assert st["iterations"] == 3
    assert_close(to_np(x), xo, 1e-11)
    S.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_dia_128_low_precision_apply(diff128, prec, k, variant):
    A, b = diff128
    S = P.Solver.from_host(A, k=k, interval="given", alpha=0.004, beta=2.0, xi=1e-3, format="dia", apply_prec=prec,
                           sell_variant=variant)
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, b, 0.004, 2.0, 1e-3, k, prec), 2e-5)
    S.close()


LAYOUTS = [dict(format="csr"), dict(format="sell", sell_C=32, sell_variant=1),
           dict(format="sell", sell_C=64, sell_variant=2), dict(format="sell", sell_C=128, sell_variant=2),
           dict(format="dia")]


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
@pytest.mark.parametrize("blocks", [1, 3])
def test_capped_grid_takes_many_rounds(layout, blocks):
    """max_blocks caps every step and vector launch, so on a 20^3 matrix the
    grid-stride loops of every kernel run many rounds (one block covers at
    most 1,024 rows per round) and the grid reductions see one or three
    blocks: the apply, the product and three PCG iterations against the
    oracle."""
    A = I.diffusion3d(20, 2.0, seed=2)
    b = I.rhs_normal(A.n, 4)
    opts = dict(LAYOUTS[layout], max_blocks=blocks)
    S = P.Solver.from_host(A, k=7, interval="given", alpha=0.01, beta=2.0, xi=1e-3, **opts)
    assert S.info()["grid_blocks"] <= blocks
    z = to_np(S.apply(torch.as_tensor(b, device="cuda")))
    assert_close(z, oracle_apply(A, b, 0.01, 2.0, 1e-3, 7), 1e-12)
    x = I.rhs_normal(A.n, 5)
    assert_close(to_np(S.operator(torch.as_tensor(x, device="cuda"))), A.matvec(x), 1e-13)
    S2 = P.Solver.from_host(A, k=7, lanczos_steps=10, rtol=0.0, maxit=3, **opts)
    xs, st = S2.solve(torch.as_tensor(b, device="cuda"), allow=(0, 1))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=7, lanczos_steps=10, rtol=0.0, maxit=3)
    assert st["iterations"] == 3
    assert_close(to_np(xs), xo, 1e-11)
