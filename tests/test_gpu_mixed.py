"""GPU parity of the precision variant: p_k(A_hat) applied with FP32 vectors
and FP32 or BF16 matrix values (FP32 accumulate), outer CG in FP64 with
flexible-CG directions.

Tolerances, derived from the arithmetic:
  * apply vs the FP64 oracle run on the *same rounded values* (so only the
    FP32 arithmetic differs): k steps of a stable three-term recurrence with
    unit roundoff 6e-8, relative error <= 2e-5 for k <= 25;
  * apply vs the exact FP64 oracle: FP32 values add a relative matrix
    perturbation of 6e-8 (stated, checked <= 1e-4); BF16 values 4e-3 (the
    error is reported, not bounded, since p_k amplifies it);
  * flexible-CG solves reach rtol 1e-8 and agree with the FP64 solve to
    within the accuracy that rtol allows.
"""
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


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest BF16 (8 significant bits, ties to even)."""
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def round_f32(x: np.ndarray) -> np.ndarray:
    return x.astype(np.float32).astype(np.float64)


def oracle_apply_rounded(A, r, alpha, beta, xi, k, prec):
    """Oracle W p_k(A~) W r where A~ holds the rounded seed-scaled values."""
    vh, w = O.jacobi_scale(A)
    vr = round_f32(vh) if prec == "f32" else round_bf16(vh)
    return w * O.cheb_apply(A, alpha, beta, xi, k, w * r, val=vr)


def oracle_apply_exact(A, r, alpha, beta, xi, k):
    vh, w = O.jacobi_scale(A)
    return w * O.cheb_apply(A, alpha, beta, xi, k, w * r, val=vh)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("C,var", [(32, 1), (64, 1), (128, 1), (32, 2), (64, 2), (128, 2)])
@pytest.mark.parametrize("k", [0, 1, 2, 7, 25])
def test_mixed_apply_matches_rounded_oracle(prec, C, var, k):
    A = I.diffusion3d(17, 2.0, seed=1)
    alpha, beta, xi = 0.05, 1.95, 1e-3
    S = P.Solver.from_host(A, k=k, interval="given", alpha=alpha, beta=beta, xi=xi, format="sell", sell_C=C,
                           sell_variant=var, apply_prec=prec)
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    ref = oracle_apply_rounded(A, r, alpha, beta, xi, k, prec)
    assert_close(z, ref, 2e-5)
    exact = oracle_apply_exact(A, r, alpha, beta, xi, k)
    if prec == "f32":
        assert_close(z, exact, 1e-4)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("k", [0, 1, 2, 7])
@pytest.mark.parametrize("N", [16, 17, 18])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_mixed_dia_apply(prec, k, N, variant):
    """Direct loads (variant 1; offsets N, N^2 multiples of the rows per
    thread or not), TMA-staged tiles (variant 2; tile ends, ranges clipped
    at both ends of the vectors, unaligned shifted starts) and plane marching
    (variant 3; even N, odd N falls back to direct loads)."""
    A = I.diffusion3d(N, 2.0, seed=1)
    S = P.Solver.from_host(A, k=k, interval="given", alpha=0.05, beta=1.95, xi=1e-3, format="dia", apply_prec=prec,
                           sell_variant=variant)
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, r, 0.05, 1.95, 1e-3, k, prec), 2e-5)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("N", [66, 68])
def test_mixed_dia_plane_marching_ragged_tiles(prec, N):
    """Plane marching with two 64-wide tiles in x, the second one ragged:
    N = 68 takes four grid columns per thread (16-row tiles in y), N = 66
    two (8-row tiles)."""
    A = I.diffusion3d(N, 2.0, seed=4)
    S = P.Solver.from_host(A, k=5, interval="given", alpha=0.05, beta=1.95, xi=1e-3, format="dia", apply_prec=prec,
                           sell_variant=3)
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, r, 0.05, 1.95, 1e-3, 5, prec), 2e-5)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("N", [18, 20])
@pytest.mark.parametrize("blocks", [1, 3])
def test_mixed_dia_plane_marching_capped_grid(prec, N, blocks):
    """max_blocks below the number of (tile, z chunk) items: the blocks walk
    the items with a grid stride (two and four grid columns per thread)."""
    A = I.diffusion3d(N, 2.0, seed=5)
    S = P.Solver.from_host(A, k=7, interval="given", alpha=0.05, beta=1.95, xi=1e-3, format="dia", apply_prec=prec,
                           sell_variant=3, max_blocks=blocks)
    assert S.info()["grid_blocks"] <= blocks
    r = I.rhs_normal(A.n, 6)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, r, 0.05, 1.95, 1e-3, 7, prec), 2e-5)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_csr_apply(prec):
    A = I.diffusion3d(9, 1.0, seed=2)
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.1, beta=1.9, xi=1e-3, format="csr", apply_prec=prec)
    r = I.rhs_normal(A.n, 1)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply_rounded(A, r, 0.1, 1.9, 1e-3, 6, prec), 2e-5)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_flexible_mixed_solve_reaches_rtol(prec):
    A = I.diffusion3d(24, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    S64 = P.Solver.from_host(A, k=16, rtol=1e-10, format="sell")
    x64, s64 = S64.solve(torch.as_tensor(b, device="cuda"))
    Sm = P.Solver.from_host(A, k=16, rtol=1e-10, format="sell", apply_prec=prec, flexible=1)
    xm, sm = Sm.solve(torch.as_tensor(b, device="cuda"))
    assert sm["status"] == 0
    assert sm["rel_res"] <= 1e-10
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=16, rtol=1e-12)
    # both GPU solutions are within the accuracy their residual allows
    assert_close(to_np(x64), xo, 1e-7)
    assert_close(to_np(xm), xo, 1e-7)
    # lower-precision preconditioner: a few more iterations at most
    assert sm["iterations"] <= 2 * s64["iterations"] + 5


def test_mixed_plain_cg_also_converges_f32():
    """FP32 p_k is nearly symmetric; plain PCG still converges on this case."""
    A = I.diffusion3d(16, 1.0, seed=3)
    b = I.rhs_normal(A.n, 2)
    S = P.Solver.from_host(A, k=10, rtol=1e-8, format="sell", apply_prec="f32")
    _, st = S.solve(torch.as_tensor(b, device="cuda"), allow=(0, 1, -2))
    assert st["status"] in (0, 1, -2)


@pytest.mark.parametrize("fmt", ["dia", "sell"])
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_fcg_with_graphs_matches_launches_and_times_steps(prec, fmt):
    """FCG(1) with the low-precision preconditioner: blocks of iterations
    replayed as CUDA graphs give the launched solve bit for bit, and the
    step-time events recorded by the graph's nodes give a positive time for
    the degree steps."""
    A = I.diffusion3d(20, 2.0, seed=4)
    b = torch.as_tensor(I.rhs_normal(A.n, 5), device="cuda")
    out = []
    for graphs in (0, 1):
        S = P.Solver.from_host(A, k=12, lanczos_steps=20, rtol=1e-8, apply_prec=prec, flexible=1, format=fmt,
                               use_graphs=graphs, check_every=5)
        x, st = S.solve(b)
        assert st["status"] == 0
        assert st["t_apply_ms"] > 0 and st["apply_launches"] > 0
        out.append((to_np(x), st["iterations"]))
        S.close()
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][0], out[1][0])
