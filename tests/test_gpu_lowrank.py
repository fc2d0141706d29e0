"""GPU parity of the low-rank acceleration (Section 3.1) against the FP64
oracle, through the C ABI.

P = W (p_k(A_hat) + V (V^T A_hat V)^{-1} V^T) W^T, with V either caller
vectors (pp_set_lowrank; V = W^{-1} U) or the Ritz vectors of the p
smallest Ritz values of a Lanczos run with full reorthogonalisation on
p_k(A_hat) A_hat.

Tolerances:
  * one application with caller vectors: <= 1e-12 (FP64; same formula);
  * the Lanczos run: Ritz values / interval to 1e-9 relative; Ritz vectors
    are compared through the preconditioner they define (sign-free) to
    1e-8, their conditioning being the gap of the Ritz values;
  * PCG for a fixed iteration count: iterates within 1e-9; converged solves
    within 1e-10 of the oracle with the same iteration count (+-1).
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def scaled(A):
    vh, w = O.jacobi_scale(A)
    return I.CSR(A.n, A.rowptr, A.col, vh), w


def oracle_ritz(Ah, steps, p, seed=0):
    a, b, Q = O.lanczos_basis(Ah, I.lanczos_start(Ah.n, seed), steps)
    V = np.column_stack([Q @ O.tridiag_eig(a, b[:-1], i)[1] for i in range(p)])
    lo, hi = O.tridiag_extremes(a, b[:-1])
    return V, lo, hi, a, b


LAYOUTS = [dict(format="csr"), dict(format="sell", sell_C=32, sell_variant=1),
           dict(format="sell", sell_C=64, sell_variant=2), dict(format="sell", sell_C=64, sell_sigma=512, sell_variant=2)]


@pytest.mark.parametrize("lay", LAYOUTS, ids=["csr", "sell32", "sell64tma", "sell64sorted"])
@pytest.mark.parametrize("p", [1, 5])
def test_apply_with_caller_vectors(lay, p):
    A = I.diffusion3d(13, 2.0, seed=1)  # 2197 rows: several slices and a ragged tail
    Ah, w = scaled(A)
    rng = np.random.default_rng(p)
    U = rng.standard_normal((A.n, p))
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.02, beta=1.9, xi=1e-3, lowrank=p, **lay)
    S.set_lowrank(dev(U.T))
    assert S.info()["lowrank"] == p
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(dev(r)))
    zo = w * O.lowrank_apply(Ah, 0.02, 1.9, 1e-3, 6, U / w[:, None], w * r)
    assert_close(z, zo, 1e-12)
    # p = 0 removes the correction
    S.set_lowrank(torch.empty(0, dtype=torch.float64, device="cuda"))
    z0 = to_np(S.apply(dev(r)))
    assert_close(z0, w * O.cheb_apply(Ah, 0.02, 1.9, 1e-3, 6, w * r), 1e-12)


def test_apply_mixed_precision_with_caller_vectors():
    """FP32 polynomial, FP64 correction: the error is that of the FP32 apply."""
    A = I.diffusion3d(13, 2.0, seed=1)
    Ah, w = scaled(A)
    U = np.random.default_rng(9).standard_normal((A.n, 2))
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.02, beta=1.9, xi=1e-3, lowrank=2, format="sell",
                           apply_prec="f32")
    S.set_lowrank(dev(U.T))
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(dev(r)))
    zo = w * O.lowrank_apply(Ah, 0.02, 1.9, 1e-3, 6, U / w[:, None], w * r)
    assert_close(z, zo, 2e-5)


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_ritz_vectors_and_interval(fmt):
    """Vectors from Lanczos on p_k(A_hat) A_hat, their Rayleigh quotients
    and the preconditioner they define; the interval is the estimator's."""
    A = I.diffusion3d(12, 2.0, seed=2)
    Ah, w = scaled(A)
    p, m, k = 3, 30, 5
    v0 = I.lanczos_start(A.n, 0)
    a, b = O.lanczos(Ah, v0, 10)
    lo, hi = O.tridiag_extremes(a, b)
    V, th = O.lowrank_vectors(Ah, v0, lo, hi, 1e-3, k, p, m)
    lo2 = lo
    S = P.Solver.from_host(A, k=k, lanczos_steps=10, lowrank=p, lowrank_steps=m, xi=1e-3, format=fmt)
    info = S.info()
    assert info["lowrank_steps_done"] == m and info["lowrank"] == p
    assert info["theta_min"] == pytest.approx(th.min(), rel=1e-9)
    assert info["alpha_hat"] == pytest.approx(lo2, rel=1e-9)
    assert info["beta_hat"] == pytest.approx(hi, rel=1e-9)
    D = Ah.to_dense()
    res = max(np.linalg.norm(D @ V[:, i] - th[i] * V[:, i]) / th[i] for i in range(p))
    assert info["ritz_resid"] <= max(1e-6, 10 * res)
    r = I.rhs_normal(A.n, 5)
    z = to_np(S.apply(dev(r)))
    zo = w * O.lowrank_apply(Ah, lo2, hi, 1e-3, k, V, w * r)
    assert_close(z, zo, 1e-8)


@pytest.mark.parametrize("p,flexible,graphs", [(1, 0, 0), (4, 0, 1), (2, 1, 0)])
def test_pcg_fixed_iterations(p, flexible, graphs):
    A = I.diffusion3d(14, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    opts = dict(k=4, lanczos_steps=30, rtol=0.0, maxit=6, xi=1e-3, lowrank=p, flexible=flexible)
    S = P.Solver.from_host(A, use_graphs=graphs, check_every=3, **opts)
    x, st = S.solve(dev(b))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), **opts)
    assert st["status"] == P.PP_MAXIT and so["status"] == 1
    assert st["iterations"] == so["iterations"] == 6
    assert_close(to_np(x), xo, 1e-9)
    assert st["dots"] == (3 + p) * 6  # Table 4 convention: (3 + p) per iteration
    assert st["mvp"] == 5 * 6


def test_pcg_converged_matches_oracle_and_dense():
    A = I.diffusion3d(12, 2.5, seed=4)
    b = I.rhs_normal(A.n, 2)
    opts = dict(k=3, lanczos_steps=50, rtol=1e-11, xi=1e-3, lowrank=3)
    S = P.Solver.from_host(A, format="sell", **opts)
    x, st = S.solve(dev(b))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), **opts)
    assert st["status"] == 0 and so["status"] == 0
    assert abs(st["iterations"] - so["iterations"]) <= 1
    assert_close(to_np(x), xo, 1e-10)
    assert_close(to_np(x), np.linalg.solve(A.to_dense(), b), 1e-9)
    assert st["dots"] == 6 * st["iterations"] and so["dots"] == 6 * so["iterations"]


def test_graphs_do_not_change_results():
    A = I.diffusion3d(16, 2.0, seed=3)
    b = I.rhs_normal(A.n, 4)
    res = []
    for graphs in (0, 1):
        S = P.Solver.from_host(A, k=5, lanczos_steps=30, lowrank=2, rtol=1e-9, use_graphs=graphs, check_every=5)
        x, st = S.solve(dev(b))
        res.append((to_np(x), st["iterations"]))
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][0], res[1][0])


def test_set_lowrank_errors():
    A = I.diffusion3d(8, 1.0, seed=1)
    S = P.Solver.from_host(A, k=3, lanczos_steps=12, lowrank=2)
    U = np.random.default_rng(0).standard_normal((A.n, 3))
    with pytest.raises(P.PolyPrecError) as ei:
        S.set_lowrank(dev(U.T))  # p = 3 > capacity 2
    assert ei.value.status == P.PP_EINVAL
    D = np.column_stack([U[:, 0], U[:, 0]])  # dependent columns: V^T A V singular
    with pytest.raises(P.PolyPrecError) as ei:
        S.set_lowrank(dev(D.T))
    assert ei.value.status in (P.PP_EBREAKDOWN,)
    assert S.info()["lowrank"] == 0
    with pytest.raises(P.PolyPrecError):
        P.Solver.from_host(A, k=3, lowrank=4, lowrank_steps=2)  # fewer steps than vectors


def test_schur_lowrank_pcg_matches_oracle():
    net = I.fracture_network(n_f=24, side_min=3.0, side_max=9.0, h=0.25, trace_min=1.0, trace_max=6.0,
                             trace_fraction=0.06, T_sigma=1.0, seed=9)
    ref = O.Schur(net)
    r = ref.rhs(net.q)
    steps = min(40, net.n_u)
    opts = dict(k=4, lanczos_steps=10, lowrank=1, lowrank_steps=steps, xi=1e-3, maxit=8, rtol=0.0)
    S = P.SchurSolver(net, **opts)
    u, st = S.solve(dev(r))
    uo, so = ref.pcg(ref.diag(), r, v0=I.lanczos_start(net.n_u, 0), **opts)
    assert st["iterations"] == so["iterations"] == 8
    assert st["alpha_hat"] == pytest.approx(so["alpha_hat"], rel=1e-9)
    assert_close(to_np(u), uo, 1e-9)
    assert st["dots"] == 4 * 8
