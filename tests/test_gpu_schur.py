"""GPU parity of the fracture-network Schur path (Section 4.2) against the
FP64 oracle (banded Cholesky per fracture, Algorithms 3 and 4 as printed,
with alpha kept).  Tolerances: relative 2-norm 1e-12 for A^{-1}, S_u r,
diag(S_u), the right-hand side and the recovery; PCG on S_hat with the same
options: same iteration count and solution within 1e-10.
"""
import numpy as np
import pytest

import oracle as O
from helpers import assert_close, rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


NETS = {
    "tiny": lambda: I.tiny_fracture_network(),
    "small": lambda: I.fracture_network(n_f=8, side_min=1.5, side_max=4.0, h=0.25, trace_min=0.5, trace_max=2.0,
                                        trace_fraction=0.1, seed=5),
    "medium": lambda: I.fracture_network(n_f=24, side_min=3.0, side_max=9.0, h=0.25, trace_min=1.0, trace_max=6.0,
                                         trace_fraction=0.06, T_sigma=1.0, seed=9),
}


@pytest.fixture(scope="module", params=list(NETS))
def pair(request):
    net = NETS[request.param]()
    return net, O.Schur(net)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_ainv(pair):
    net, ref = pair
    S = P.SchurSolver(net, k=4)
    v = I.rhs_normal(net.n_h, 3)
    y = to_np(S.ainv(dev(v)))
    assert_close(y, ref.ainv(v), TOL)
    assert_close(net.A.matvec(y), v, TOL)


def test_schur_apply(pair):
    net, ref = pair
    S = P.SchurSolver(net, k=4)
    for seed in (1, 2):
        r = I.rhs_normal(net.n_u, seed)
        assert_close(to_np(S.schur_apply(dev(r))), ref.apply(r), TOL)
    # the right-hand side also takes one product with the trace blocks
    assert_close(to_np(S.rhs(dev(net.q))), ref.rhs(net.q), TOL)


def test_schur_diag_alg4(pair):
    net, ref = pair
    S = P.SchurSolver(net, k=4)
    assert_close(to_np(S.diag()), ref.diag(), TOL)


def test_rhs_and_recovery(pair):
    net, ref = pair
    S = P.SchurSolver(net, k=4)
    r = to_np(S.rhs(dev(net.q)))
    assert_close(r, ref.rhs(net.q), TOL)
    u = I.rhs_normal(net.n_u, 4)
    h, p = S.recover(dev(net.q), dev(u))
    ho, po = ref.recover(net.q, u)
    assert_close(to_np(h), ho, TOL)
    assert_close(to_np(p), po, TOL)


@pytest.mark.parametrize("k", [0, 3, 8])
def test_pcg_on_scaled_schur(pair, k):
    net, ref = pair
    steps = min(10, net.n_u)
    S = P.SchurSolver(net, k=k, lanczos_steps=steps, rtol=1e-10, maxit=500)
    r = ref.rhs(net.q)
    u, st = S.solve(dev(r))
    uo, so = ref.pcg(ref.diag(), r, v0=I.lanczos_start(net.n_u, 0), k=k, lanczos_steps=steps, rtol=1e-10, maxit=500)
    assert st["status"] == 0 and so["status"] == 0
    assert st["alpha_hat"] == pytest.approx(so["alpha_hat"], rel=1e-9)
    assert st["beta_hat"] == pytest.approx(so["beta_hat"], rel=1e-9)
    if so["iterations"] <= 100 and not (k == 0 and st["iterations"] != so["iterations"]):
        assert st["iterations"] == so["iterations"]
        # up to 100 CG steps whose reductions round in a different order: the
        # relative solution error 1e-10, and twice that per element (scaled
        # by the largest entry)
        assert_close(to_np(u), uo, 1e-10, elem_tol=2e-10)
    else:
        # k = 0 (diagonal seed only, tens to hundreds of CG steps): the
        # stopping step is decided by the rounding order of the reductions
        # and of the products, so compare the count to 3% (at least one
        # step) and the solutions to the accuracy rtol 1e-10 allows
        assert abs(st["iterations"] - so["iterations"]) <= max(1, 0.03 * so["iterations"])
        assert_close(to_np(u), uo, 1e-7)
    assert st["mvp"] == st["iterations"] * (k + 1)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pcg_on_schur_with_graphs_matches_launches(pair, prec):
    """Blocks of PCG iterations on S_hat replayed as CUDA graphs give the
    launched-one-by-one solve exactly: the same kernels in the same order
    (FP64 and the FP32 preconditioner inside FCG(1))."""
    net, ref = pair
    steps = min(10, net.n_u)
    r = dev(ref.rhs(net.q))
    out = []
    for graphs in (0, 1):
        S = P.SchurSolver(net, k=6, lanczos_steps=steps, rtol=1e-10, maxit=500, use_graphs=graphs, check_every=4,
                          apply_prec=prec, flexible=1 if prec == "f32" else 0)
        u, st = S.solve(r)
        assert st["status"] == 0
        out.append((to_np(u), st["iterations"]))
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][0], out[1][0])


def test_polyprec_apply_on_schur(pair):
    """p_k(S_hat) by Algorithm 2 with the composite operator."""
    net, ref = pair
    S = P.SchurSolver(net, k=5, interval="given", alpha=0.05, beta=2.5, xi=1e-3)
    r = I.rhs_normal(net.n_u, 9)
    z = to_np(S.apply(dev(r)))
    ds = ref.diag()
    w = 1.0 / np.sqrt(ds)
    c = O.cheb_coeffs(0.05, 2.5, 1e-3, 5)

    # Algorithm 2 on S_hat = W S W with the oracle operator (dense columns)
    Sd = np.column_stack([ref.apply(e) for e in np.eye(net.n_u)]) if net.n_u <= 400 else None
    if Sd is None:
        pytest.skip("dense check only on small networks")
    Sh = (w[:, None] * Sd) * w[None, :]
    Ah = I.dense_to_csr(Sh)
    zo = w * O.cheb_apply(Ah, 0.05, 2.5, 1e-3, 5, w * r)
    assert_close(z, zo, 1e-11)
    assert c.theta_bar > 0


def test_end_to_end_matches_dense_K0():
    """GPU right-hand side, PCG on S_hat, recovery of h and p == dense K_0 solve."""
    net = I.tiny_fracture_network()
    A, C, B, Gh, Gu = (M.to_dense() for M in (net.A, net.C, net.B, net.Gh, net.Gu))
    a = net.alpha
    nh, nu = net.n_h, net.n_u
    K0 = np.block([[Gh, -a * B, A], [-a * B.T, Gu, -C.T], [A, -C, np.zeros((nh, nh))]])
    sol = np.linalg.solve(K0, np.concatenate([np.zeros(nh + nu), net.q]))
    S = P.SchurSolver(net, k=6, lanczos_steps=nu, rtol=1e-13, maxit=1000)
    q = dev(net.q)
    u, st = S.solve(S.rhs(q))
    h, p = S.recover(q, u)
    assert st["status"] == 0
    assert_close(to_np(u), sol[nh:nh + nu], 1e-9)
    assert_close(to_np(h), sol[:nh], 1e-9)
    assert_close(to_np(p), sol[nh + nu:], 1e-9)


def test_schur_rejects_bf16():
    """FP32 trace blocks are supported inside p_k; BF16 is not."""
    net = I.tiny_fracture_network()
    with pytest.raises(P.PolyPrecError) as ei:
        P.SchurSolver(net, apply_prec="bf16", flexible=1)
    assert ei.value.status == P.PP_EUNSUPPORTED


@pytest.mark.slow
def test_full_size_network_properties():
    """The 200-fracture network (seed 2): properties that hold at any size."""
    net = I.fracture_network()
    S = P.SchurSolver(net, k=20, lanczos_steps=10, rtol=1e-8, maxit=2000)
    v = I.rhs_normal(net.n_h, 1)
    y = to_np(S.ainv(dev(v)))
    assert_close(net.A.matvec(y), v, 1e-11)
    x1, x2 = I.rhs_normal(net.n_u, 1), I.rhs_normal(net.n_u, 2)
    s1, s2 = to_np(S.schur_apply(dev(x1))), to_np(S.schur_apply(dev(x2)))
    assert abs(x2 @ s1 - x1 @ s2) <= 1e-10 * abs(x2 @ s1)  # symmetric
    assert x1 @ s1 > 0 and x2 @ s2 > 0
    ds = to_np(S.diag())
    for i in (0, 17, net.n_u // 2, net.n_u - 1):
        e = np.zeros(net.n_u)
        e[i] = 1.0
        assert to_np(S.schur_apply(dev(e)))[i] == pytest.approx(ds[i], rel=1e-10)  # Algorithm 4 == Algorithm 3
    r = S.rhs(dev(net.q))
    u, st = S.solve(r)
    assert st["status"] == 0
    res = to_np(r) - to_np(S.schur_apply(u))
    assert np.linalg.norm(res) / np.linalg.norm(to_np(r)) <= 1e-6


@pytest.mark.parametrize("k", [3, 8])
def test_fp32_schur_preconditioner(pair, k):
    """p_k(S_hat) applied with the FP32 copy of the trace blocks (FP32 vectors,
    FP32 accumulation): within FP32 rounding of the FP64 apply; the outer
    flexible CG in FP64 still reaches the FP64 oracle's solution."""
    net, ref = pair
    S64 = P.SchurSolver(net, k=k, interval="given", alpha=0.05, beta=2.5, xi=1e-3)
    S32 = P.SchurSolver(net, k=k, interval="given", alpha=0.05, beta=2.5, xi=1e-3, apply_prec="f32", flexible=1)
    r = I.rhs_normal(net.n_u, 9)
    z64 = to_np(S64.apply(dev(r)))
    z32 = to_np(S32.apply(dev(r)))
    assert_close(z32, z64, 1e-4)
    steps = min(10, net.n_u)
    Sm = P.SchurSolver(net, k=k, lanczos_steps=steps, rtol=1e-10, maxit=800, apply_prec="f32", flexible=1)
    rr = ref.rhs(net.q)
    u, st = Sm.solve(dev(rr))
    uo, so = ref.pcg(ref.diag(), rr, v0=I.lanczos_start(net.n_u, 0), k=k, lanczos_steps=steps, rtol=1e-12,
                     maxit=5000)
    assert st["status"] == 0 and so["status"] == 0
    assert_close(to_np(u), uo, 1e-7)
