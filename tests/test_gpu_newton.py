"""GPU parity of the Newton-form preconditioner (Algorithm 1, opt.poly =
PP_POLY_NEWTON) against the oracle's Algorithm 1, and its equality with the
Chebyshev recurrence (Algorithm 2) at the same degree 2^nlev - 1.

Tolerances: one application within 1e-12 of the oracle's Newton form
(FP64); Newton and Chebyshev forms of the same polynomial within 1e-10 up to
nlev = 5 (they differ by rounding only); PCG iterates with the Newton form
within 1e-9 of the oracle's PCG with the Chebyshev form for a fixed
iteration count.
"""
import numpy as np
import pytest

import oracle as O
from helpers import assert_close, oracle_apply, rel, to_np
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


def oracle_newton(A, r, alpha, beta, xi, nlev):
    vh, w = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh)
    return w * O.newton_apply(Ah, alpha, beta, xi, nlev, w * r)


@pytest.mark.parametrize("nlev", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("fmt", ["csr", "sell", "dia"])
def test_newton_apply_matches_oracle(nlev, fmt):
    A = I.diffusion3d(13, 2.0, seed=1)
    k = 2 ** nlev - 1
    S = P.Solver.from_host(A, k=k, interval="given", alpha=0.05, beta=1.95, xi=1e-3, poly="newton", format=fmt)
    r = I.rhs_normal(A.n, 4)
    z = to_np(S.apply(dev(r)))
    assert_close(z, oracle_newton(A, r, 0.05, 1.95, 1e-3, nlev), 1e-12)
    if nlev <= 5:
        assert_close(z, oracle_apply(A, r, 0.05, 1.95, 1e-3, k), 1e-10)


def test_newton_pcg_matches_chebyshev_pcg():
    A = I.diffusion3d(16, 2.0, seed=2)
    b = I.rhs_normal(A.n, 3)
    S = P.Solver.from_host(A, k=7, poly="newton", rtol=0.0, maxit=6, format="dia")
    x, st = S.solve(dev(b))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=7, rtol=0.0, maxit=6)
    assert st["iterations"] == 6
    assert_close(to_np(x), xo, 1e-9)
    S2 = P.Solver.from_host(A, k=15, poly="newton", rtol=1e-10, use_graphs=1, check_every=4)
    x2, st2 = S2.solve(dev(b))
    xo2, so2 = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=15, rtol=1e-10)
    assert st2["status"] == 0 and abs(st2["iterations"] - so2["iterations"]) <= 1
    assert_close(to_np(x2), xo2, 1e-9)
    assert st2["mvp"] == 16 * st2["iterations"]


def test_newton_on_schur():
    net = I.fracture_network(n_f=8, side_min=1.5, side_max=4.0, h=0.25, trace_min=0.5, trace_max=2.0,
                             trace_fraction=0.1, seed=5)
    ref = O.Schur(net)
    r = ref.rhs(net.q)
    S = P.SchurSolver(net, k=3, poly="newton", lanczos_steps=10, xi=1e-3, maxit=5, rtol=0.0)
    u, st = S.solve(dev(r))
    uo, so = ref.pcg(ref.diag(), r, v0=I.lanczos_start(net.n_u, 0), k=3, lanczos_steps=10, xi=1e-3, maxit=5, rtol=0.0)
    assert st["iterations"] == 5
    assert_close(to_np(u), uo, 1e-9)


def test_newton_rejects_bad_degree_and_mixed():
    A = I.poisson3d(5)
    with pytest.raises(P.PolyPrecError) as ei:
        P.Solver.from_host(A, k=6, poly="newton")
    assert ei.value.status == P.PP_EINVAL
    with pytest.raises(P.PolyPrecError) as ei:
        P.Solver.from_host(A, k=7, poly="newton", apply_prec="f32", flexible=1)
    assert ei.value.status == P.PP_EUNSUPPORTED
