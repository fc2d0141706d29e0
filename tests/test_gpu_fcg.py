"""GPU parity of truncated flexible CG, FCG(m) (opt.flexible = m >= 2),
against the FP64 oracle's FCG(m), through the C ABI.

Tolerances: with the FP64 apply (a fixed SPD preconditioner) the iterates
match the oracle within 1e-10 for a fixed iteration count and converged
solutions within 1e-10 (same iteration count +-1); with the FP32/BF16
apply the outer FP64 FCG(m) still reaches rtol 1e-8 and agrees with a tight
FP64 oracle solve within the accuracy that rtol allows (1e-7).
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


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("fmt", ["csr", "sell", "dia"])
def test_fixed_iterations_match_oracle(m, fmt):
    A = I.diffusion3d(16, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    opts = dict(k=5, rtol=0.0, maxit=11, flexible=m)
    S = P.Solver.from_host(A, format=fmt, check_every=3, **opts)
    x, st = S.solve(dev(b))
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), **opts)
    assert st["iterations"] == so["iterations"] == 11
    assert_close(to_np(x), xo, 1e-10)
    assert st["dots"] == (3 + m) * 11


@pytest.mark.parametrize("m", [2, 5])
def test_converged_solve_and_graphs(m):
    A = I.diffusion3d(18, 2.5, seed=3)
    b = I.rhs_normal(A.n, 2)
    xo, so = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=6, rtol=1e-10, flexible=m)
    res = []
    for graphs in (0, 1):
        S = P.Solver.from_host(A, k=6, rtol=1e-10, flexible=m, use_graphs=graphs, check_every=7)
        x, st = S.solve(dev(b))
        assert st["status"] == 0
        assert abs(st["iterations"] - so["iterations"]) <= 1
        assert_close(to_np(x), xo, 1e-10)
        res.append((to_np(x), st["iterations"]))
    assert res[0][1] == res[1][1] and np.array_equal(res[0][0], res[1][0])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_precision_fcg_m(prec):
    A = I.diffusion3d(24, 2.0, seed=2)
    b = I.rhs_normal(A.n, 5)
    xo, _ = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=12, rtol=1e-12)
    its = {}
    for m in (1, 4):
        S = P.Solver.from_host(A, k=12, rtol=1e-8, format="dia", apply_prec=prec, flexible=m)
        x, st = S.solve(dev(b))
        assert st["status"] == 0
        assert_close(to_np(x), xo, 1e-7)
        its[m] = st["iterations"]
    assert its[4] <= its[1] + 2


def test_schur_fcg_m_matches_oracle():
    net = I.fracture_network(n_f=24, side_min=3.0, side_max=9.0, h=0.25, trace_min=1.0, trace_max=6.0,
                             trace_fraction=0.06, T_sigma=1.0, seed=9)
    ref = O.Schur(net)
    r = ref.rhs(net.q)
    opts = dict(k=4, lanczos_steps=10, xi=1e-3, maxit=9, rtol=0.0, flexible=3)
    S = P.SchurSolver(net, **opts)
    u, st = S.solve(dev(r))
    uo, so = ref.pcg(ref.diag(), r, v0=I.lanczos_start(net.n_u, 0), **opts)
    assert st["iterations"] == so["iterations"] == 9
    assert_close(to_np(u), uo, 1e-10)


def test_flexible_out_of_range_rejected():
    A = I.poisson3d(4)
    with pytest.raises(P.PolyPrecError) as ei:
        P.Solver.from_host(A, k=3, flexible=9)
    assert ei.value.status == P.PP_EINVAL
