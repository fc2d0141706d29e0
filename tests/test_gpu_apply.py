"""GPU parity of polyprec_apply (Algorithm 2), the Lanczos interval and the
operator product against the FP64 CPU oracle, through the C ABI.

Tolerance: FP64 apply, relative 2-norm error <= 1e-12 (k fused steps of a
stable three-term recurrence; the GPU and the oracle differ only in the
rounding order of each row sum and in FMA contraction).
"""
import numpy as np
import pytest

from helpers import assert_close, oracle_apply, oracle_interval, rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

APPLY_TOL = 1e-12

MATS = {
    "poisson5": lambda: I.poisson3d(5),
    "diff11": lambda: I.diffusion3d(11, 2.0, seed=1),
    "diff23": lambda: I.diffusion3d(23, 1.0, seed=3),
}
LAYOUTS = [
    dict(format="csr"),
    dict(format="sell", sell_C=32, sell_variant=1),
    dict(format="sell", sell_C=64, sell_variant=1),
    dict(format="sell", sell_C=32, sell_variant=2),
    dict(format="sell", sell_C=64, sell_variant=2),
    dict(format="sell", sell_C=64, sell_sigma=256, sell_variant=1),
    dict(format="sell", sell_C=64, sell_sigma=256, sell_variant=2),
    dict(format="dia"),
]


def width8_matrix(n=1024):
    """SPD matrix with offsets 0, +-1, +-2, +-3 and one partner i ^ 64: eight
    entries in interior rows (the widest slice staged through shared memory)."""
    D = np.zeros((n, n))
    for i in range(n):
        for d, v in ((1, -1.0), (2, -0.5), (3, -0.25)):
            if i + d < n:
                D[i, i + d] = D[i + d, i] = v
        D[i, i ^ 64] = -0.3
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 1.0)
    return I.dense_to_csr(D)


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
@pytest.mark.parametrize("k", [0, 1, 2, 3, 8, 25])
def test_apply_matches_oracle(mat, layout, k):
    A = MATS[mat]()
    alpha, beta, xi = 0.05, 1.95, 1e-3
    S = P.Solver.from_host(A, k=k, interval="given", alpha=alpha, beta=beta, xi=xi, **LAYOUTS[layout])
    r = I.rhs_normal(A.n, 7)
    z = S.apply(torch.as_tensor(r, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle_apply(A, r, alpha, beta, xi, k)
    assert_close(to_np(z), ref, APPLY_TOL)


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
def test_apply_without_seed_scaling(layout):
    A = I.diffusion3d(9, 0.5, seed=2)
    S = P.Solver.from_host(A, k=5, interval="given", alpha=0.5, beta=14.0, xi=0.0, seed_scaling=False,
                           **LAYOUTS[layout])
    r = I.rhs_normal(A.n, 1)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply(A, r, 0.5, 14.0, 0.0, 5, seed_scaling=False), APPLY_TOL)


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
@pytest.mark.parametrize("which", ["w8", "dense60"])
def test_apply_wide_slices(layout, which):
    """Slices of width 8 (straight-line path) and 60 (wider than the shared
    memory staging buffer: direct-load fallback inside the TMA kernel)."""
    A = width8_matrix() if which == "w8" else I.dense_to_csr(I.random_spd(60, seed=3, cond=30.0))
    if which == "dense60" and LAYOUTS[layout]["format"] == "dia":
        with pytest.raises(P.PolyPrecError) as ei:  # 60 diagonals: DIA does not apply
            P.Solver.from_host(A, k=6, interval="given", alpha=0.05, beta=1.95, **LAYOUTS[layout])
        assert ei.value.status == P.PP_EUNSUPPORTED
        return
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.05, beta=1.95, xi=1e-3, **LAYOUTS[layout])
    r = I.rhs_normal(A.n, 2)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply(A, r, 0.05, 1.95, 1e-3, 6), APPLY_TOL)


def test_apply_multiple_rhs():
    A = I.diffusion3d(10, 1.0, seed=4)
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.1, beta=1.9, xi=1e-3, format="sell")
    R = np.stack([I.rhs_normal(A.n, s) for s in range(3)])
    Z = to_np(S.apply(torch.as_tensor(R, device="cuda")))
    for j in range(3):
        assert_close(Z[j], oracle_apply(A, R[j], 0.1, 1.9, 1e-3, 6), APPLY_TOL)


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
@pytest.mark.parametrize("steps", [10, 30])
def test_lanczos_interval_matches_oracle(layout, steps):
    A = I.diffusion3d(12, 2.0, seed=1)
    S = P.Solver.from_host(A, k=4, lanczos_steps=steps, seed=5, **LAYOUTS[layout])
    info = S.info()
    lo, hi = oracle_interval(A, 5, steps)
    assert info["lanczos_steps_done"] == steps
    assert info["alpha_hat"] == pytest.approx(lo, rel=1e-9)
    assert info["beta_hat"] == pytest.approx(hi, rel=1e-9)
    assert info["xi"] == pytest.approx(min(max(10 * lo / hi, 1e-6), 1e-2), rel=1e-12)


def test_lanczos_start_vector_bits():
    """The device SplitMix64 stream equals the shared generator bit for bit:
    with n Lanczos steps on a tiny diagonal matrix the Ritz values are exact,
    and the first step's alpha_1 = v^T A v / v^T v depends on every bit."""
    A = I.diagonal(50)
    S = P.Solver.from_host(A, k=1, lanczos_steps=1, seed=11, seed_scaling=False)
    v = I.lanczos_start(50, 11)
    a1 = float(v @ (np.arange(1, 51) * v) / (v @ v))
    assert S.info()["alpha_hat"] == pytest.approx(a1, rel=1e-14)


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
def test_operator_product(layout):
    A = I.diffusion3d(13, 2.0, seed=3)
    S = P.Solver.from_host(A, k=2, **LAYOUTS[layout])
    x = I.rhs_normal(A.n, 3)
    y = to_np(S.operator(torch.as_tensor(x, device="cuda")))
    assert_close(y, A.matvec(x), 1e-13)


def test_ragged_sizes_and_tiny():
    for n in (1, 2, 63, 65, 127, 129):
        A = I.diagonal(n)
        for fmt in ("csr", "sell", "dia"):
            S = P.Solver.from_host(A, k=3, interval="given", alpha=1.0, beta=float(n) + 1.0, xi=0.0,
                                   seed_scaling=False, format=fmt)
            r = I.rhs_uniform(n, 2)
            z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
            assert_close(z, oracle_apply(A, r, 1.0, float(n) + 1.0, 0.0, 3, seed_scaling=False), APPLY_TOL)


def test_invalid_setup_reports_error():
    A = I.poisson3d(3)
    with pytest.raises(P.PolyPrecError) as ei:
        P.Solver.from_host(A, k=3, interval="given", alpha=2.0, beta=1.0)
    assert ei.value.status == P.PP_EINVAL
    B = I.dense_to_csr(np.diag([1.0, -1.0, 2.0]))
    with pytest.raises(P.PolyPrecError):
        P.Solver.from_host(B, k=3)


def test_dia_rejects_unsymmetric_and_missing_diagonal():
    D = I.poisson3d(4).to_dense()
    D[0, 1] = -0.9  # a(0,1) != a(1,0)
    with pytest.raises(P.PolyPrecError) as ei:
        P.Solver.from_host(I.dense_to_csr(D), k=3, format="dia")
    assert ei.value.status == P.PP_EUNSUPPORTED
    E = np.diag([2.0, 2.0, 2.0])
    E[0, 1] = E[1, 0] = -1.0
    A = I.dense_to_csr(E)
    S = P.Solver.from_host(A, k=2, format="dia", interval="given", alpha=0.5, beta=3.5)
    assert S.info()["format"] == 3 and S.info()["ndiag"] == 1  # Jacobi: the unit diagonal is not stored
    S = P.Solver.from_host(A, k=2, format="dia", interval="given", alpha=0.5, beta=3.5, seed_scaling=False)
    assert S.info()["ndiag"] == 2


def test_dia_diagonals_for_the_7_point_stencil():
    """Jacobi-scaled: the diagonal is 1 by construction and only the upper
    diagonals (1, N, N^2) are stored; unscaled: the main diagonal too."""
    A = I.diffusion3d(17, 2.0, seed=5)
    x = I.rhs_normal(A.n, 6)
    for scaling, nd in ((True, 3), (False, 4)):
        S = P.Solver.from_host(A, k=5, format="dia", seed_scaling=scaling, interval="given", alpha=0.05,
                               beta=14.0 if not scaling else 1.95)
        info = S.info()
        assert info["format"] == 3 and info["ndiag"] == nd
        assert_close(to_np(S.operator(torch.as_tensor(x, device="cuda"))), A.matvec(x), 1e-13)


@pytest.mark.parametrize("N", [16, 17, 18, 20])
@pytest.mark.parametrize("k", [1, 6])
def test_dia_partner_paths(N, k):
    """Grid sizes whose offsets N, N^2 are (16, 20), are not (17) or are only
    for pairs of rows (18) multiples of the rows per thread: aligned vector,
    scalar and shuffle partner paths of the DIA kernel, FP64 (2 rows per
    thread) against the oracle."""
    A = I.diffusion3d(N, 2.0, seed=N)
    S = P.Solver.from_host(A, k=k, interval="given", alpha=0.05, beta=1.95, xi=1e-3, format="dia")
    r = I.rhs_normal(A.n, 8)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    assert_close(z, oracle_apply(A, r, 0.05, 1.95, 1e-3, k), APPLY_TOL)
    x = I.rhs_normal(A.n, 9)
    assert_close(to_np(S.operator(torch.as_tensor(x, device="cuda"))), A.matvec(x), 1e-13)


def mixed_width_matrix(N=12, seed=9):
    """7-point diffusion matrix with extra symmetric couplings on a few
    scattered rows: their slices are 8-10 entries wide (wider than the TMA
    staging buffer, so loaded directly) while every other slice is at most
    7 wide (staged), and the staged/direct paths alternate along a warp's
    slice sequence."""
    A = I.diffusion3d(N, 1.5, seed=seed)
    D = A.to_dense()
    rng = np.random.default_rng(seed)
    rows = rng.choice(A.n, size=12, replace=False)
    for i in rows:
        for j in rng.choice(A.n, size=3, replace=False):
            if j != i:
                D[i, j] = D[j, i] = -0.05
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 0.5)
    return I.dense_to_csr(D)


@pytest.mark.parametrize("C", [32, 64, 128])
@pytest.mark.parametrize("sigma", [0, 256])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tma_mixed_staged_and_direct_slices(C, sigma, prec):
    A = mixed_width_matrix()
    S = P.Solver.from_host(A, k=6, interval="given", alpha=0.05, beta=1.95, xi=1e-3, format="sell", sell_C=C,
                           sell_sigma=sigma, sell_variant=2, apply_prec=prec)
    r = I.rhs_normal(A.n, 3)
    z = to_np(S.apply(torch.as_tensor(r, device="cuda")))
    if prec == "f64":
        assert_close(z, oracle_apply(A, r, 0.05, 1.95, 1e-3, 6), APPLY_TOL)
    else:
        import oracle as O

        vh, w = O.jacobi_scale(A)
        ref = w * O.cheb_apply(A, 0.05, 1.95, 1e-3, 6, w * r, val=vh.astype(np.float32).astype(np.float64))
        assert_close(z, ref, 2e-5)
