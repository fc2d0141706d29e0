"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these checks retypes the oracle's own formulas: each compares the
oracle with a closed form, a printed table, a theorem, a library routine
used as a step (numpy eigh/solve), or brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2208_01339_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cheb_T(n, y):
    """T_n(y) from its trigonometric / hyperbolic closed form."""
    y = np.asarray(y, dtype=np.float64)
    out = np.empty_like(y)
    inside = np.abs(y) <= 1.0
    out[inside] = np.cos(n * np.arccos(y[inside]))
    big = ~inside
    s = np.sign(y[big])
    out[big] = (s ** n) * np.cosh(n * np.arccosh(np.abs(y[big])))
    return out


# ---------------------------------------------------------------------------
# Chebyshev polynomial (Section 2.2, Eq. polycheb / rhocheb / thetamod)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 2, 3, 7, 20, 63])
@pytest.mark.parametrize("alpha,beta,xi", [(1.0, 10.0, 0.0), (0.01, 2.0, 1e-3), (3.0, 3e4, 1e-2)])
def test_residual_polynomial_closed_form(k, alpha, beta, xi):
    """1 - x p_k(x) = T_{k+1}((theta_bar - x)/delta) / T_{k+1}(sigma_bar)."""
    c = O.cheb_coeffs(alpha, beta, xi, k)
    theta = 0.5 * (alpha + beta)
    delta = 0.5 * (beta - alpha)
    assert c.theta_bar == pytest.approx(theta * (1 + xi), rel=1e-15)
    assert c.delta == pytest.approx(delta, rel=1e-15)
    xs = np.concatenate([np.linspace(alpha, beta, 41), [0.5 * alpha, 1.5 * beta]])
    got = np.array([1.0 - x * O.cheb_poly(x, alpha, beta, xi, k) for x in xs])
    want = cheb_T(k + 1, (c.theta_bar - xs) / c.delta) / cheb_T(k + 1, np.array([c.sigma_bar]))[0]
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("k", [1, 4, 15, 40])
def test_equioscillation_extrema(k):
    """x p_k(x) = 1 - (-1)^j / T_{k+1}(sigma_bar) at x_j = theta_bar - delta cos(j pi/(k+1))."""
    alpha, beta, xi = 0.05, 2.0, 2e-3
    c = O.cheb_coeffs(alpha, beta, xi, k)
    j = np.arange(k + 2)
    xj = c.theta_bar - c.delta * np.cos(j * np.pi / (k + 1))
    t = cheb_T(k + 1, np.array([c.sigma_bar]))[0]
    got = np.array([x * O.cheb_poly(x, alpha, beta, xi, k) for x in xj])
    np.testing.assert_allclose(got, 1.0 - (-1.0) ** j / t, rtol=1e-10, atol=1e-13)


def test_rho_closed_form():
    """rho_j = T_j(sigma_bar) / T_{j+1}(sigma_bar) (follows from Eq. rhocheb)."""
    c = O.cheb_coeffs(0.2, 3.0, 1e-3, 30)
    j = np.arange(31)
    s = np.array([c.sigma_bar])
    want = np.array([cheb_T(i, s)[0] / cheb_T(i + 1, s)[0] for i in j])
    np.testing.assert_allclose(c.rho, want, rtol=1e-12)


def test_coeffs_reject_bad_interval():
    with pytest.raises(ValueError):
        O.cheb_coeffs(2.0, 1.0, 0.0, 3)
    with pytest.raises(ValueError):
        O.cheb_coeffs(0.0, 1.0, 0.0, 3)


# ---------------------------------------------------------------------------
# Algorithm 2 on matrices: spectral mapping, symmetry and positivity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 2, 5, 16])
def test_apply_spectral_mapping_dense(k):
    """p_k(A) built column by column from Algorithm 2 equals V p_k(Lam) V^T,
    is symmetric, and p_k(A) A is positive definite (eigenvalues in (0,2))."""
    n = 14
    D = I.random_spd(n, seed=11 + k, cond=50.0)
    A = I.dense_to_csr(D)
    lam, V = np.linalg.eigh(D)
    alpha, beta, xi = lam[0], lam[-1], 1e-3
    P = np.column_stack([O.cheb_apply(A, alpha, beta, xi, k, e) for e in np.eye(n)])
    np.testing.assert_allclose(P, P.T, atol=1e-12 * np.abs(P).max())
    c = O.cheb_coeffs(alpha, beta, xi, k)
    s = np.array([c.sigma_bar])
    resid = cheb_T(k + 1, (c.theta_bar - lam) / c.delta) / cheb_T(k + 1, s)[0]
    p_of_lam = (1.0 - resid) / lam
    np.testing.assert_allclose(P, (V * p_of_lam) @ V.T, rtol=1e-9, atol=1e-11 * np.abs(P).max())
    mu = np.linalg.eigvalsh(0.5 * ((P @ D) + (P @ D).T))
    assert mu.min() > 0.0 and mu.max() < 2.0


def test_apply_indefinite_when_interval_too_small():
    """With odd k the residual polynomial T_{k+1} is even and grows without
    bound, so p_k(A) A turns negative once lambda_max(A) lies well beyond
    2 theta_bar: the breakdown case a solver must report."""
    n = 10
    D = np.diag(np.linspace(1.0, 10.0, n))
    A = I.dense_to_csr(D)
    P = np.column_stack([O.cheb_apply(A, 1.0, 4.0, 0.0, 3, e) for e in np.eye(n)])
    assert np.linalg.eigvalsh(P @ D).min() < 0.0


def test_table1_eigenvalues_and_iterations():
    """Table 1: diagonal A_ii = i, n = 1e5, degree 63, tol 1e-10."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1.txt"))
    n = 100000
    A = I.diagonal(n)
    b = I.rhs_uniform(n, 0)
    for xi, iters, l1, l2, l5, l10, kap, kap10 in rows:
        z = O.cheb_apply(A, 1.0, float(n), xi, 63, np.ones(n))
        lam = np.sort(np.arange(1, n + 1) * z)
        lm = lam[-1]
        got = lam[[0, 1, 4, 9]] / lm
        np.testing.assert_allclose(got, [l1, l2, l5, l10], atol=1.01e-5)
        k_tol = 5e-4 if xi != 1e-2 else 1e-3
        assert lm / lam[0] == pytest.approx(kap, rel=k_tol)
        if xi == 0.0:
            assert lm / lam[9] == pytest.approx(lm / lam[0], rel=1e-5)  # printed 25.83 is a typo
        else:
            assert lm / lam[9] == pytest.approx(kap10, rel=1e-3)
        x, st = O.pcg_csr(A, b, k=63, xi=float(xi), interval="given", alpha=1.0, beta=float(n),
                          seed_scaling=False, rtol=1e-10)
        assert st["status"] == 0
        assert st["iterations"] == int(iters)
        assert st["mvp"] == st["iterations"] * 64
        assert st["dots"] == 3 * st["iterations"]


# ---------------------------------------------------------------------------
# Algorithm 1 (Newton) == Algorithm 2 at degree 2^nlev - 1 (Eq. T2k)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nlev", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("xi", [0.0, 1e-3])
def test_newton_equals_chebyshev(nlev, xi):
    A = I.diffusion3d(6, 1.0, seed=3)
    vh, _ = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh)
    r = I.rhs_normal(A.n, 5)
    lam = np.linalg.eigvalsh(Ah.to_dense())
    zn = O.newton_apply(Ah, lam[0], lam[-1], xi, nlev, r)
    zc = O.cheb_apply(Ah, lam[0], lam[-1], xi, 2 ** nlev - 1, r)
    np.testing.assert_allclose(zn, zc, rtol=1e-10, atol=1e-12 * np.abs(zc).max())


# ---------------------------------------------------------------------------
# Theorems 2.2 and 2.3 (first Newton/Chebyshev level, degree 1)
# ---------------------------------------------------------------------------

def test_theorem_2_2_condition_number_growth():
    """kappa_eta / kappa = 1 + xi + O(xi^2) for xi = O(1/kappa)."""
    alpha, beta = 1.0, 1e4
    xs = np.array([alpha, beta])

    def kappa(xi):
        v = np.array([x * O.cheb_poly(x, alpha, beta, xi, 1) for x in xs])
        m = np.max([x * O.cheb_poly(x, alpha, beta, xi, 1) for x in np.linspace(alpha, beta, 2001)])
        return m / v.min()

    k0 = kappa(0.0)
    for xi in (1e-5, 1e-4, 5e-4):
        ratio = kappa(xi) / k0
        assert abs(ratio - (1.0 + xi)) < 10.0 * xi * xi + 2.0 * xi / k0


@pytest.mark.parametrize("xi", [0.0, 0.05])
def test_theorem_2_3_unclustering_figure1(xi):
    """Figure 1: eigenvalues 0.1, 0.14, 0.18 ... 1.82, 1.86, 1.9 (theta = 1).
    With xi = 0 the ends fold onto the same smallest eigenvalues of P_1 A;
    with xi = 0.05 the three smallest eigenvalues of P_1 A are the images of
    0.1, 0.14, 0.18 in order (Theorem 2.3, threshold alpha_hat_eta + 2(1-eta))."""
    lam = np.array([0.1, 0.14, 0.18, 0.5, 1.0, 1.5, 1.82, 1.86, 1.9])
    alpha, beta = 0.1, 1.9
    mu = np.array([x * O.cheb_poly(x, alpha, beta, xi, 1) for x in lam])
    if xi == 0.0:
        np.testing.assert_allclose(mu[[0, 1, 2]], mu[[8, 7, 6]], rtol=1e-12)
    else:
        eta = 1.0 / (1.0 + xi)
        thr = eta * alpha + 2.0 * (1.0 - eta)
        assert np.all(eta * lam[:3] <= thr)
        order = np.argsort(mu)
        assert list(order[:3]) == [0, 1, 2]
        assert mu[6:].min() > mu[2]


# ---------------------------------------------------------------------------
# Lanczos + Sturm bisection (interval estimate)
# ---------------------------------------------------------------------------

def test_sturm_matches_eigvalsh():
    a = I.uniform(1, 9, 12) * 4.0
    b = I.uniform(2, 9, 11) + 0.1
    lo, hi = O.tridiag_extremes(a, b)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ev = np.linalg.eigvalsh(T)
    assert lo == pytest.approx(ev[0], abs=1e-12)
    assert hi == pytest.approx(ev[-1], abs=1e-12)


def test_lanczos_interlacing_and_poisson_closed_form():
    N = 6
    A = I.poisson3d(N)
    v0 = I.lanczos_start(A.n, 0)
    exact_min = 3 * (2 - 2 * np.cos(np.pi / (N + 1)))
    exact_max = 3 * (2 + 2 * np.cos(np.pi / (N + 1)))
    a, b = O.lanczos(A, v0, 10)
    lo, hi = O.tridiag_extremes(a, b)
    assert exact_min - 1e-12 <= lo <= hi <= exact_max + 1e-12
    a, b = O.lanczos(A, v0, 120)
    lo, hi = O.tridiag_extremes(a, b)
    assert lo == pytest.approx(exact_min, rel=1e-8)
    assert hi == pytest.approx(exact_max, rel=1e-8)


def test_lanczos_tridiagonal_is_projection():
    """T_m = V_m^T A V_m for the Lanczos basis (checked through its
    eigenvalues: Ritz values interlace the dense spectrum)."""
    D = I.random_spd(30, seed=4, cond=1e3)
    A = I.dense_to_csr(D)
    lam = np.linalg.eigvalsh(D)
    a, b = O.lanczos(A, I.lanczos_start(30, 1), 8)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ritz = np.linalg.eigvalsh(T)
    assert lam[0] - 1e-9 <= ritz[0] and ritz[-1] <= lam[-1] + 1e-9
    # Cauchy interlacing: k-th Ritz value >= k-th eigenvalue, <= (n-m+k)-th
    m = len(ritz)
    for kk in range(m):
        assert lam[kk] - 1e-9 <= ritz[kk] <= lam[30 - m + kk] + 1e-9


def test_jacobi_scaling_unit_diagonal():
    A = I.diffusion3d(5, 2.0, seed=1)
    vh, w = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh).to_dense()
    np.testing.assert_allclose(np.diag(Ah), 1.0, rtol=1e-14)
    np.testing.assert_allclose(w, 1.0 / np.sqrt(np.diag(A.to_dense())), rtol=1e-15)
    np.testing.assert_allclose(Ah, Ah.T, atol=1e-15)


# ---------------------------------------------------------------------------
# PCG (Section 1) against dense solves; Table 4 work model
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 3, 10])
def test_pcg_matches_dense_solve(k):
    D = I.random_spd(40, seed=21, cond=300.0)
    A = I.dense_to_csr(D)
    b = I.rhs_normal(40, 3)
    x, st = O.pcg_csr(A, b, v0=I.lanczos_start(40, 0), k=k, lanczos_steps=40, rtol=1e-13, maxit=1000)
    assert st["status"] == 0
    xd = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert st["mvp"] == st["iterations"] * (k + 1)
    assert st["dots"] == 3 * st["iterations"]


def test_work_model_table4():
    rows = np.loadtxt(os.path.join(GOLDEN, "table4_counts.txt"))
    for m, it, mvp, ddot in rows:
        assert mvp == it * (m + 1) and ddot == 3 * it
    A = I.diffusion3d(8, 1.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    for m in (0, 1, 3, 7, 15):
        _, st = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=m, xi=1e-3, rtol=1e-8)
        assert st["mvp"] == st["iterations"] * (m + 1)
        assert st["dots"] == 3 * st["iterations"]


def test_flexible_cg_matches_plain_for_fixed_spd_preconditioner():
    A = I.diffusion3d(8, 1.5, seed=2)
    b = I.rhs_normal(A.n, 1)
    x1, s1 = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=6, rtol=1e-10)
    x2, s2 = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=6, rtol=1e-10, flexible=True)
    assert abs(s1["iterations"] - s2["iterations"]) <= 1
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-8


def test_breakdown_reported_for_bad_interval():
    """beta far below lambda_max makes p_k(A) A indefinite: status -2 (or the
    solve fails to converge), never a silent wrong answer."""
    A = I.diagonal(200)
    b = I.rhs_uniform(200, 0)
    _, st = O.pcg_csr(A, b, k=3, interval="given", alpha=1.0, beta=20.0, xi=0.0, seed_scaling=False,
                      rtol=1e-10, maxit=50)
    assert st["status"] in (-2, 1)


def test_true_residual_reported():
    A = I.poisson3d(10)
    b = I.rhs_ones_plus_noise(A, 0)
    x, st = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=8, rtol=1e-10)
    assert st["status"] == 0
    r = b - A.matvec(x)
    assert st["true_rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-6)
    assert st["true_rel_res"] < 1e-9
