"""Pins of the oracle's low-rank acceleration (Section 3.1) and of the
Lanczos run that supplies its vectors.  CPU only.

What fixes each result independently of the oracle's own code:
  * the Lanczos relation: Q^T Q = I, Q^T A Q = T_m, and the residual of the
    last step has norm beta_m; n steps reproduce the whole spectrum;
  * eigenpairs of the tridiagonal T_m agree with LAPACK (numpy.linalg.eigh);
  * for exact eigenvectors V the preconditioned spectrum is the plain
    one with the p smallest images raised by one (Section 3.1);
  * P depends on span(V) only (V -> V R) and is symmetric positive definite;
  * the work counts of Table 4 (right block): ddot = (3 + p) iter,
    MVP = (m + 1) iter;
  * Lanczos on p_k(A) A returns the leftmost eigenpairs of A (LAPACK).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2208_01339_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _spd_with_eigenvectors(n, seed, lo=1e-3, hi=1.0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), n)))
    A = (U * d) @ U.T
    A = 0.5 * (A + A.T)
    return I.dense_to_csr(A), d, U


def test_lanczos_basis_relation():
    A = I.diffusion3d(6, 1.5, seed=3)
    vh, _ = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh)
    D = Ah.to_dense()
    a, b, Q = O.lanczos_basis(Ah, I.lanczos_start(A.n, 0), 30)
    m = len(a)
    assert m == 30
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    np.testing.assert_allclose(Q.T @ D @ Q, T, atol=1e-12)
    # A Q = Q T + beta_m q_{m+1} e_m^T: the residual lives in the last column
    R = D @ Q - Q @ T
    assert np.linalg.norm(R[:, :-1]) < 1e-12
    assert np.linalg.norm(R[:, -1]) == pytest.approx(b[-1], rel=1e-10)
    # plain three-term Lanczos agrees on T while orthogonality holds
    a0, b0 = O.lanczos(Ah, I.lanczos_start(A.n, 0), 10)
    np.testing.assert_allclose(a[:10], a0, rtol=1e-10)
    np.testing.assert_allclose(b[:9], b0, rtol=1e-10)


def test_lanczos_basis_full_run_gives_spectrum():
    A, d, _ = _spd_with_eigenvectors(24, seed=4)
    a, b, _ = O.lanczos_basis(A, I.lanczos_start(24, 1), 24)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    np.testing.assert_allclose(np.linalg.eigvalsh(T), d, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tridiag_eig_matches_lapack(seed):
    rng = np.random.default_rng(seed)
    m = 25
    a = rng.uniform(0, 4, m)
    b = rng.uniform(0.1, 1.0, m - 1)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    w, S = np.linalg.eigh(T)
    for i in range(m):
        lam, y = O.tridiag_eig(a, b, i)
        assert lam == pytest.approx(w[i], abs=1e-12 * np.abs(w).max())
        assert abs(abs(y @ S[:, i]) - 1.0) < 1e-10
        assert np.linalg.norm(T @ y - lam * y) < 1e-11
        assert np.abs(y).max() == pytest.approx(y.max())  # sign convention


def test_ritz_residual_estimate():
    """||A (Q y) - theta Q y|| = beta_m |y_m| for every Ritz pair."""
    A = I.diffusion3d(6, 2.0, seed=5)
    vh, _ = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh)
    a, b, Q = O.lanczos_basis(Ah, I.lanczos_start(A.n, 2), 40)
    for i in (0, 1, 2, 39):
        th, y = O.tridiag_eig(a, b[:-1], i)
        v = Q @ y
        res = np.linalg.norm(O.spmv(Ah, v) - th * v)
        assert res == pytest.approx(b[-1] * abs(y[-1]), rel=1e-6, abs=1e-13)


def _dense_prec(A, alpha, beta, xi, k, V):
    return np.column_stack([O.lowrank_apply(A, alpha, beta, xi, k, V, e) for e in np.eye(A.n)])


@pytest.mark.parametrize("p", [1, 3])
def test_exact_eigenvectors_raise_smallest_images_by_one(p):
    """Section 3.1: with V = the p leftmost eigenvectors, P A v_j =
    (lambda_j p_k(lambda_j) + 1) v_j for j <= p and the rest is unchanged."""
    n, k, xi = 30, 5, 1e-3
    A, d, U = _spd_with_eigenvectors(n, seed=6)
    P = _dense_prec(A, d[0], d[-1], xi, k, U[:, :p])
    got = np.sort(np.linalg.eigvals(P @ A.to_dense()).real)
    img = np.array([lam * O.cheb_poly(lam, d[0], d[-1], xi, k) for lam in d])
    img[:p] += 1.0
    np.testing.assert_allclose(got, np.sort(img), rtol=1e-9, atol=1e-12)


def test_correction_depends_on_span_only_and_is_spd():
    n, k = 30, 4
    A, d, U = _spd_with_eigenvectors(n, seed=7)
    rng = np.random.default_rng(8)
    V = rng.standard_normal((n, 3))  # any full-rank V, not only eigenvectors
    R = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    r = rng.standard_normal(n)
    z1 = O.lowrank_apply(A, d[0], d[-1], 1e-3, k, V, r)
    z2 = O.lowrank_apply(A, d[0], d[-1], 1e-3, k, V @ R, r)
    np.testing.assert_allclose(z1, z2, rtol=1e-11, atol=1e-12 * np.abs(z1).max())
    z0 = O.cheb_apply(A, d[0], d[-1], 1e-3, k, r)
    Ad = A.to_dense()
    corr = V @ np.linalg.solve(V.T @ Ad @ V, V.T @ r)  # the definition, by LAPACK
    np.testing.assert_allclose(z1 - z0, corr, rtol=1e-9, atol=1e-12 * np.abs(corr).max())
    P = _dense_prec(A, d[0], d[-1], 1e-3, k, V)
    assert np.abs(P - P.T).max() < 1e-10 * np.abs(P).max()
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0


def test_pcg_lowrank_solution_and_table4_work_counts():
    rows = np.loadtxt(os.path.join(GOLDEN, "table4_rank_one.txt"))
    for m, it, mvp, ddot, flag in rows:
        assert mvp == it * (m + 1)
        assert (ddot == 4 * it) == (flag == 0)
    A = I.diffusion3d(7, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    v0 = I.lanczos_start(A.n, 0)
    xd = np.linalg.solve(A.to_dense(), b)
    for p in (1, 4):
        x, st = O.pcg_csr(A, b, v0=v0, k=3, xi=1e-3, rtol=1e-12, lanczos_steps=30, lowrank=p)
        assert st["status"] == 0
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
        assert st["mvp"] == st["iterations"] * 4
        assert st["dots"] == (3 + p) * st["iterations"]


def test_rank_one_reduces_iterations_when_leftmost_is_isolated():
    """Table 4 (right): the rank-one correction with the leftmost eigenpair
    cuts iterations.  Here lambda_1 is isolated (A = diag(1e-3, 0.1..1))
    and its eigenvector is exact after enough Lanczos steps."""
    n = 200
    dvals = np.concatenate([[1e-3], np.linspace(0.1, 1.0, n - 1)])
    A = I.dense_to_csr(np.diag(dvals))
    b = I.rhs_uniform(n, 0)
    v0 = I.lanczos_start(n, 3)
    common = dict(k=3, xi=1e-3, rtol=1e-10, seed_scaling=False, interval="given", alpha=1e-3, beta=1.0)
    _, s0 = O.pcg_csr(A, b, v0=v0, **common)
    V = np.zeros((n, 1))
    V[0, 0] = 1.0
    x1, s1 = O.pcg_csr(A, b, v0=v0, lr_V=V, **common)
    assert s1["status"] == 0 and s0["status"] == 0
    assert s1["iterations"] < s0["iterations"]
    # the same vector found by Lanczos on p_k(A) A (40 steps)
    _, s2 = O.pcg_csr(A, b, v0=v0, lowrank_steps=40, lowrank=1, **common)
    assert s2["iterations"] <= s1["iterations"] + 1


def test_lowrank_vectors_are_leftmost_eigenvectors():
    """Lanczos on B = p_k(A) A finds the leftmost eigenpairs of A: B is a
    polynomial in A (same eigenvectors) that keeps the smallest eigenvalues
    of A smallest (Theorem 2.3).  Checked against LAPACK eigenpairs; using
    p_k(A) alone (decreasing in lambda) would return the rightmost ones."""
    A = I.diffusion3d(10, 2.0, seed=1)
    vh, _ = O.jacobi_scale(A)
    Ah = I.CSR(A.n, A.rowptr, A.col, vh)
    D = Ah.to_dense()
    ev, E = np.linalg.eigh(D)
    a, b = O.lanczos(Ah, I.lanczos_start(A.n, 0), 10)
    lo, hi = O.tridiag_extremes(a, b)
    V, th = O.lowrank_vectors(Ah, I.lanczos_start(A.n, 0), lo, hi, 1e-3, 8, 2, 30)
    np.testing.assert_allclose(th, ev[:2], rtol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(2), atol=1e-12)
    for i in range(2):
        assert np.linalg.norm(D @ V[:, i] - th[i] * V[:, i]) <= 1e-9 * th[i]
        assert abs(abs(V[:, i] @ E[:, i]) - 1.0) < 1e-10
    # plain Lanczos with the same number of steps is far from converged
    a2, b2, Q = O.lanczos_basis(Ah, I.lanczos_start(A.n, 0), 30)
    t0, y0 = O.tridiag_eig(a2, b2[:-1], 0)
    v = Q @ y0
    assert np.linalg.norm(D @ v - t0 * v) > 1e3 * np.linalg.norm(D @ V[:, 0] - th[0] * V[:, 0])


def test_correction_keeps_interval():
    """The interval comes from the estimator alone; the correction adds
    (3 + p) - 3 = p inner products per iteration and nothing else."""
    A = I.diffusion3d(10, 2.0, seed=1)
    b = I.rhs_normal(A.n, 1)
    _, s0 = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=8, rtol=1e-10)
    _, s1 = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=8, rtol=1e-10, lowrank=2, lowrank_steps=30)
    assert (s1["alpha_hat"], s1["beta_hat"], s1["xi"]) == (s0["alpha_hat"], s0["beta_hat"], s0["xi"])
    assert s1["status"] == 0 and s1["iterations"] <= s0["iterations"]
