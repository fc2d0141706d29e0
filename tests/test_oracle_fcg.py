"""Pins of the oracle's truncated flexible CG, FCG(m) (the outer iteration
of the mixed-precision solver), independent of its own code:
  * the last m directions are A-orthogonal, whatever the preconditioner;
  * with the full window (m >= n) and a nonsymmetric preconditioner the
    solve terminates in at most n iterations (A-orthogonal directions span
    R^n), checked against LAPACK's solution;
  * with a fixed SPD preconditioner FCG(m) reproduces plain PCG (equal in
    exact arithmetic), for m = 2, 4 against the oracle's PCG and a dense
    solve.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_01339_gb300 import inputs as I


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.exp(np.linspace(0.0, np.log(cond), n))
    return (U * d) @ U.T


@pytest.mark.parametrize("m", [2, 3, 5])
def test_last_m_directions_are_A_orthogonal(m):
    n = 40
    A = _spd(n, 1)
    rng = np.random.default_rng(2)
    M = np.linalg.inv(A + 0.3 * np.eye(n)) + 0.05 * rng.standard_normal((n, n)) / n  # nonsymmetric
    b = rng.standard_normal(n)
    _, D, st = O.fcg_dense(A, M, b, m, maxit=25, rtol=0.0)
    assert len(D) >= 20
    An = np.sqrt(np.einsum("ij,jk,ik->i", D, A, D))
    for i in range(len(D)):
        for j in range(max(0, i - m), i):
            assert abs(D[i] @ A @ D[j]) <= 1e-9 * An[i] * An[j], (i, j)
    # directions further apart than m are not orthogonal in general
    far = [abs(D[i] @ A @ D[i - m - 2]) / (An[i] * An[i - m - 2]) for i in range(m + 2, len(D))]
    assert max(far) > 1e-6


def test_full_window_terminates_with_nonsymmetric_preconditioner():
    n = 12
    A = _spd(n, 3, cond=1e4)
    rng = np.random.default_rng(4)
    M = np.eye(n) + 0.4 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x, _, st = O.fcg_dense(A, M, b, m=n, maxit=n, rtol=1e-12)
    assert st["iterations"] <= n
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-8 * np.linalg.norm(np.linalg.solve(A, b))


@pytest.mark.parametrize("m", [2, 4])
def test_fcg_m_equals_pcg_for_fixed_spd_preconditioner(m):
    A = I.diffusion3d(8, 1.5, seed=2)
    b = I.rhs_normal(A.n, 1)
    v0 = I.lanczos_start(A.n, 0)
    x0, s0 = O.pcg_csr(A, b, v0=v0, k=6, rtol=1e-11)
    xm, sm = O.pcg_csr(A, b, v0=v0, k=6, rtol=1e-11, flexible=m)
    assert s0["status"] == 0 and sm["status"] == 0
    assert abs(s0["iterations"] - sm["iterations"]) <= 1
    assert np.linalg.norm(xm - x0) / np.linalg.norm(x0) <= 1e-9
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(xm - xd) / np.linalg.norm(xd) <= 1e-9
    # fixed iteration count: the iterates of FCG(m) and PCG agree to rounding
    xa, _ = O.pcg_csr(A, b, v0=v0, k=6, rtol=0.0, maxit=7)
    xb, _ = O.pcg_csr(A, b, v0=v0, k=6, rtol=0.0, maxit=7, flexible=m)
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xa) <= 1e-11
