"""Shared helpers of the GPU parity tests (oracle references, error norms)."""
from __future__ import annotations

import numpy as np

import oracle as O


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rel_inf(a, b) -> float:
    """Largest element error scaled by the reference's largest entry:
    max_i |a_i - b_i| / max_i |b_i|.  Unlike the 2-norm ratio it cannot hide
    a few wrong rows among many right ones."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = float(np.max(np.abs(b))) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (nb if nb > 0 else 1.0)) if a.size else 0.0


def assert_close(a, b, tol: float, elem_tol: float | None = None) -> None:
    """Parity check of a GPU result a against the oracle's b: the relative
    2-norm error <= tol and the per-element error max|a - b| / max|b| <=
    elem_tol (default tol), and no non-finite entry."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    assert np.all(np.isfinite(a)), "non-finite entries in the result"
    et = tol if elem_tol is None else elem_tol
    e2, ei = rel(a, b), rel_inf(a, b)
    assert e2 <= tol and ei <= et, f"rel 2-norm {e2:.3e} (tol {tol:.1e}), per-element {ei:.3e} (tol {et:.1e})"


def oracle_apply(A, r, alpha, beta, xi, k, seed_scaling=True):
    """Oracle z = W p_k(W^T A W) W^T r (Section 3 + Algorithm 2)."""
    if seed_scaling:
        vh, w = O.jacobi_scale(A)
    else:
        vh, w = A.val, np.ones(A.n)
    return w * O.cheb_apply(A, alpha, beta, xi, k, w * r, val=vh)


def oracle_interval(A, seed, steps, seed_scaling=True):
    """Lanczos interval of W^T A W from the shared start vector."""
    from paper_2208_01339_gb300 import inputs as I

    vh = O.jacobi_scale(A)[0] if seed_scaling else A.val
    a, b = O.lanczos(A, I.lanczos_start(A.n, seed), steps, val=vh)
    return O.tridiag_extremes(a, b)


def to_np(t):
    return t.detach().cpu().numpy()
