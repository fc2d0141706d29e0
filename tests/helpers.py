"""Shared helpers of the GPU parity tests (oracle references, error norms)."""
import numpy as np

import oracle as O


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


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
