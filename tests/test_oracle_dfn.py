"""Pins of the oracle's Schur-complement path (Section 4.2) to dense algebra.

The dense references below are built from the block definitions with
numpy (inverse, solve, eigvalsh as library steps): the expansion of S_u,
its diagonal, the right-hand side r = W^T M^{-1} f_1 and the full 3x3
saddle-point system K_0 x = f_0 (Eq. sys).
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_01339_gb300 import inputs as I


def small_net(seed=5):
    return I.fracture_network(n_f=8, side_min=1.5, side_max=4.0, h=0.25, trace_min=0.5, trace_max=2.0,
                              trace_fraction=0.1, seed=seed)


def dense_blocks(net):
    A = net.A.to_dense()
    C = net.C.to_dense()
    B = net.B.to_dense()
    Gh = net.Gh.to_dense()
    Gu = net.Gu.to_dense()
    return A, C, B, Gh, Gu


def dense_schur(net):
    A, C, B, Gh, Gu = dense_blocks(net)
    Ai = np.linalg.inv(A)
    a = net.alpha
    return Gu - a * B.T @ Ai @ C - a * C.T @ Ai @ B + C.T @ Ai @ Gh @ Ai @ C


NETS = {
    "tiny": lambda: I.tiny_fracture_network(),
    "small5": lambda: small_net(5),
    "small9": lambda: small_net(9),
    # general fracture blocks: P1 stiffness on jittered triangulations with
    # lognormal coefficients, nodes renumbered at random; and one dense block
    "p1_tiny": lambda: I.general_fracture_network(I.tiny_fracture_network(), seed=3),
    "p1_small5": lambda: I.general_fracture_network(small_net(5)),
    "dense_small9": lambda: I.with_dense_block(small_net(9), 2),
}


@pytest.fixture(scope="module", params=list(NETS))
def net(request):
    return NETS[request.param]()


def test_block_properties(net):
    A, C, B, Gh, Gu = dense_blocks(net)
    # A SPD and block diagonal by fracture
    assert np.linalg.eigvalsh(A).min() > 0
    off = net.offset
    for f in range(net.n_f):
        blk = np.zeros_like(A, dtype=bool)
        blk[off[f]:off[f + 1], off[f]:off[f + 1]] = True
        assert np.all(A[~blk][:0] == 0)
    mask = np.zeros_like(A, dtype=bool)
    for f in range(net.n_f):
        mask[off[f]:off[f + 1], off[f]:off[f + 1]] = True
    assert np.all(A[~mask] == 0)
    # C has distinct unit columns, E = B - C is zero where C is nonzero
    assert np.all(C.sum(axis=0) == 1) and np.all(C.sum(axis=1) <= 1)
    E = B - C
    assert np.all(E[C != 0] == 0) and np.all(E >= 0)
    # G^h and G^u symmetric positive semidefinite, rank deficient
    for G in (Gh, Gu):
        assert np.allclose(G, G.T)
        ev = np.linalg.eigvalsh(G)
        assert ev.min() > -1e-12
        assert np.linalg.matrix_rank(G) < G.shape[0]


def test_ainv_matches_dense_solve(net):
    S = O.Schur(net)
    A = net.A.to_dense()
    v = I.rhs_normal(net.n_h, 3)
    np.testing.assert_allclose(S.ainv(v), np.linalg.solve(A, v), rtol=1e-11, atol=1e-12)


def test_alg3_matches_expansion(net):
    """Algorithm 3 column by column equals the expansion of S_u."""
    S = O.Schur(net)
    Sd = dense_schur(net)
    cols = np.column_stack([S.apply(e) for e in np.eye(net.n_u)])
    np.testing.assert_allclose(cols, Sd, rtol=1e-10, atol=1e-12 * np.abs(Sd).max())
    np.testing.assert_allclose(cols, cols.T, atol=1e-12 * np.abs(Sd).max())


def test_su_spd_for_half_alpha(net):
    """With alpha = 1/2 the synthetic S_u is SPD (B^T B = 2 G^u here, so
    S_u = (1 - 2 alpha^2) G^u + (G^h A^{-1} C - alpha B)^T (...))."""
    Sd = dense_schur(net)
    assert np.linalg.eigvalsh(0.5 * (Sd + Sd.T)).min() > 0


def test_alg4_diag(net):
    S = O.Schur(net)
    np.testing.assert_allclose(S.diag(), np.diag(dense_schur(net)), rtol=1e-11)


def test_rhs_matches_block_elimination(net):
    A, C, B, Gh, Gu = dense_blocks(net)
    Ai = np.linalg.inv(A)
    r = net.alpha * B.T @ Ai @ net.q - C.T @ Ai @ Gh @ Ai @ net.q
    np.testing.assert_allclose(O.Schur(net).rhs(net.q), r, rtol=1e-10, atol=1e-12 * np.abs(r).max())


def test_schur_solve_and_recovery_match_K0(net):
    """PCG on the D_S-scaled S_u plus the recovery of h and p solves the full
    saddle-point system K_0 [h; u; p] = [0; 0; q] (Eq. sys)."""
    A, C, B, Gh, Gu = dense_blocks(net)
    a = net.alpha
    nh, nu = net.n_h, net.n_u
    K0 = np.block([[Gh, -a * B, A], [-a * B.T, Gu, -C.T], [A, -C, np.zeros((nh, nh))]])
    f0 = np.concatenate([np.zeros(nh), np.zeros(nu), net.q])
    sol = np.linalg.solve(K0, f0)
    h_ref, u_ref, p_ref = sol[:nh], sol[nh:nh + nu], sol[nh + nu:]
    S = O.Schur(net)
    r = S.rhs(net.q)
    u, st = S.pcg(S.diag(), r, v0=I.lanczos_start(nu, 0), k=6, lanczos_steps=nu, rtol=1e-13, maxit=2000)
    assert st["status"] == 0
    h, p = S.recover(net.q, u)
    for got, ref in ((u, u_ref), (h, h_ref), (p, p_ref)):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9


def test_general_blocks_are_general():
    """The general blocks leave the rectangle form: obtuse triangles give
    positive off-diagonal entries, rows have up to 9 entries, and the random
    numbering spreads each block over its whole index range."""
    base = small_net(5)
    g = I.general_fracture_network(base)
    A = g.A.to_dense()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    off = ~np.eye(g.n_h, dtype=bool)
    assert (A[off] > 0).any() and np.diff(g.A.rowptr).max() > 5
    rows = np.repeat(np.arange(g.n_h), np.diff(g.A.rowptr))
    assert np.abs(rows - g.A.col).max() > 4 * int(np.minimum(base.nx, base.ny).max())
    # the numbering is a relabelling: S_u is unchanged by it
    unshuffled = I.general_fracture_network(base, shuffle=False)
    np.testing.assert_allclose(dense_schur(g), dense_schur(unshuffled), rtol=0, atol=1e-12 * np.abs(dense_schur(g)).max())
