"""GPU parity of the Schur path with general fracture blocks (Section 4.2
with the exact Cholesky factor of A): A is handed to the library as CSR,
each block is reordered and factored as a band matrix on the GPU, and the
trace blocks M_f and the full solves come from that factor.

Against the FP64 oracle (banded Cholesky in the given numbering, Algorithms
3 and 4 as printed): relative 2-norm 1e-11 for A^{-1}, S_u r, diag(S_u),
the right-hand side and the recovery (the two sides factor in different
orders); PCG on S_hat: same iteration count, solution within 1e-9.  On
rectangles the factor path must agree with the closed-form path to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from helpers import assert_close, rel, to_np
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")

TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small(seed=5):
    return I.fracture_network(n_f=8, side_min=1.5, side_max=4.0, h=0.25, trace_min=0.5, trace_max=2.0,
                              trace_fraction=0.1, seed=seed)


def medium():
    return I.fracture_network(n_f=24, side_min=3.0, side_max=9.0, h=0.25, trace_min=1.0, trace_max=6.0,
                              trace_fraction=0.06, T_sigma=1.0, seed=9)


def wide_block_fracture(net):
    """A fracture with 240..768 nodes: dense, its band (n_f - 1 wide) needs
    the factor window in global memory."""
    sizes = np.diff(net.offset)
    ok = np.nonzero((sizes >= 240) & (sizes <= 768))[0]
    assert ok.size, sizes
    return int(ok[0])


NETS = {
    "rect_small": lambda: small(),
    "p1_tiny": lambda: I.general_fracture_network(I.tiny_fracture_network(), seed=3),
    "p1_small": lambda: I.general_fracture_network(small()),
    "p1_medium": lambda: I.general_fracture_network(medium(), seed=21),
    "dense_small": lambda: I.with_dense_block(small(9), 2),
    "dense_wide": lambda: (lambda n: I.with_dense_block(n, wide_block_fracture(n)))(medium()),
}


@pytest.fixture(scope="module", params=list(NETS))
def pair(request):
    net = NETS[request.param]()
    return net, O.Schur(net)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_ainv(pair):
    net, ref = pair
    S = P.SchurSolver(net, general=True, k=4)
    v = I.rhs_normal(net.n_h, 3)
    y = to_np(S.ainv(dev(v)))
    assert_close(y, ref.ainv(v), TOL)
    assert_close(net.A.matvec(y), v, TOL)
    info = S.info()
    assert info["band_max"] > 0 and info["band_elems"] > 0 and info["t_factor_ms"] > 0 and info["t_trace_ms"] > 0


def test_schur_apply_and_diag(pair):
    net, ref = pair
    S = P.SchurSolver(net, general=True, k=4)
    for seed in (1, 2):
        r = I.rhs_normal(net.n_u, seed)
        assert_close(to_np(S.schur_apply(dev(r))), ref.apply(r), TOL)
    assert_close(to_np(S.diag()), ref.diag(), TOL)


def test_rhs_and_recovery(pair):
    net, ref = pair
    S = P.SchurSolver(net, general=True, k=4)
    r = to_np(S.rhs(dev(net.q)))
    assert_close(r, ref.rhs(net.q), TOL)
    u = I.rhs_normal(net.n_u, 4)
    h, p = S.recover(dev(net.q), dev(u))
    ho, po = ref.recover(net.q, u)
    assert_close(to_np(h), ho, TOL)
    assert_close(to_np(p), po, TOL)


@pytest.mark.parametrize("k", [0, 5])
def test_pcg_on_scaled_schur(pair, k):
    net, ref = pair
    opts = dict(k=k, lanczos_steps=min(10, net.n_u), rtol=1e-10, maxit=3000)
    S = P.SchurSolver(net, general=True, **opts)
    r = ref.rhs(net.q)
    x, st = S.solve(dev(r))
    xo, so = ref.pcg(ref.diag(), r, v0=I.lanczos_start(net.n_u, 0), **opts)
    assert so["status"] == 0 and st["status"] == 0
    assert st["alpha_hat"] == pytest.approx(so["alpha_hat"], rel=1e-9)
    # the two sides factor in different orders (reordered band with pivot
    # reciprocals vs the given numbering), so M differs in the last bits; the
    # iteration at which the residual crosses rtol may move by one
    d_it = abs(st["iterations"] - so["iterations"])
    if so["iterations"] <= 100:
        assert d_it <= 1
        assert_close(to_np(x), xo, (1e-9 if d_it == 0 else 1e-7))
    else:
        assert d_it <= 0.03 * so["iterations"]
        assert_close(to_np(x), xo, 1e-7)


def test_factor_path_equals_closed_form_on_rectangles():
    net = medium()
    G = P.SchurSolver(net, general=True, k=5, lanczos_steps=10)
    R = P.SchurSolver(net, general=False, k=5, lanczos_steps=10)
    r = I.rhs_normal(net.n_u, 7)
    assert_close(to_np(G.schur_apply(dev(r))), to_np(R.schur_apply(dev(r))), 1e-12)
    assert_close(to_np(G.diag()), to_np(R.diag()), 1e-12)
    v = I.rhs_normal(net.n_h, 8)
    assert_close(to_np(G.ainv(dev(v))), to_np(R.ainv(dev(v))), 1e-12)
    rhs = to_np(R.rhs(dev(net.q)))
    assert_close(to_np(G.rhs(dev(net.q))), rhs, 1e-12)
    xg, sg = G.solve(dev(rhs))
    xr, sr = R.solve(dev(rhs))
    assert sg["iterations"] == sr["iterations"]
    assert_close(to_np(xg), to_np(xr), 1e-10)
    # natural numbering of a rectangle already has the narrowest band it can get
    assert R.info()["band_max"] == 0
    assert G.info()["band_max"] <= int(np.maximum(net.nx, net.ny).max())


def test_reordering_recovers_the_band():
    """The renumbered blocks have no band in the given numbering; reverse
    Cuthill-McKee brings the half-bandwidth back to about the short side."""
    base = medium()
    net = I.general_fracture_network(base, seed=21)
    S = P.SchurSolver(net, general=True, k=3)
    short = int(np.minimum(base.nx, base.ny).max())
    assert S.info()["band_max"] <= 3 * short
    rows = np.repeat(np.arange(net.n_h), np.diff(net.A.rowptr))
    assert np.abs(rows - net.A.col).max() > 4 * short  # the given numbering is far wider


def test_fp32_preconditioner_on_general_blocks():
    net = I.general_fracture_network(medium(), seed=21)
    ref = O.Schur(net)
    r = ref.rhs(net.q)
    S64 = P.SchurSolver(net, k=8, lanczos_steps=10, rtol=1e-8)
    S32 = P.SchurSolver(net, k=8, lanczos_steps=10, rtol=1e-8, apply_prec="f32", flexible=1)
    x64, s64 = S64.solve(dev(r))
    x32, s32 = S32.solve(dev(r))
    assert s64["status"] == 0 and s32["status"] == 0
    assert abs(s32["iterations"] - s64["iterations"]) <= 2
    assert_close(ref.apply(to_np(x32)), r, 1e-7)


def _with_block(net, f, fn):
    """net with A_f replaced by fn(dense A_f) (fn keeps the sparsity pattern
    or fills the block)."""
    o, e = int(net.offset[f]), int(net.offset[f + 1])
    D = net.A.to_dense()
    D[o:e, o:e] = fn(D[o:e, o:e].copy())
    A = I.dense_to_csr(D)
    out = I.FractureNetwork(**{k: getattr(net, k) for k in ("nx", "ny", "T", "offset", "C", "B", "CT", "BT", "Gh",
                                                             "Gu", "q", "alpha", "own_node", "partner_node", "pair")},
                            A=A, meta=dict(net.meta, general=True))
    return out


def test_indefinite_block_is_breakdown():
    """Positive diagonal but indefinite (off-diagonals tripled): the device
    pivot check reports the failing fracture as PP_EBREAKDOWN."""
    net = I.general_fracture_network(small(), seed=4)

    def triple_off(B):
        d = np.diag(B).copy()
        B = 3.0 * B
        np.fill_diagonal(B, d)
        return B

    bad = _with_block(net, 3, triple_off)
    with pytest.raises(P.PolyPrecError) as ei:
        P.SchurSolver(bad, general=True, k=3)
    assert ei.value.status == P.PP_EBREAKDOWN
    assert "fracture 3" in str(ei.value)


def test_invalid_general_blocks_rejected():
    net = I.general_fracture_network(small(), seed=4)
    o = int(net.offset[1])

    def asym(B):
        i, j = np.nonzero(np.triu(B, 1))
        B[i[0], j[0]] *= 1.5
        return B

    with pytest.raises(P.PolyPrecError) as ei:
        P.SchurSolver(_with_block(net, 1, asym), general=True, k=3)
    assert ei.value.status == P.PP_EINVAL and "symmetric" in str(ei.value)
    # a coupling between two fractures
    D = net.A.to_dense()
    D[o - 1, o] = D[o, o - 1] = -0.1
    cross = I.FractureNetwork(**{k: getattr(net, k) for k in ("nx", "ny", "T", "offset", "C", "B", "CT", "BT", "Gh",
                                                               "Gu", "q", "alpha", "own_node", "partner_node",
                                                               "pair")}, A=I.dense_to_csr(D), meta=dict(net.meta))
    with pytest.raises(P.PolyPrecError) as ei:
        P.SchurSolver(cross, general=True, k=3)
    assert ei.value.status == P.PP_EINVAL and "block diagonal" in str(ei.value)
