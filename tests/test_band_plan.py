"""Host planning of the general fracture blocks (no GPU): the reordering
and half-bandwidth schur_setup would use, and its checks of A, through
pp_fracture_bands.

Pins: on a 5-point rectangle the narrowest band of any numbering is
min(nx, ny) (the bandwidth of the m x n grid graph, Chvatalova 1975), and
the x-fastest numbering has band nx; on a triangulated grid
with diagonal links the natural numbering has band nx + 1; a random
renumbering is undone to within a small factor of the short side.
"""
import numpy as np
import pytest

from paper_2208_01339_gb300 import inputs as I

P = pytest.importorskip("paper_2208_01339_gb300.polyprec")


@pytest.fixture(scope="module")
def lib():
    try:
        return P.lib()
    except Exception as e:  # pragma: no cover - the library is built by build()
        pytest.skip(f"library not built: {e}")


def net24():
    return I.fracture_network(n_f=24, side_min=3.0, side_max=9.0, h=0.25, trace_min=1.0, trace_max=6.0,
                              trace_fraction=0.06, T_sigma=1.0, seed=9)


def test_rectangles_get_the_short_side(lib):
    net = net24()
    w, rcm = P.fracture_bands(net.offset, net.A)
    short = np.minimum(net.nx, net.ny)
    assert np.all(w <= net.nx)               # never wider than the given numbering
    assert np.all(w <= short + 1)
    assert np.all(w >= short)                # no numbering beats the short side
    np.testing.assert_array_equal(rcm, w < net.nx)


def test_triangulated_blocks_natural_and_renumbered(lib):
    base = net24()
    nat = I.general_fracture_network(base, seed=21, shuffle=False)
    w, rcm = P.fracture_bands(nat.offset, nat.A)
    np.testing.assert_array_equal(w, np.minimum(base.nx + 1, w))  # at most the natural band nx + 1
    assert np.all(w[~rcm] == base.nx[~rcm] + 1)
    shuffled = I.general_fracture_network(base, seed=21)
    w2, rcm2 = P.fracture_bands(shuffled.offset, shuffled.A)
    sizes = np.diff(shuffled.offset)
    assert rcm2.all()
    assert np.all(w2 <= 3 * np.minimum(base.nx, base.ny) + 2)
    assert np.all(w2 < sizes // 4)           # the random numbering itself spans the whole block


def _replace_block(net, f, fn):
    o, e = int(net.offset[f]), int(net.offset[f + 1])
    D = net.A.to_dense()
    D[o:e, o:e] = fn(D[o:e, o:e].copy())
    return I.dense_to_csr(D)


def _small():
    return I.fracture_network(n_f=6, side_min=1.5, side_max=3.0, h=0.25, trace_min=0.5, trace_max=1.0,
                              trace_fraction=0.1, seed=5)


def test_dense_block_bands(lib):
    net = _small()
    A = _replace_block(net, 0, lambda B: B + 0.01)
    w, _ = P.fracture_bands(net.offset, A)
    assert w[0] == int(net.offset[1] - net.offset[0]) - 1


@pytest.mark.parametrize("case,status,text", [
    ("asymmetric", "PP_EINVAL", "symmetric"),
    ("coupled", "PP_EINVAL", "block diagonal"),
    ("negative_diagonal", "PP_EBREAKDOWN", "positive"),
    ("missing_diagonal", "PP_EINVAL", "diagonal"),
])
def test_invalid_blocks_rejected(lib, case, status, text):
    net = _small()
    if case == "asymmetric":
        def fn(B):
            i, j = np.nonzero(np.triu(B, 1))
            B[i[0], j[0]] *= 2.0
            return B
        A = _replace_block(net, 1, fn)
    elif case == "coupled":
        D = net.A.to_dense()
        o = int(net.offset[2])
        D[o - 1, o] = D[o, o - 1] = -0.5
        A = I.dense_to_csr(D)
    elif case == "negative_diagonal":
        def fn(B):
            B[0, 0] = -1.0
            return B
        A = _replace_block(net, 1, fn)
    else:
        def fn(B):
            B[3, 3] = 0.0
            return B
        A = _replace_block(net, 1, fn)
    with pytest.raises(P.PolyPrecError) as ei:
        P.fracture_bands(net.offset, A)
    assert ei.value.status == getattr(P, status)
    assert text in str(ei.value)


def test_repeated_entry_and_wide_band_rejected(lib):
    net = _small()
    A = net.A
    # repeat the first entry of row 0
    rp = A.rowptr.copy()
    rp[1:] += 1
    col = np.insert(A.col, 0, A.col[0])
    val = np.insert(A.val, 0, A.val[0])
    rep = I.CSR(A.n, rp, col, val, {})
    with pytest.raises(P.PolyPrecError) as ei:
        P.fracture_bands(net.offset, rep)
    assert ei.value.status == P.PP_EINVAL and "repeated" in str(ei.value)
    # one dense block of 800 nodes: no ordering narrows it below 768
    n = 800
    g = np.linspace(1.0, 2.0, n)
    D = np.outer(g, g) + n * np.eye(n)
    with pytest.raises(P.PolyPrecError) as ei:
        P.fracture_bands(np.array([0, n]), I.dense_to_csr(D))
    assert ei.value.status == P.PP_EUNSUPPORTED
