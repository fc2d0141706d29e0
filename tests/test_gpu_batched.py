"""GPU parity of the batched solver (many instances, many right-hand sides,
one global slice list) against the FP64 oracle, column by column.

FP64 apply: every column's iteration count and solution equal those of the
oracle's single solve with the same interval (Lanczos from the same start
vector, or the interval set for that column) -- solution within 1e-10.
FP32 apply: converges to rtol, within 1e-7 of the oracle solution.
"""
import numpy as np
import pytest

import oracle as O
from helpers import assert_close, rel
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


SPECS = [I.BatchSpec(6, 0.5, 1, 11), I.BatchSpec(9, 2.0, 3, 12), I.BatchSpec(5, 1.0, 2, 13),
         I.BatchSpec(11, 3.0, 4, 14), I.BatchSpec(8, 1.5, 8, 15)]


@pytest.fixture(scope="module")
def problem():
    mats = [I.batch_instance(s) for s in SPECS]
    rhs = [I.batch_rhs(s) for s in SPECS]
    return mats, rhs


def oracle_cols(mats, rhs, k, seed, steps, abx=None, rtol=1e-10, flexible=False):
    out = []
    g = 0
    for i, (A, B) in enumerate(zip(mats, rhs)):
        for r in range(B.shape[1]):
            if abx is None:
                x, st = O.pcg_csr(A, B[:, r], v0=I.lanczos_start(A.n, seed + i), k=k, lanczos_steps=steps, rtol=rtol,
                                  flexible=flexible)
            else:
                a, b, xi = abx[g]
                x, st = O.pcg_csr(A, B[:, r], k=k, interval="given", alpha=a, beta=b, xi=xi, rtol=rtol,
                                  flexible=flexible)
            out.append((x, st))
            g += 1
    return out


FMTS = ["sell", "dia"]  # global SELL-32 slice list, or per-instance symmetric DIA


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("k", [0, 1, 6])
def test_batch_f64_matches_oracle_per_column(problem, graphs, k, fmt):
    mats, rhs = problem
    S = P.BatchSolver(mats, [s.nrhs for s in SPECS], k=k, lanczos_steps=10, seed=3, rtol=1e-10, use_graphs=graphs,
                      check_every=3, format=fmt)
    x, it, stv, st = S.solve(S.pack(rhs))
    xs = S.unpack(x)
    ref = oracle_cols(mats, rhs, k, 3, 10)
    g = 0
    for i, Xi in enumerate(xs):
        for r in range(Xi.shape[1]):
            xo, so = ref[g]
            assert stv[g] == 0 and so["status"] == 0
            assert it[g] == so["iterations"], (i, r)
            assert_close(Xi[:, r], xo, 1e-10)
            g += 1
    abx = S.intervals()
    for i, A in enumerate(mats):
        vh, _ = O.jacobi_scale(A)
        a, b = O.lanczos(A, I.lanczos_start(A.n, 3 + i), 10, val=vh)
        lo, hi = O.tridiag_extremes(a, b)
        c0 = sum(s.nrhs for s in SPECS[:i])
        assert abx[c0, 0] == pytest.approx(lo, rel=1e-9) and abx[c0, 1] == pytest.approx(hi, rel=1e-9)


def oracle_intervals(mats, seed, steps):
    """Per column (alpha, beta) from the oracle's Lanczos on each instance."""
    out = []
    for i, (A, s) in enumerate(zip(mats, SPECS)):
        vh, _ = O.jacobi_scale(A)
        a, b = O.lanczos(A, I.lanczos_start(A.n, seed + i), steps, val=vh)
        lo, hi = O.tridiag_extremes(a, b)
        out += [(lo, hi)] * s.nrhs
    return np.array(out)


@pytest.mark.parametrize("fmt", FMTS)
def test_batch_per_column_intervals(problem, fmt):
    mats, rhs = problem
    S = P.BatchSolver(mats, [s.nrhs for s in SPECS], k=5, rtol=1e-10, format=fmt)
    ab = oracle_intervals(mats, 0, 10)
    u = I.uniform(7, 9, 3 * S.ncols)
    abx = np.zeros((S.ncols, 3))
    abx[:, 0] = ab[:, 0] * (0.3 + u[0::3])  # different interval and xi in every column
    abx[:, 1] = ab[:, 1] * (1.0 + 0.2 * u[1::3])
    abx[:, 2] = 10.0 ** (-5 + 3 * u[2::3])
    S.intervals(abx)
    x, it, stv, st = S.solve(S.pack(rhs))
    ref = oracle_cols(mats, rhs, 5, 0, 10, abx=abx)
    xs = S.unpack(x)
    g = 0
    for Xi in xs:
        for r in range(Xi.shape[1]):
            xo, so = ref[g]
            assert it[g] == so["iterations"]
            assert_close(Xi[:, r], xo, 1e-10)
            g += 1


@pytest.mark.parametrize("fmt", FMTS)
def test_batch_f32_apply_converges(problem, fmt):
    mats, rhs = problem
    S = P.BatchSolver(mats, [s.nrhs for s in SPECS], k=6, rtol=1e-9, apply_prec="f32", flexible=1, use_graphs=1,
                      format=fmt)
    x, it, stv, st = S.solve(S.pack(rhs))
    assert (stv == 0).all()
    xs = S.unpack(x)
    ref = oracle_cols(mats, rhs, 6, 0, 10, rtol=1e-12)
    g = 0
    for i, Xi in enumerate(xs):
        for r in range(Xi.shape[1]):
            assert_close(Xi[:, r], ref[g][0], 1e-7)
            assert it[g] <= 2 * ref[g][1]["iterations"] + 5
            g += 1


@pytest.mark.parametrize("fmt", FMTS)
def test_batch_zero_rhs_column_and_features(problem, fmt):
    mats, rhs = problem
    rhs = [b.copy() for b in rhs]
    rhs[1][:, 1] = 0.0
    S = P.BatchSolver(mats, [s.nrhs for s in SPECS], k=3, rtol=1e-9, format=fmt)
    x, it, stv, st = S.solve(S.pack(rhs))
    assert it[SPECS[0].nrhs + 1] == 0 and stv[SPECS[0].nrhs + 1] == 0
    assert not S.unpack(x)[1][:, 1].any()
    F = S.features()
    for i, A in enumerate(mats):
        d = np.diag(A.to_dense())
        assert F[i, 0] == pytest.approx(np.log10(A.n))
        assert F[i, 1] == pytest.approx(np.log(d).mean(), rel=1e-12, abs=1e-12)
        assert F[i, 2] == pytest.approx(np.log(d).std(), rel=1e-9, abs=1e-12)
        vh, _ = O.jacobi_scale(A)
        Ah = I.CSR(A.n, A.rowptr, A.col, vh).to_dense()
        off = np.abs(Ah).sum(axis=1) - np.diag(Ah)
        assert F[i, 3] == pytest.approx((np.diag(Ah) + off).max(), rel=1e-12)
        assert F[i, 4] == pytest.approx((np.diag(Ah) - off).min(), rel=1e-12, abs=1e-12)


def test_batch_dia_rejects_unbanded_instance(problem):
    """DIA takes each instance's offsets from its first row; an instance with
    entries off those diagonals (here a dense SPD block) is refused."""
    mats, _ = problem
    D = I.dense_to_csr(I.random_spd(40, seed=2, cond=10.0))
    with pytest.raises(P.PolyPrecError) as ei:
        P.BatchSolver([mats[0], D], [1, 2], k=3, format="dia")
    assert ei.value.status in (P.PP_EUNSUPPORTED,)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_autotune_and_step_timer(problem, prec):
    """pp_batch_autotune times both layouts of these stencil instances and
    picks one; the solve in the chosen layout still matches the oracle;
    pp_batch_time_step reports a positive time and leaves the solver usable."""
    mats, rhs = problem
    fmt, table = P.batch_autotune(mats, [s.nrhs for s in SPECS], k=6, apply_prec=prec,
                                  flexible=1 if prec == "f32" else 0)
    assert fmt in ("dia", "sell")
    assert {t["format"] for t in table if t["status"] == 0} == {2, 3}
    assert all(t["us_per_step"] > 0 for t in table if t["status"] == 0)
    S = P.BatchSolver(mats, [s.nrhs for s in SPECS], k=6, lanczos_steps=8, rtol=1e-10, format=fmt, apply_prec=prec,
                      flexible=1 if prec == "f32" else 0, seed=100)
    assert S.time_step(reps=3) > 0
    x, it, st, _ = S.solve(S.pack(rhs))
    assert (st == 0).all()
    xs = S.unpack(x)
    ref = oracle_cols(mats, rhs, 6, 100, 8)
    g = 0
    for i, B in enumerate(rhs):
        for r in range(B.shape[1]):
            xo, so = ref[g]
            if prec == "f64":
                assert it[g] == so["iterations"]
                assert_close(xs[i][:, r], xo, 1e-10)
            else:
                assert_close(xs[i][:, r], xo, 1e-7)
            g += 1


# Instances for the FP32 DIA apply: grids with two 32-wide tiles in x, five
# 8-row tiles in y and two z chunks (N = 40), and R = 1..8 right-hand sides
# (all three register classes of the plane-marching step).
ZSPECS = [I.BatchSpec(40, 2.0, 5, 21), I.BatchSpec(6, 1.0, 1, 22), I.BatchSpec(12, 1.5, 7, 23),
          I.BatchSpec(9, 0.5, 2, 24), I.BatchSpec(7, 1.0, 4, 25), I.BatchSpec(5, 1.0, 3, 26),
          I.BatchSpec(8, 2.0, 8, 27), I.BatchSpec(4, 1.0, 6, 28)]


def banded_spd(n, offs, seed):
    """Symmetric banded matrix with the given upper offsets, every band entry
    nonzero and negative, made SPD by diagonal dominance."""
    D = np.zeros((n, n))
    u = I.uniform(seed, 5, n * len(offs))
    for t, o in enumerate(offs):
        v = -(0.1 + 0.8 * u[t * n:(t + 1) * n])[: n - o]
        D[np.arange(n - o), np.arange(o, n)] = v
        D[np.arange(o, n), np.arange(n - o)] = v
    D[np.arange(n), np.arange(n)] = np.abs(D).sum(axis=1) + 0.5
    return I.dense_to_csr(D)


def round_f32(x):
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("with_other", [0, 1])
def test_batch_f32_dia_apply_matches_rounded_oracle(with_other):
    """One FCG iteration from x0 = 0 gives x1 = (b, z) / (z, A z) z with
    z = W p_k(A_hat) W b, so every column's x1 checks the FP32 DIA apply of
    Algorithm 2 (plane marching for the grid instances; with_other adds
    instances it does not take, a 1-diagonal band and a 3-diagonal band whose
    size is not a grid, which the slice kernel steps in the same launch
    sequence) against the oracle run on the same FP32-rounded values, with
    the intervals given per column."""
    mats = [I.batch_instance(s) for s in ZSPECS]
    nrhs = [s.nrhs for s in ZSPECS]
    rhs = [I.batch_rhs(s) for s in ZSPECS]
    if with_other:
        mats += [banded_spd(300, [1], 31), banded_spd(100, [1, 5, 12], 32)]
        nrhs += [2, 3]
        rhs += [I.normal(33, 1, 600).reshape(300, 2), I.normal(34, 1, 300).reshape(100, 3)]
    k = 5
    S = P.BatchSolver(mats, nrhs, k=k, rtol=0.0, maxit=1, apply_prec="f32", flexible=1, format="dia")
    u = I.uniform(8, 9, 3 * S.ncols)
    abx = np.stack([0.02 + 0.05 * u[0::3], 1.9 + 0.1 * u[1::3], 10.0 ** (-4 + 2 * u[2::3])], axis=1)
    S.intervals(abx)
    x, it, stv, _ = S.solve(S.pack(rhs), allow=(P.PP_OK, P.PP_MAXIT))
    xs = S.unpack(x)
    g = 0
    for A, B, Xi in zip(mats, rhs, xs):
        vh, w = O.jacobi_scale(A)
        for r in range(B.shape[1]):
            a, b, xi = abx[g]
            z = w * O.cheb_apply(A, a, b, xi, k, w * B[:, r], val=round_f32(vh))
            x1 = (B[:, r] @ z) / (z @ A.matvec(z)) * z
            assert it[g] == 1
            assert_close(Xi[:, r], x1, 2e-5)
            g += 1
    S.close()
