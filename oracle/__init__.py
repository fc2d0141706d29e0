"""FP64 CPU oracle for polynomial-preconditioned CG (arXiv 2208.01339).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()``
and the cpu_baseline / reference leg of ``bench.py`` -- never by the
product path (``paper_2208_01339_gb300``), which shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, single thread); this module
compiles it with gcc on first use and wraps it with ctypes.

Parity status of each routine (how it is pinned independently of itself):
  cheb_coeffs / cheb_poly   closed form 1 - x p_k(x) = T_{k+1}(y)/T_{k+1}(sigma),
                            equioscillation extrema, Table 1 eigenvalues
  cheb_apply                spectral mapping on dense eigendecompositions,
                            symmetry/positivity of p_k(A)A, Table 1
  newton_apply              equals cheb_apply at degree 2^nlev - 1, Table 1
  lanczos / extremes        numpy eigvalsh of T, interlacing, exact
                            extremes after n steps, Poisson closed form
  lanczos_basis             Q^T Q = I and Q^T A Q = T_m, n steps give the
                            exact spectrum
  tridiag_eig               numpy eigh of T (up to sign), residuals
  lowrank_vectors           eigenvectors of A (residuals) on a spectrum
                            with an isolated leftmost eigenvalue
  lowrank_apply             spectrum of P A for exact eigenvectors
                            (eigenvalue + 1, Section 3.1), invariance
                            under V -> V R, symmetry
  pcg_csr                   dense solves, Table 1 iteration counts,
                            Table 4 work counts; FCG(m) equals PCG for a
                            fixed SPD preconditioner
  fcg_dense                 A-orthogonality of the last m directions and
                            finite termination with a nonsymmetric M
  schur_*                   dense S_u from its expansion, diag, dense K_0
                            solve of the saddle-point system
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_omp = None


def _compile(out: str, srcs, extra, force: bool) -> str:
    deps = list(srcs) + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off"] + extra + ["-o", tmp] + list(srcs) + [
        "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, portable flags), and
    oracle.c + oracle_omp.c into liboracle_omp.so (-fopenmp), the timed
    all-core CPU baseline."""
    src = os.path.join(_HERE, "oracle.c")
    _compile(_OMP_PATH, [src, os.path.join(_HERE, "oracle_omp.c")], ["-fopenmp"], force)
    return _compile(_LIB_PATH, [src], [], force)


_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)
_ll = ctypes.POINTER(ctypes.c_longlong)


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("mvp", ctypes.c_longlong), ("dots", ctypes.c_longlong),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("alpha_hat", ctypes.c_double), ("beta_hat", ctypes.c_double), ("xi", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Options(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("xi", ctypes.c_double), ("interval", ctypes.c_int),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("lanczos_steps", ctypes.c_int),
                ("seed_scaling", ctypes.c_int), ("flexible", ctypes.c_int), ("maxit", ctypes.c_int),
                ("rtol", ctypes.c_double), ("lowrank", ctypes.c_int), ("lowrank_steps", ctypes.c_int),
                ("lr_V", ctypes.POINTER(ctypes.c_double))]


class Dfn(ctypes.Structure):
    _fields_ = [("n_f", ctypes.c_int), ("n_h", ctypes.c_int), ("n_u", ctypes.c_int), ("offset", _ll)] + [
        (f"{m}_{p}", t) for m in ("A", "C", "B", "CT", "BT", "Gh", "Gu")
        for p, t in (("rowptr", _i), ("col", _i), ("val", _d))] + [("alpha_reg", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.oracle_cheb_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         _d, _d, _d, _d]
        L.oracle_cheb_poly.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int]
        L.oracle_cheb_poly.restype = ctypes.c_double
        L.oracle_spmv.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d]
        L.oracle_cheb_apply.argtypes = [ctypes.c_int, _i, _i, _d, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _d, _d]
        L.oracle_newton_apply.argtypes = L.oracle_cheb_apply.argtypes
        L.oracle_jacobi_scale.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d]
        L.oracle_lanczos.argtypes = [ctypes.c_int, _i, _i, _d, _d, ctypes.c_int, _d, _d]
        L.oracle_tridiag_extremes.argtypes = [ctypes.c_int, _d, _d, _d, _d]
        L.oracle_lanczos_basis.argtypes = [ctypes.c_int, _i, _i, _d, _d, ctypes.c_int, _d, _d, _d]
        L.oracle_tridiag_eig.argtypes = [ctypes.c_int, _d, _d, ctypes.c_int, _d, _d]
        L.oracle_lowrank_vectors.argtypes = [ctypes.c_int, _i, _i, _d, _d, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, _d]
        L.oracle_lowrank_apply.argtypes = [ctypes.c_int, _i, _i, _d, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, _d, _d, _d]
        L.oracle_fcg_dense.argtypes = [ctypes.c_int, _d, _d, _d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_double, _d,
                                       ctypes.POINTER(Stats)]
        L.oracle_pcg_csr.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d, _d, ctypes.POINTER(Options),
                                     ctypes.POINTER(Stats)]
        L.oracle_schur_create.argtypes = [ctypes.POINTER(Dfn)]
        L.oracle_schur_create.restype = ctypes.c_void_p
        L.oracle_schur_free.argtypes = [ctypes.c_void_p]
        for name in ("oracle_ainv", "oracle_schur_apply", "oracle_schur_rhs"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _d, _d]
        L.oracle_schur_diag.argtypes = [ctypes.c_void_p, _d]
        L.oracle_schur_recover.argtypes = [ctypes.c_void_p, _d, _d, _d, _d]
        L.oracle_pcg_schur.argtypes = [ctypes.c_void_p, _d, _d, _d, _d, ctypes.POINTER(Options),
                                       ctypes.POINTER(Stats)]
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Coeffs:
    theta_bar: float
    delta: float
    sigma_bar: float
    rho: np.ndarray


def cheb_coeffs(alpha: float, beta: float, xi: float, k: int) -> Coeffs:
    tb, d, sb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rho = np.zeros(k + 1)
    rc = lib().oracle_cheb_coeffs(alpha, beta, xi, k, ctypes.byref(tb), ctypes.byref(d), ctypes.byref(sb),
                                  _p(rho, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_cheb_coeffs: status {rc}")
    return Coeffs(tb.value, d.value, sb.value, rho)


def cheb_poly(x: float, alpha: float, beta: float, xi: float, k: int) -> float:
    return lib().oracle_cheb_poly(float(x), alpha, beta, xi, k)


def spmv(A, x) -> np.ndarray:
    x = _f64(x)
    y = np.zeros(A.n)
    rp, ci, va = _i32(A.rowptr), _i32(A.col), _f64(A.val)
    lib().oracle_spmv(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                      _p(x, ctypes.c_double), _p(y, ctypes.c_double))
    return y


def _apply(fn, A, alpha, beta, xi, k, r, val=None) -> np.ndarray:
    r = _f64(r)
    z = np.zeros(A.n)
    rp, ci = _i32(A.rowptr), _i32(A.col)
    va = _f64(A.val if val is None else val)
    rc = fn(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double), alpha, beta, xi, k,
            _p(r, ctypes.c_double), _p(z, ctypes.c_double))
    if rc:
        raise RuntimeError(f"oracle apply status {rc}")
    return z


def cheb_apply(A, alpha: float, beta: float, xi: float, k: int, r, val=None) -> np.ndarray:
    """z = p_k(A) r by Algorithm 2 (A as a CSR with optional replacement values)."""
    return _apply(lib().oracle_cheb_apply, A, alpha, beta, xi, k, r, val)


def newton_apply(A, alpha: float, beta: float, xi: float, nlev: int, r) -> np.ndarray:
    """z = P_nlev r by Algorithm 1 (degree 2^nlev - 1)."""
    return _apply(lib().oracle_newton_apply, A, alpha, beta, xi, nlev, r)


def jacobi_scale(A):
    """(values of W^T A W, W) with W = diag(A)^{-1/2}."""
    vh = np.zeros(A.nnz)
    w = np.zeros(A.n)
    rp, ci, va = _i32(A.rowptr), _i32(A.col), _f64(A.val)
    rc = lib().oracle_jacobi_scale(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                                   _p(vh, ctypes.c_double), _p(w, ctypes.c_double))
    if rc:
        raise RuntimeError(f"jacobi_scale status {rc}")
    return vh, w


def lanczos(A, v0, m: int, val=None):
    """(a, b) of the m-step Lanczos tridiagonal T_m started from v0."""
    a = np.zeros(m)
    b = np.zeros(max(m, 1))
    rp, ci = _i32(A.rowptr), _i32(A.col)
    va = _f64(A.val if val is None else val)
    v0 = _f64(v0)
    steps = lib().oracle_lanczos(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                                 _p(v0, ctypes.c_double), m, _p(a, ctypes.c_double), _p(b, ctypes.c_double))
    return a[:steps], b[:max(steps - 1, 0)]


def tridiag_extremes(a, b):
    a, b = _f64(a), _f64(np.append(b, 0.0))
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_tridiag_extremes(len(a), _p(a, ctypes.c_double), _p(b, ctypes.c_double), ctypes.byref(lo),
                                       ctypes.byref(hi))
    if rc:
        raise RuntimeError("tridiag_extremes")
    return lo.value, hi.value


def lanczos_basis(A, v0, m: int, val=None):
    """(a, b, Q) of m Lanczos steps keeping the basis (full reorthogonalisation).

    b has one entry per step: b[-1] is beta_m, the coupling to the next vector.
    Q is n x steps with the Lanczos vectors as columns."""
    a = np.zeros(m)
    b = np.zeros(m)
    Q = np.zeros((m, A.n))
    rp, ci = _i32(A.rowptr), _i32(A.col)
    va = _f64(A.val if val is None else val)
    v0 = _f64(v0)
    steps = lib().oracle_lanczos_basis(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                                       _p(v0, ctypes.c_double), m, _p(a, ctypes.c_double), _p(b, ctypes.c_double),
                                       _p(Q, ctypes.c_double))
    return a[:steps], b[:steps], Q[:steps].T.copy()


def tridiag_eig(a, b, i: int):
    """(lambda_i, y_i): the i-th smallest eigenpair of the tridiagonal (a, b)."""
    a, b = _f64(a), _f64(np.append(b, 0.0))
    lam = ctypes.c_double()
    y = np.zeros(len(a))
    rc = lib().oracle_tridiag_eig(len(a), _p(a, ctypes.c_double), _p(b, ctypes.c_double), i, ctypes.byref(lam),
                                  _p(y, ctypes.c_double))
    if rc:
        raise RuntimeError("tridiag_eig")
    return lam.value, y


def lowrank_vectors(A, v0, alpha: float, beta: float, xi: float, k: int, p: int, m: int, val=None):
    """(V, theta): Ritz vectors of the p smallest Ritz values of m Lanczos steps
    (full reorthogonalisation) on p_k(A) A from v0, and v^T A v for each."""
    V = np.zeros((p, A.n))
    theta = np.zeros(p)
    rp, ci = _i32(A.rowptr), _i32(A.col)
    va = _f64(A.val if val is None else val)
    v0 = _f64(v0)
    rc = lib().oracle_lowrank_vectors(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                                      _p(v0, ctypes.c_double), alpha, beta, xi, k, p, m, _p(V, ctypes.c_double),
                                      _p(theta, ctypes.c_double))
    if rc:
        raise RuntimeError(f"oracle lowrank_vectors status {rc}")
    return V.T.copy(), theta


def lowrank_apply(A, alpha: float, beta: float, xi: float, k: int, V, r, val=None) -> np.ndarray:
    """z = p_k(A) r + V (V^T A V)^{-1} V^T r (Section 3.1); V is n x p."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Vc = np.ascontiguousarray(V.T)
    r = _f64(r)
    z = np.zeros(A.n)
    rp, ci = _i32(A.rowptr), _i32(A.col)
    va = _f64(A.val if val is None else val)
    rc = lib().oracle_lowrank_apply(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double), alpha,
                                    beta, xi, k, V.shape[1], _p(Vc, ctypes.c_double), _p(r, ctypes.c_double),
                                    _p(z, ctypes.c_double))
    if rc:
        raise RuntimeError(f"oracle lowrank_apply status {rc}")
    return z


def make_options(k=20, xi=-1.0, interval="lanczos", alpha=0.0, beta=0.0, lanczos_steps=10, seed_scaling=True,
                 flexible=False, maxit=10000, rtol=1e-8, lowrank=0, lowrank_steps=0, lr_V=None) -> Options:
    """Options; lr_V (n x p, seed-scaled space) must stay alive while they are used."""
    o = Options(k=k, xi=xi, interval=0 if interval == "lanczos" else 1, alpha=alpha, beta=beta,
                lanczos_steps=lanczos_steps, seed_scaling=1 if seed_scaling else 0,
                flexible=1 if flexible else 0, maxit=maxit, rtol=rtol, lowrank=lowrank, lowrank_steps=lowrank_steps)
    if lr_V is not None:
        o._keep = np.ascontiguousarray(np.asarray(lr_V, dtype=np.float64).T)
        o.lowrank = lr_V.shape[1]
        o.lr_V = _p(o._keep, ctypes.c_double)
    return o


def fcg_dense(A, M, b, m: int, maxit: int, rtol: float = 0.0, x0=None):
    """FCG(m) (m >= 2) on dense A with the dense preconditioner M.
    Returns (x, directions [iterations+1 x n], stats dict)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    n = A.shape[0]
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    dirs = np.zeros((maxit + 1, n))
    st = Stats()
    lib().oracle_fcg_dense(n, _p(A, ctypes.c_double), _p(M, ctypes.c_double), _p(b, ctypes.c_double),
                           _p(x, ctypes.c_double), m, maxit, rtol, _p(dirs, ctypes.c_double), ctypes.byref(st))
    return x, dirs[:st.iterations + 1], st.as_dict()


def pcg_csr(A, b, x0=None, v0=None, **opts):
    """Full solve: Jacobi seed, interval, xi, coefficients, PCG. Returns (x, stats dict)."""
    o = make_options(**opts)
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    v0 = np.ones(A.n) if v0 is None else _f64(v0)
    st = Stats()
    rp, ci, va = _i32(A.rowptr), _i32(A.col), _f64(A.val)
    lib().oracle_pcg_csr(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                         _p(b, ctypes.c_double), _p(x, ctypes.c_double), _p(v0, ctypes.c_double),
                         ctypes.byref(o), ctypes.byref(st))
    return x, st.as_dict()


class Schur:
    """Oracle Schur-complement operator of a ``FractureNetwork`` (Section 4.2)."""

    def __init__(self, net):
        self._keep = []

        def keep(a, conv):
            a = conv(a)
            self._keep.append(a)
            return a

        d = Dfn()
        d.n_f, d.n_h, d.n_u = net.n_f, net.n_h, net.n_u
        off = keep(net.offset, lambda a: np.ascontiguousarray(a, dtype=np.int64))
        d.offset = _p(off, ctypes.c_longlong)
        for m, M in (("A", net.A), ("C", net.C), ("B", net.B), ("CT", net.CT), ("BT", net.BT), ("Gh", net.Gh),
                     ("Gu", net.Gu)):
            setattr(d, f"{m}_rowptr", _p(keep(M.rowptr, _i32), ctypes.c_int))
            setattr(d, f"{m}_col", _p(keep(M.col, _i32), ctypes.c_int))
            setattr(d, f"{m}_val", _p(keep(M.val, _f64), ctypes.c_double))
        d.alpha_reg = net.alpha
        self._d = d
        self.n_h, self.n_u = net.n_h, net.n_u
        self._h = lib().oracle_schur_create(ctypes.byref(d))
        if not self._h:
            raise RuntimeError("oracle_schur_create failed (A block not SPD?)")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_schur_free(self._h)
            self._h = None

    def ainv(self, v):
        v = _f64(v)
        y = np.zeros(self.n_h)
        lib().oracle_ainv(self._h, _p(v, ctypes.c_double), _p(y, ctypes.c_double))
        return y

    def apply(self, r):
        r = _f64(r)
        y = np.zeros(self.n_u)
        rc = lib().oracle_schur_apply(self._h, _p(r, ctypes.c_double), _p(y, ctypes.c_double))
        if rc:
            raise RuntimeError(f"schur_apply status {rc}")
        return y

    def diag(self):
        ds = np.zeros(self.n_u)
        rc = lib().oracle_schur_diag(self._h, _p(ds, ctypes.c_double))
        if rc:
            raise RuntimeError(f"schur_diag status {rc}")
        return ds

    def rhs(self, q):
        q = _f64(q)
        r = np.zeros(self.n_u)
        lib().oracle_schur_rhs(self._h, _p(q, ctypes.c_double), _p(r, ctypes.c_double))
        return r

    def recover(self, q, u):
        q, u = _f64(q), _f64(u)
        h = np.zeros(self.n_h)
        p = np.zeros(self.n_h)
        lib().oracle_schur_recover(self._h, _p(q, ctypes.c_double), _p(u, ctypes.c_double), _p(h, ctypes.c_double),
                                   _p(p, ctypes.c_double))
        return h, p

    def pcg(self, ds, r, u0=None, v0=None, **opts):
        o = make_options(**opts)
        r = _f64(r)
        ds = _f64(ds)
        u = np.zeros(self.n_u) if u0 is None else _f64(u0).copy()
        v0 = np.ones(self.n_u) if v0 is None else _f64(v0)
        st = Stats()
        lib().oracle_pcg_schur(self._h, _p(ds, ctypes.c_double), _p(r, ctypes.c_double), _p(u, ctypes.c_double),
                               _p(v0, ctypes.c_double), ctypes.byref(o), ctypes.byref(st))
        return u, st.as_dict()


def omp_lib():
    """liboracle_omp.so: the oracle's loops with OpenMP over rows (timed CPU
    baseline only; parity uses the single-thread lib())."""
    global _omp
    if _omp is None:
        build()
        L = ctypes.CDLL(_OMP_PATH)
        L.oracle_omp_threads.restype = ctypes.c_int
        L.oracle_omp_solve.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d, _d, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(Stats), _d]
        _omp = L
    return _omp


def omp_threads() -> int:
    return int(omp_lib().oracle_omp_threads())


def omp_solve(A, b, v0, k: int, lanczos_steps: int, rtol: float = 1e-8, maxit: int = 10000, xi: float = -1.0):
    """All-core PCG solve from x = 0 (Jacobi seed, Lanczos interval, p_k by
    Algorithm 2).  Returns (x, stats dict, setup seconds, PCG seconds)."""
    b = _f64(b)
    v0 = _f64(v0)
    x = np.zeros(A.n)
    st = Stats()
    sec = np.zeros(2)
    rp, ci, va = _i32(A.rowptr), _i32(A.col), _f64(A.val)
    omp_lib().oracle_omp_solve(A.n, _p(rp, ctypes.c_int), _p(ci, ctypes.c_int), _p(va, ctypes.c_double),
                               _p(b, ctypes.c_double), _p(x, ctypes.c_double), _p(v0, ctypes.c_double), int(k),
                               int(lanczos_steps), float(xi), float(rtol), int(maxit), ctypes.byref(st),
                               _p(sec, ctypes.c_double))
    return x, st.as_dict(), float(sec[0]), float(sec[1])
