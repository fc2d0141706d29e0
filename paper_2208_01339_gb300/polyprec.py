"""Python binding of libpolyprec (argument marshalling only).

Every step of the method runs inside the CUDA library declared in
include/polyprec.h; this module passes device pointers (PyTorch tensors),
sizes and the current CUDA stream through ctypes.  There is no CPU or
PyTorch fallback: if the library is missing, importing ``lib()`` raises.

Entry points mirror the C ABI: ``polyprec_coeffs``, ``Solver`` (pcg_setup /
polyprec_apply / pp_operator_apply / pcg_solve / pp_destroy) and
``SchurSolver`` (schur_setup / schur_apply / schur_diag / schur_rhs /
schur_recover / pcg_solve).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolyprec.so")

PP_OK, PP_MAXIT, PP_EINVAL, PP_EBREAKDOWN, PP_ENONFINITE, PP_ECUDA, PP_ETIMEOUT, PP_EUNSUPPORTED = 0, 1, -1, -2, -3, -4, -5, -6
INTERVAL = {"lanczos": 0, "given": 1}
FORMAT = {"auto": 0, "csr": 1, "sell": 2, "dia": 3}
PREC = {"f64": 0, "f32": 1, "bf16": 2}
SEED = {"none": 0, "jacobi": 1}

_vp = ctypes.c_void_p


class PolyPrecError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libpolyprec status {status}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_longlong), ("rowptr", _vp), ("col", _vp), ("val", _vp)]


class Options(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("xi", ctypes.c_double), ("interval", ctypes.c_int),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("lanczos_steps", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("seed_scaling", ctypes.c_int), ("format", ctypes.c_int),
                ("sell_C", ctypes.c_int), ("sell_sigma", ctypes.c_int), ("apply_prec", ctypes.c_int),
                ("flexible", ctypes.c_int), ("maxit", ctypes.c_int), ("rtol", ctypes.c_double),
                ("zero_guess", ctypes.c_int), ("check_every", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("sell_variant", ctypes.c_int), ("lowrank", ctypes.c_int),
                ("lowrank_steps", ctypes.c_int), ("poly", ctypes.c_int), ("max_blocks", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("mvp", ctypes.c_longlong), ("dots", ctypes.c_longlong),
                ("rel_res", ctypes.c_double), ("alpha_hat", ctypes.c_double), ("beta_hat", ctypes.c_double),
                ("xi", ctypes.c_double), ("theta_bar", ctypes.c_double), ("delta", ctypes.c_double),
                ("sigma_bar", ctypes.c_double), ("t_solve_ms", ctypes.c_double), ("t_apply_ms", ctypes.c_double),
                ("apply_launches", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("format", ctypes.c_int), ("sell_C", ctypes.c_int), ("sell_sigma", ctypes.c_int),
                ("nnz", ctypes.c_longlong), ("nnz_padded", ctypes.c_longlong), ("alpha_hat", ctypes.c_double),
                ("beta_hat", ctypes.c_double), ("xi", ctypes.c_double), ("theta_bar", ctypes.c_double),
                ("delta", ctypes.c_double), ("sigma_bar", ctypes.c_double), ("k", ctypes.c_int),
                ("apply_prec", ctypes.c_int), ("lanczos_steps_done", ctypes.c_int), ("t_setup_ms", ctypes.c_double),
                ("grid_blocks", ctypes.c_int), ("ndiag", ctypes.c_int), ("lowrank", ctypes.c_int),
                ("lowrank_steps_done", ctypes.c_int), ("ritz_resid", ctypes.c_double), ("theta_min", ctypes.c_double),
                ("band_max", ctypes.c_int), ("band_elems", ctypes.c_longlong), ("t_factor_ms", ctypes.c_double),
                ("t_trace_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneEntry(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int), ("sell_C", ctypes.c_int), ("sell_sigma", ctypes.c_int),
                ("sell_variant", ctypes.c_int), ("us_per_step", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_longlong), ("rowptr", _vp), ("col", _vp), ("val", _vp),
                ("nrhs", ctypes.c_int)]


BATCH_NFEAT = 8

_DFN_MATS = ("C", "B", "CT", "BT", "Gh", "Gu")


class Dfn(ctypes.Structure):
    _fields_ = [("n_f", ctypes.c_int), ("n_h", ctypes.c_int), ("n_u", ctypes.c_int), ("nx", _vp), ("ny", _vp),
                ("T", _vp), ("offset", _vp)] + [
        (f"{m}_{p}", _vp) for m in _DFN_MATS for p in ("rowptr", "col", "val")] + [("alpha_reg", ctypes.c_double)] + [
        (f"A_{p}", _vp) for p in ("rowptr", "col", "val")]


_lib = None

# (name, restype, argtypes) of every exported function of include/polyprec.h
SIGNATURES = [
    ("pp_options_default", None, [ctypes.POINTER(Options)]),
    ("polyprec_coeffs", ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("pp_workspace_size", ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_size_t)]),
    ("pcg_setup", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Csr), ctypes.POINTER(Options), _vp,
                                 ctypes.c_size_t, _vp]),
    ("polyprec_apply", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    ("pp_operator_apply", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    ("pcg_solve", ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(Stats), _vp]),
    ("pp_get_info", ctypes.c_int, [_vp, ctypes.POINTER(Info)]),
    ("pp_set_lowrank", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_longlong, _vp]),
    ("pp_autotune_workspace_size", ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Options),
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    ("pp_autotune", ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Options), _vp, ctypes.c_size_t,
                                   ctypes.POINTER(TuneEntry), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp]),
    ("pp_destroy", ctypes.c_int, [_vp]),
    ("pp_last_error", ctypes.c_char_p, [_vp]),
    ("pp_schur_workspace_size", ctypes.c_int, [ctypes.POINTER(Dfn), ctypes.POINTER(Options),
                                               ctypes.POINTER(ctypes.c_size_t)]),
    ("schur_setup", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Dfn), ctypes.POINTER(Options), _vp,
                                   ctypes.c_size_t, _vp]),
    ("schur_apply", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("schur_diag", ctypes.c_int, [_vp, _vp, _vp]),
    ("schur_rhs", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("schur_recover", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("schur_ainv", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("pp_fracture_bands", ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("pp_batch_workspace_size", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(Options),
                                               ctypes.POINTER(ctypes.c_size_t)]),
    ("pp_batch_setup", ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.c_int, ctypes.POINTER(Options), _vp,
                                      ctypes.c_size_t, _vp]),
    ("pp_batch_intervals", ctypes.c_int, [_vp, _vp, _vp]),
    ("pp_batch_features", ctypes.c_int, [_vp, _vp]),
    ("pp_batch_solve", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(Stats), _vp]),
    ("pp_batch_time_step", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    ("pp_batch_autotune_workspace_size", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(Options),
                                                        ctypes.POINTER(ctypes.c_size_t)]),
    ("pp_batch_autotune", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(Options), _vp, ctypes.c_size_t,
                                         ctypes.POINTER(TuneEntry), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp]),
    ("pp_mlp_workspace_size", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("pp_mlp_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_ulonglong, _vp, ctypes.c_size_t]),
    ("pp_mlp_params", ctypes.c_int, [_vp, _vp, _vp]),
    ("pp_mlp_forward", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    ("pp_mlp_grad", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp]),
    ("pp_mlp_train_step", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp, _vp]),
    ("pp_mlp_destroy", ctypes.c_int, [_vp]),
    ("pp_fp64_fma_rate", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    ("polyprec_apply_csr_static", ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, _vp, _vp, _vp, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, _vp, _vp]),
]


def lib() -> ctypes.CDLL:
    """Load the in-tree libpolyprec.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpolyprec.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _err(ctx=None) -> str:
    m = lib().pp_last_error(ctx)
    return m.decode() if m else ""


def _check(rc: int, ctx=None, allow=(PP_OK,)) -> int:
    if rc not in allow:
        raise PolyPrecError(rc, _err(ctx))
    return rc


def polyprec_coeffs(alpha: float, beta: float, xi: float, k: int):
    """(theta_bar, delta, sigma_bar, rho[0..k]) -- host-side coefficient table."""
    tb, d, sb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rho = np.zeros(k + 1)
    rc = lib().polyprec_coeffs(alpha, beta, xi, k, ctypes.byref(tb), ctypes.byref(d), ctypes.byref(sb),
                               rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc)
    return tb.value, d.value, sb.value, rho


def fracture_bands(offset, A):
    """(w, rcm): per fracture, the half-bandwidth of the banded Cholesky
    factor that schur_setup would build for the general blocks A (host CSR
    with rowptr/col/val) and whether reverse Cuthill-McKee was chosen.
    Host only (pp_fracture_bands)."""
    off = np.ascontiguousarray(offset, dtype=np.int64)
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    n_f = off.size - 1
    w = np.zeros(n_f, dtype=np.int32)
    rcm = np.zeros(n_f, dtype=np.int32)
    _check(lib().pp_fracture_bands(n_f, _vp(off.ctypes.data), _vp(rp.ctypes.data), _vp(ci.ctypes.data),
                                   _vp(va.ctypes.data), _vp(w.ctypes.data), _vp(rcm.ctypes.data)))
    return w, rcm.astype(bool)


def make_options(**kw) -> Options:
    o = Options()
    lib().pp_options_default(ctypes.byref(o))
    for key, v in kw.items():
        if key == "interval":
            v = INTERVAL[v] if isinstance(v, str) else v
        elif key == "format":
            v = FORMAT[v] if isinstance(v, str) else v
        elif key == "apply_prec":
            v = PREC[v] if isinstance(v, str) else v
        elif key == "poly":
            v = {"cheb": 0, "newton": 1}[v] if isinstance(v, str) else v
        elif key == "seed_scaling":
            v = SEED[v] if isinstance(v, str) else (1 if v is True else (0 if v is False else v))
        elif isinstance(v, bool):
            v = int(v)
        if not hasattr(o, key):
            raise KeyError(f"unknown option {key}")
        setattr(o, key, v)
    return o


def _torch():
    import torch  # noqa: PLC0415  (device memory and streams only)
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _ptr(t) -> _vp:
    return _vp(t.data_ptr())


def to_device_csr(A, device="cuda"):
    """Upload a host CSR (rowptr/col int32, val float64) to device tensors."""
    torch = _torch()
    rp = torch.as_tensor(np.ascontiguousarray(A.rowptr, dtype=np.int32), device=device)
    ci = torch.as_tensor(np.ascontiguousarray(A.col, dtype=np.int32), device=device)
    va = torch.as_tensor(np.ascontiguousarray(A.val, dtype=np.float64), device=device)
    return rp, ci, va


def apply_csr_static(rowptr, col, val, n: int, alpha: float, beta: float, xi: float, k: int, r, z=None,
                     stream=None):
    """z = p_k(A) r without a workspace (polyprec_apply_csr_static): for
    callers that cannot allocate device memory; n <= 262,144."""
    torch = _torch()
    if z is None:
        z = torch.empty_like(r)
    rc = lib().polyprec_apply_csr_static(int(n), int(val.numel()), _ptr(rowptr), _ptr(col), _ptr(val), alpha, beta,
                                         xi, int(k), _ptr(r), _ptr(z), _stream(stream))
    _check(rc)
    return z


def fp64_fma_rate(reps: int = 5, device="cuda", stream=None) -> float:
    """Measured FP64 FMA rate of the device in TFLOP/s (pp_fp64_fma_rate)."""
    torch = _torch()
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    tf = ctypes.c_double()
    _check(lib().pp_fp64_fma_rate(_ptr(sink), int(reps), ctypes.byref(tf), _stream(stream)))
    return tf.value


FORMAT_NAME = {1: "csr", 2: "sell", 3: "dia"}


def autotune(rowptr, col, val, n: int, stream=None, **options):
    """Time every storage layout of the fused degree step on this matrix
    (pp_autotune) and return (options dict with the fastest layout, list of
    per-layout results)."""
    torch = _torch()
    opts = make_options(**options)
    csr = Csr(int(n), int(val.numel()), _ptr(rowptr), _ptr(col), _ptr(val))
    nbytes = ctypes.c_size_t()
    _check(lib().pp_autotune_workspace_size(ctypes.byref(csr), ctypes.byref(opts), ctypes.byref(nbytes)))
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=val.device)
    ent = (TuneEntry * 16)()
    cnt = ctypes.c_int()
    _check(lib().pp_autotune(ctypes.byref(csr), ctypes.byref(opts), _ptr(ws), ws.numel(), ent, 16, ctypes.byref(cnt),
                             _stream(stream)))
    del ws
    chosen = dict(options)
    chosen.update(format=FORMAT_NAME[opts.format], sell_C=opts.sell_C, sell_sigma=opts.sell_sigma,
                  sell_variant=opts.sell_variant)
    return chosen, [ent[i].as_dict() for i in range(cnt.value)]


class Solver:
    """PCG with P = W p_k(W^T A W) W^T on one sparse SPD matrix (device CSR)."""

    def __init__(self, rowptr, col, val, n: int, stream=None, **options):
        torch = _torch()
        self.n = int(n)
        self.opts = make_options(**options)
        self._keep = (rowptr, col, val)
        csr = Csr(self.n, int(val.numel()), _ptr(rowptr), _ptr(col), _ptr(val))
        nbytes = ctypes.c_size_t()
        _check(lib().pp_workspace_size(ctypes.byref(csr), ctypes.byref(self.opts), ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=val.device)
        ctx = _vp()
        s = _stream(stream)
        _check(lib().pcg_setup(ctypes.byref(ctx), ctypes.byref(csr), ctypes.byref(self.opts),
                               _ptr(self.workspace), self.workspace.numel(), s))
        self.ctx = ctx
        self.device = val.device

    @classmethod
    def from_host(cls, A, device="cuda", **options):
        rp, ci, va = to_device_csr(A, device)
        return cls(rp, ci, va, A.n, **options)

    def info(self) -> dict:
        i = Info()
        _check(lib().pp_get_info(self.ctx, ctypes.byref(i)), self.ctx)
        return i.as_dict()

    def apply(self, r, z=None, stream=None):
        """z = P r; r is (n,) or (nrhs, n) FP64 on the device."""
        torch = _torch()
        r = r.contiguous()
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        if z is None:
            z = torch.empty_like(r)
        _check(lib().polyprec_apply(self.ctx, _ptr(r), _ptr(z), nrhs, _stream(stream)), self.ctx)
        return z

    def set_lowrank(self, U, stream=None):
        """Use the caller vectors U ((p, n) FP64 on the device, unscaled space)
        for the Section 3.1 correction U (U^T A U)^{-1} U^T; p = 0 removes it."""
        U = U.contiguous()
        p = 0 if U.numel() == 0 else (1 if U.dim() == 1 else U.shape[0])
        _check(lib().pp_set_lowrank(self.ctx, _ptr(U) if p else None, p, self.n, _stream(stream)), self.ctx)

    def operator(self, x, y=None, stream=None):
        torch = _torch()
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = torch.empty_like(x)
        _check(lib().pp_operator_apply(self.ctx, _ptr(x), _ptr(y), nrhs, _stream(stream)), self.ctx)
        return y

    def solve(self, b, x=None, stream=None, allow=(PP_OK, PP_MAXIT)):
        """Solve A x = b; returns (x, stats dict).  Statuses outside `allow` raise."""
        torch = _torch()
        if x is None:
            x = torch.zeros_like(b)
        st = Stats()
        rc = lib().pcg_solve(self.ctx, _ptr(b), _ptr(x), ctypes.byref(st), _stream(stream))
        _check(rc, self.ctx, allow)
        d = st.as_dict()
        d["status"] = rc
        return x, d

    def close(self):
        if getattr(self, "ctx", None):
            lib().pp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SchurSolver(Solver):
    """PCG on the D_S-scaled Schur complement S_u of a fracture network.

    general=True hands the network's block-diagonal A to the library
    (banded Cholesky factors of the fracture blocks) instead of the
    rectangle metadata (closed-form inverse blocks); the default follows
    net.meta["general"]."""

    def __init__(self, net, device="cuda", stream=None, general=None, **options):  # noqa: D401
        torch = _torch()
        self.n = int(net.n_u)
        self.opts = make_options(**options)
        keep = []

        def dev(a, dt):
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device=device)
            keep.append(t)
            return _ptr(t)

        def host(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return _vp(a.ctypes.data)

        d = Dfn()
        d.n_f, d.n_h, d.n_u = net.n_f, net.n_h, net.n_u
        d.nx = host(net.nx, np.int32)
        d.ny = host(net.ny, np.int32)
        d.T = host(net.T, np.float64)
        d.offset = host(net.offset, np.int64)
        for m in _DFN_MATS:
            M = getattr(net, m)
            setattr(d, f"{m}_rowptr", dev(M.rowptr, np.int32))
            setattr(d, f"{m}_col", dev(M.col, np.int32))
            setattr(d, f"{m}_val", dev(M.val, np.float64))
        d.alpha_reg = float(net.alpha)
        if general is None:
            general = bool(net.meta.get("general", False))
        if general:
            d.A_rowptr = dev(net.A.rowptr, np.int32)
            d.A_col = dev(net.A.col, np.int32)
            d.A_val = dev(net.A.val, np.float64)
        self._keep = keep
        self._dfn = d
        nbytes = ctypes.c_size_t()
        _check(lib().pp_schur_workspace_size(ctypes.byref(d), ctypes.byref(self.opts), ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        ctx = _vp()
        _check(lib().schur_setup(ctypes.byref(ctx), ctypes.byref(d), ctypes.byref(self.opts), _ptr(self.workspace),
                                 self.workspace.numel(), _stream(stream)))
        self.ctx = ctx
        self.n_h = int(net.n_h)
        self.device = torch.device(device)

    def schur_apply(self, r, y=None, stream=None):
        torch = _torch()
        y = torch.empty_like(r) if y is None else y
        _check(lib().schur_apply(self.ctx, _ptr(r), _ptr(y), _stream(stream)), self.ctx)
        return y

    def diag(self, stream=None):
        torch = _torch()
        ds = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(lib().schur_diag(self.ctx, _ptr(ds), _stream(stream)), self.ctx)
        return ds

    def rhs(self, q, stream=None):
        torch = _torch()
        r = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(lib().schur_rhs(self.ctx, _ptr(q), _ptr(r), _stream(stream)), self.ctx)
        return r

    def recover(self, q, u, stream=None):
        torch = _torch()
        h = torch.empty(self.n_h, dtype=torch.float64, device=self.device)
        p = torch.empty(self.n_h, dtype=torch.float64, device=self.device)
        _check(lib().schur_recover(self.ctx, _ptr(q), _ptr(u), _ptr(h), _ptr(p), _stream(stream)), self.ctx)
        return h, p

    def ainv(self, v, stream=None):
        torch = _torch()
        y = torch.empty_like(v)
        _check(lib().schur_ainv(self.ctx, _ptr(v), _ptr(y), _stream(stream)), self.ctx)
        return y


def batch_items(mats, nrhs, device="cuda"):
    """(ctypes array of pp_batch_item, device tensors to keep alive)."""
    items = (BatchItem * len(mats))()
    keep = []
    for i, A in enumerate(mats):
        rp, ci, va = to_device_csr(A, device)
        keep.append((rp, ci, va))
        items[i] = BatchItem(A.n, int(A.nnz), _ptr(rp), _ptr(ci), _ptr(va), int(nrhs[i]))
    return items, keep


def batch_autotune(mats, nrhs, device="cuda", stream=None, **options):
    """Time the batch's degree step in every applicable layout
    (pp_batch_autotune); returns (format name, list of per-layout results)."""
    torch = _torch()
    opts = make_options(**options)
    items, keep = batch_items(mats, nrhs, device)
    nbytes = ctypes.c_size_t()
    _check(lib().pp_batch_autotune_workspace_size(ctypes.cast(items, _vp), len(mats), ctypes.byref(opts),
                                                  ctypes.byref(nbytes)))
    ws = torch.empty(max(256, int(nbytes.value)), dtype=torch.uint8, device=device)
    ent = (TuneEntry * 4)()
    cnt = ctypes.c_int()
    _check(lib().pp_batch_autotune(ctypes.cast(items, _vp), len(mats), ctypes.byref(opts), _ptr(ws), ws.numel(), ent,
                                   4, ctypes.byref(cnt), _stream(stream)))
    del ws, keep
    return FORMAT_NAME.get(opts.format, "sell"), [ent[i].as_dict() for i in range(cnt.value)]


class BatchSolver:
    """Many SPD instances (each with 1..8 right-hand sides) solved together
    by one set of persistent launches (pp_batch_setup / pp_batch_solve)."""

    def __init__(self, mats, nrhs, device="cuda", stream=None, **options):
        torch = _torch()
        self.opts = make_options(**options)
        self.nrhs = [int(r) for r in nrhs]
        self.sizes = [int(A.n) for A in mats]
        items, keep = batch_items(mats, self.nrhs, device)
        self._items = items
        nbytes = ctypes.c_size_t()
        _check(lib().pp_batch_workspace_size(ctypes.cast(items, _vp), len(mats), ctypes.byref(self.opts),
                                             ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        ctx = _vp()
        _check(lib().pp_batch_setup(ctypes.byref(ctx), ctypes.cast(items, _vp), len(mats), ctypes.byref(self.opts),
                                    _ptr(self.workspace), self.workspace.numel(), _stream(stream)))
        self.ctx = ctx
        del keep  # the matrices are copied into the workspace at setup
        self.device = torch.device(device)
        self.ncols = sum(self.nrhs)
        self.offsets = np.concatenate([[0], np.cumsum([n * r for n, r in zip(self.sizes, self.nrhs)])]).astype(np.int64)

    def intervals(self, abx=None) -> np.ndarray:
        out = np.zeros((self.ncols, 3))
        inp = None if abx is None else np.ascontiguousarray(abx, dtype=np.float64).reshape(self.ncols, 3)
        _check(lib().pp_batch_intervals(self.ctx, _vp(out.ctypes.data), None if inp is None else _vp(inp.ctypes.data)),
               self.ctx)
        return out

    def features(self) -> np.ndarray:
        f = np.zeros((len(self.sizes), BATCH_NFEAT))
        _check(lib().pp_batch_features(self.ctx, _vp(f.ctypes.data)), self.ctx)
        return f

    def pack(self, blocks) -> "object":
        """Concatenate per-instance (n_i, nrhs_i) arrays into one device vector."""
        torch = _torch()
        flat = np.concatenate([np.ascontiguousarray(b, dtype=np.float64).reshape(-1) for b in blocks])
        return torch.as_tensor(flat, device=self.device)

    def unpack(self, x):
        h = x.detach().cpu().numpy()
        return [h[self.offsets[i]:self.offsets[i + 1]].reshape(self.sizes[i], self.nrhs[i])
                for i in range(len(self.sizes))]

    def solve(self, b, x=None, stream=None, allow=(PP_OK, PP_MAXIT)):
        torch = _torch()
        if x is None:
            x = torch.zeros_like(b)
        it = np.zeros(self.ncols, dtype=np.int32)
        stv = np.zeros(self.ncols, dtype=np.int32)
        st = Stats()
        rc = lib().pp_batch_solve(self.ctx, _ptr(b), _ptr(x), _vp(it.ctypes.data), _vp(stv.ctypes.data),
                                  ctypes.byref(st), _stream(stream))
        _check(rc, self.ctx, allow)
        d = st.as_dict()
        d["status"] = rc
        return x, it, stv, d

    def time_step(self, reps: int = 5, stream=None) -> float:
        """Microseconds per degree step of p_k over all columns (pp_batch_time_step)."""
        us = ctypes.c_double()
        _check(lib().pp_batch_time_step(self.ctx, int(reps), ctypes.byref(us), _stream(stream)), self.ctx)
        return us.value

    def close(self):
        if getattr(self, "ctx", None):
            lib().pp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_NIN, MLP_NHID, MLP_NOUT, MLP_NPARAM = 8, 128, 3, 19720


class Mlp:
    """The interval/xi predictor: forward, gradient and Adam steps run in the
    library's tensor-core kernels (pp_mlp_*)."""

    def __init__(self, max_batch: int = 4096, seed: int = 0, device="cuda"):
        torch = _torch()
        nbytes = ctypes.c_size_t()
        _check(lib().pp_mlp_workspace_size(int(max_batch), ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        h = _vp()
        _check(lib().pp_mlp_create(ctypes.byref(h), int(max_batch), int(seed), _ptr(self.workspace),
                                   self.workspace.numel()))
        self.h = h
        self.device = torch.device(device)
        self.max_batch = int(max_batch)

    def params(self, new=None) -> np.ndarray:
        out = np.zeros(MLP_NPARAM, dtype=np.float32)
        inp = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        _check(lib().pp_mlp_params(self.h, _vp(out.ctypes.data), None if inp is None else _vp(inp.ctypes.data)))
        return out if new is None else inp

    def _f32(self, a):
        torch = _torch()
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=self.device)

    def forward(self, x) -> np.ndarray:
        xt = self._f32(x)
        B = xt.shape[0]
        y = _torch().empty((B, MLP_NOUT), dtype=_torch().float32, device=self.device)
        _check(lib().pp_mlp_forward(self.h, _ptr(xt), _ptr(y), B, _stream(None)))
        return y.cpu().numpy()

    def grad(self, x, t):
        xt, tt = self._f32(x), self._f32(t)
        loss = ctypes.c_float()
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(lib().pp_mlp_grad(self.h, _ptr(xt), _ptr(tt), xt.shape[0], _vp(ctypes.addressof(loss)),
                                 _vp(g.ctypes.data), _stream(None)))
        return float(loss.value), g

    def train_step(self, x, t, lr: float) -> float:
        xt, tt = self._f32(x), self._f32(t)
        loss = ctypes.c_float()
        _check(lib().pp_mlp_train_step(self.h, _ptr(xt), _ptr(tt), xt.shape[0], float(lr),
                                       _vp(ctypes.addressof(loss)), _stream(None)))
        return float(loss.value)

    def close(self):
        if getattr(self, "h", None):
            lib().pp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
