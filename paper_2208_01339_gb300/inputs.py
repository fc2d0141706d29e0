"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only builds *data*: sparse SPD test matrices, right-hand sides
and the synthetic fracture network.  It holds none of the method's
arithmetic (no Chebyshev coefficients, no recurrence, no Krylov step, no
Schur-complement product), so the oracle and the GPU path can both read the
arrays it returns without sharing any method code.

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output i of stream s under seed S is
    key = mix(S ^ mix(s + C0)),   u64_i = mix(key + (i + 1) * GOLDEN)
where mix(z) is the SplitMix64 finaliser.  Uniform doubles take the top 53
bits; normals use Box-Muller on consecutive uniform pairs.

Workloads (all synthetic; the paper's own matrices are not available):
  * ``diagonal(n)``          -- A_ii = i, the diagonal test of the paper's
                                Section 2.4 (Table 1).
  * ``poisson3d(N)``         -- 7-point Laplacian on an N^3 grid, Dirichlet
                                boundary eliminated (stands in for the
                                paper's structured-mesh SPD matrices).
  * ``diffusion3d(N, s, S)`` -- variable-coefficient 7-point diffusion with
                                lognormal(0, s) cell conductivities and
                                harmonic-mean faces.
  * ``fracture_network(...)``-- synthetic DFN blocks (A, C, B = C + E, G^h,
                                G^u) with the block properties of the paper's
                                Section 4.1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C0 = np.uint64(0x632BE59BD9B4E019)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Named stream ids (documented so that every consumer draws the same numbers).
STREAM_RHS = 0
STREAM_CONDUCTIVITY = 1
STREAM_RHS_NORMAL = 2
STREAM_LANCZOS = 3
STREAM_FRACTURE = 4
STREAM_TRACE = 5
STREAM_BATCH = 6
STREAM_GENERAL = 8  # general fracture blocks (mesh jitter, diagonals, coefficients, numbering)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        inner = _mix(np.uint64(stream) + _C0)
        return _mix(np.uint64(seed) ^ inner)


def raw_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    key = stream_key(seed, stream)
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + i * _GOLDEN)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) doubles, 53-bit resolution."""
    return (raw_u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm(seed: int, stream: int, n: int, half_width: float = 1.0) -> np.ndarray:
    """U[-w, w) doubles."""
    return (2.0 * uniform(seed, stream, n) - 1.0) * half_width


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on uniform pairs (2i, 2i+1)."""
    u = uniform(seed, stream, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class CSR:
    """Square sparse matrix in CSR, int32 indices, float64 values, columns ascending."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """Plain product, used only to build right-hand sides such as A*ones."""
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        y = np.zeros(self.n)
        np.add.at(y, rows, self.val * x[self.col])
        return y


def diagonal(n: int) -> CSR:
    """A = diag(1, 2, ..., n): the diagonal test of the paper (Table 1)."""
    rowptr = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    val = np.arange(1, n + 1, dtype=np.float64)
    return CSR(n, rowptr, col, val, {"kind": "diagonal"})


def _stencil7(N: int, face):
    """Assemble a 7-point operator on an N^3 grid (x fastest).

    ``face(axis, side)`` returns, for every cell, the coefficient of the face
    towards the neighbour at offset side (-1/+1) along ``axis`` (0=x,1=y,2=z),
    with boundary faces included.  Off-diagonals are -face for interior
    faces; the diagonal is the sum of all six faces (Dirichlet boundary
    eliminated).
    """
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    coords = (ix, iy, iz)
    strides = (1, N, N * N)
    # column slots in ascending order: -z, -y, -x, diag, +x, +y, +z
    order = [(2, -1), (1, -1), (0, -1), None, (0, 1), (1, 1), (2, 1)]
    cols = np.empty((n, 7), dtype=np.int32)
    vals = np.empty((n, 7), dtype=np.float64)
    mask = np.ones((n, 7), dtype=bool)
    diag = np.zeros(n)
    for slot, o in enumerate(order):
        if o is None:
            continue
        axis, side = o
        f = face(axis, side)
        diag += f
        c = coords[axis]
        inside = (c + side >= 0) & (c + side < N)
        cols[:, slot] = idx + side * strides[axis]
        vals[:, slot] = -f
        mask[:, slot] = inside
    cols[:, 3] = idx
    vals[:, 3] = diag
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[mask].astype(np.int32)
    val = vals[mask]
    return rowptr.astype(np.int32), col, val


def poisson3d(N: int) -> CSR:
    """7-point Laplacian (diag 6, off-diagonal -1) on N^3, Dirichlet eliminated."""
    one = np.ones(N ** 3)
    rowptr, col, val = _stencil7(N, lambda axis, side: one)
    return CSR(N ** 3, rowptr, col, val, {"kind": "poisson3d", "N": N})


def conductivity(N: int, sigma_ln: float, seed: int) -> np.ndarray:
    """Cell conductivities exp(sigma_ln * N(0,1)), one per cell."""
    return np.exp(sigma_ln * normal(seed, STREAM_CONDUCTIVITY, N ** 3))


def diffusion3d(N: int, sigma_ln: float, seed: int) -> CSR:
    """Variable-coefficient 7-point diffusion on N^3.

    Interior face between cells p, q: harmonic mean 2 k_p k_q / (k_p + k_q).
    Boundary face: k_p (the eliminated Dirichlet node sits one spacing away,
    as in the vertex-centred Laplacian), so sigma_ln = 0 gives exactly
    ``poisson3d(N)``.  No 1/h^2 factor (the method is scale-invariant).
    """
    kap = conductivity(N, sigma_ln, seed)
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    coords = (idx % N, (idx // N) % N, idx // (N * N))
    strides = (1, N, N * N)

    def face(axis, side):
        c = coords[axis]
        inside = (c + side >= 0) & (c + side < N)
        nb = np.where(inside, idx + side * strides[axis], idx)
        kq = kap[nb]
        h = 2.0 * kap * kq / (kap + kq)
        return np.where(inside, h, kap)

    rowptr, col, val = _stencil7(N, face)
    return CSR(n, rowptr, col, val, {"kind": "diffusion3d", "N": N, "sigma_ln": sigma_ln, "seed": seed})


def rhs_ones_plus_noise(A: CSR, seed: int = 0, noise: float = 1e-3) -> np.ndarray:
    """b = A * ones + U[-noise, noise) (the 32^3 Poisson workload)."""
    return A.matvec(np.ones(A.n)) + uniform_pm(seed, STREAM_RHS, A.n, noise)


def rhs_normal(n: int, seed: int) -> np.ndarray:
    return normal(seed, STREAM_RHS_NORMAL, n)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """U[-1, 1) right-hand side (the diagonal test)."""
    return uniform_pm(seed, STREAM_RHS, n, 1.0)


def lanczos_start(n: int, seed: int) -> np.ndarray:
    """The Lanczos start vector both sides draw: U[-1,1) on stream STREAM_LANCZOS.

    The CUDA path generates the same numbers on the device from the same
    SplitMix64 definition; this copy is for the oracle.
    """
    return uniform_pm(seed, STREAM_LANCZOS, n, 1.0)


def random_spd(n: int, seed: int, cond: float = 100.0) -> np.ndarray:
    """Small dense SPD matrix with eigenvalues log-spaced in [1, cond]."""
    g = normal(seed, STREAM_BATCH, n * n).reshape(n, n)
    q, _ = np.linalg.qr(g)
    lam = np.logspace(0.0, np.log10(cond), n)
    return (q * lam) @ q.T


def dense_to_csr(D: np.ndarray, drop: float = 0.0) -> CSR:
    n = D.shape[0]
    mask = np.abs(D) > drop
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    rows, cols = np.nonzero(mask)
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), D[rows, cols].astype(np.float64),
               {"kind": "dense"})


# ---------------------------------------------------------------------------
# Synthetic discrete fracture network (Section 4.1 block properties)
# ---------------------------------------------------------------------------


def _coo_to_csr(nrows: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> tuple:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=nrows)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


@dataclass
class RectCSR:
    """Rectangular CSR (nrows x ncols)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols))
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        np.add.at(d, (rows, self.col), self.val)
        return d


@dataclass
class FractureNetwork:
    """Blocks of the DFN saddle-point system (the paper's Eq. algebraic_model).

    Fracture f is an nx[f] x ny[f] grid of interior nodes (x fastest), its
    unknowns occupy h-indices [offset[f], offset[f+1]).  A is block diagonal
    with A_f = T[f] * (2-D 5-point Laplacian, Dirichlet on every side).
    C, B = C + E (n_h x n_u), G^h (n_h x n_h) and G^u (n_u x n_u) are general
    sparse matrices; their transposes CT, BT are stored as well (they are the
    third block row of the permuted system).  q is the forcing term.
    """

    nx: np.ndarray
    ny: np.ndarray
    T: np.ndarray
    offset: np.ndarray
    A: CSR
    C: RectCSR
    B: RectCSR
    CT: RectCSR
    BT: RectCSR
    Gh: CSR
    Gu: CSR
    q: np.ndarray
    alpha: float
    own_node: np.ndarray
    partner_node: np.ndarray
    pair: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_h(self) -> int:
        return int(self.offset[-1])

    @property
    def n_u(self) -> int:
        return int(self.own_node.shape[0])

    @property
    def n_f(self) -> int:
        return int(self.nx.shape[0])


def _laplace5_blocks(nx, ny, T, offset) -> CSR:
    rows_l, cols_l, vals_l = [], [], []
    for f in range(len(nx)):
        mx, my, t, o = int(nx[f]), int(ny[f]), float(T[f]), int(offset[f])
        ix = np.tile(np.arange(mx), my)
        iy = np.repeat(np.arange(my), mx)
        node = o + iy * mx + ix
        rows_l.append(node); cols_l.append(node); vals_l.append(np.full(node.size, 4.0 * t))
        for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            ok = (ix + dx >= 0) & (ix + dx < mx) & (iy + dy >= 0) & (iy + dy < my)
            rows_l.append(node[ok])
            cols_l.append(o + (iy[ok] + dy) * mx + ix[ok] + dx)
            vals_l.append(np.full(int(ok.sum()), -t))
    n = int(offset[-1])
    rowptr, col, val = _coo_to_csr(n, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(vals_l))
    return CSR(n, rowptr, col, val, {"kind": "dfn_A"})


def fracture_network(n_f: int = 200, side_min: float = 5.0, side_max: float = 50.0, h: float = 0.25,
                     trace_min: float = 5.0, trace_max: float = 50.0, trace_fraction: float = 0.05,
                     T_sigma: float = 1.0, alpha: float = 0.5, seed: int = 2,
                     max_traces: int | None = None) -> FractureNetwork:
    """Seeded synthetic DFN with the block structure of the paper's Section 4.1.

    * n_f rectangular fractures, sides U(side_min, side_max) metres, mesh
      size h: round(L/h) - 1 interior nodes per side; transmissivity
      T_f = exp(T_sigma * N(0,1)).
    * A trace couples a random fracture pair (i, j): an axis-aligned run of
      L_t consecutive nodes on each side, L_t = round(U(trace_min,
      trace_max)/h) clipped to fit, matched point by point.  Trace nodes on
      a fracture never overlap.  Each trace point l gives two flux unknowns
      u_{t,i,l}, u_{t,j,l}.
    * C[node_i(l), u_{t,i,l}] = 1 (fracture-local), E[node_j(l), u_{t,i,l}]
      = 1 (its partner), and symmetrically for side j; B = C + E.
    * G^h = sum over trace nodes of e e^T (block-local, SPSD, rank
      deficient); G^u = sum over trace points of the 2x2 all-ones block on
      (u_{t,i,l}, u_{t,j,l}) (global, SPSD).
    * Traces are added until n_u >= trace_fraction * n_h.
    * q ~ N(0,1) on all fracture nodes.
    """
    u = uniform(seed, STREAM_FRACTURE, 3 * n_f)
    Lx = side_min + (side_max - side_min) * u[0::3]
    Ly = side_min + (side_max - side_min) * u[1::3]
    nx = np.maximum(np.rint(Lx / h).astype(np.int64) - 1, 1)
    ny = np.maximum(np.rint(Ly / h).astype(np.int64) - 1, 1)
    T = np.exp(T_sigma * normal(seed, STREAM_FRACTURE + 100, n_f))
    offset = np.zeros(n_f + 1, dtype=np.int64)
    np.cumsum(nx * ny, out=offset[1:])
    n_h = int(offset[-1])
    occupied = [np.zeros(int(nx[f] * ny[f]), dtype=bool) for f in range(n_f)]

    # Draw candidate traces from one long stream; reject overlaps.
    own, partner, pair = [], [], []
    n_u = 0
    draws = uniform(seed, STREAM_TRACE, 8 * 200000)
    d = 0
    n_traces = 0
    target = trace_fraction * n_h
    while n_u < target and d + 8 <= draws.size:
        if max_traces is not None and n_traces >= max_traces:
            break
        w = draws[d:d + 8]
        d += 8
        i = int(w[0] * n_f)
        j = int(w[1] * (n_f - 1))
        if j >= i:
            j += 1
        if n_f < 2:
            break
        L = int(np.rint((trace_min + (trace_max - trace_min) * w[2]) / h))
        L = max(1, min(L, int(max(nx[i], ny[i])), int(max(nx[j], ny[j]))))
        sides = []
        ok = True
        for f, wo, wa, wb in ((i, w[3], w[4], w[5]), (j, w[6], w[4], w[7])):
            mx, my = int(nx[f]), int(ny[f])
            axes = [a for a, m in ((0, mx), (1, my)) if m >= L]
            axis = axes[int(wo * len(axes))]
            if axis == 0:
                iy = int(wb * my)
                ix0 = int(wa * (mx - L + 1))
                loc = iy * mx + ix0 + np.arange(L)
            else:
                ix = int(wb * mx)
                iy0 = int(wa * (my - L + 1))
                loc = (iy0 + np.arange(L)) * mx + ix
            if occupied[f][loc].any():
                ok = False
                break
            sides.append((f, loc))
        if not ok:
            continue
        for f, loc in sides:
            occupied[f][loc] = True
        (fi, li), (fj, lj) = sides
        gi = offset[fi] + li
        gj = offset[fj] + lj
        base = n_u
        ui = base + np.arange(L)
        uj = base + L + np.arange(L)
        own.append(gi); partner.append(gj); pair.append(uj)
        own.append(gj); partner.append(gi); pair.append(ui)
        n_u += 2 * L
        n_traces += 1

    own_node = np.concatenate(own).astype(np.int64) if own else np.zeros(0, np.int64)
    partner_node = np.concatenate(partner).astype(np.int64) if partner else np.zeros(0, np.int64)
    pair_arr = np.concatenate(pair).astype(np.int64) if pair else np.zeros(0, np.int64)
    ucols = np.arange(n_u, dtype=np.int64)
    ones = np.ones(n_u)

    rp, cc, vv = _coo_to_csr(n_h, own_node, ucols, ones)
    Cm = RectCSR(n_h, n_u, rp, cc, vv)
    rp, cc, vv = _coo_to_csr(n_u, ucols, own_node, ones)
    CT = RectCSR(n_u, n_h, rp, cc, vv)
    brow = np.concatenate([own_node, partner_node])
    bcol = np.concatenate([ucols, ucols])
    rp, cc, vv = _coo_to_csr(n_h, brow, bcol, np.ones(2 * n_u))
    Bm = RectCSR(n_h, n_u, rp, cc, vv)
    rp, cc, vv = _coo_to_csr(n_u, bcol, brow, np.ones(2 * n_u))
    BT = RectCSR(n_u, n_h, rp, cc, vv)
    tnodes = np.unique(own_node)
    rp, cc, vv = _coo_to_csr(n_h, tnodes, tnodes, np.ones(tnodes.size))
    Gh = CSR(n_h, rp, cc, vv, {"kind": "dfn_Gh"})
    grow = np.concatenate([ucols, ucols])
    gcol = np.concatenate([ucols, pair_arr])
    rp, cc, vv = _coo_to_csr(n_u, grow, gcol, np.ones(2 * n_u))
    Gu = CSR(n_u, rp, cc, vv, {"kind": "dfn_Gu"})
    A = _laplace5_blocks(nx, ny, T, offset)
    q = normal(seed, STREAM_FRACTURE + 200, n_h)
    return FractureNetwork(nx=nx.astype(np.int32), ny=ny.astype(np.int32), T=T, offset=offset, A=A,
                           C=Cm, B=Bm, CT=CT, BT=BT, Gh=Gh, Gu=Gu, q=q, alpha=float(alpha),
                           own_node=own_node, partner_node=partner_node, pair=pair_arr,
                           meta={"n_traces": n_traces, "seed": seed, "h": h})


def _coo_sum_to_csr(nrows: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> tuple:
    """CSR with repeated (row, col) entries summed in their input order."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    first = np.ones(rows.size, dtype=bool)
    first[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
    starts = np.nonzero(first)[0]
    sums = np.add.reduceat(vals, starts) if vals.size else vals
    return _coo_to_csr(nrows, rows[starts], cols[starts], sums)


def _p1_blocks(nx, ny, T, offset, jitter: float, k_sigma: float, seed: int) -> CSR:
    """P1 finite-element stiffness of -div(k grad h) on each fracture.

    The fracture's node grid, with a boundary ring of Dirichlet nodes around
    the nx x ny interior nodes (eliminated), is moved by jitter * U(-1,1)
    per interior coordinate (grid units; jitter < 1/2 keeps every triangle
    positively oriented) and every cell is split along a random diagonal.
    Each triangle has k = T_f exp(k_sigma N(0,1)).  Element matrices
    k (b_a b_b + c_a c_b) / (4 area) (b, c the edge-normal components).
    Interior node (ix, iy) keeps the index iy*nx + ix of the rectangle, so
    trace nodes are unchanged.  The lower triangle is assembled and mirrored,
    so the matrix is exactly symmetric.
    """
    rows_l, cols_l, vals_l = [], [], []
    ofs = 0
    for f in range(len(nx)):
        mx, my, o = int(nx[f]), int(ny[f]), int(offset[f])
        ex, ey = mx + 2, my + 2
        ncell = (mx + 1) * (my + 1)
        gx = np.tile(np.arange(ex, dtype=np.float64), ey)
        gy = np.repeat(np.arange(ey, dtype=np.float64), ex)
        ix = np.tile(np.arange(ex), ey)
        iy = np.repeat(np.arange(ey), ex)
        inner = (ix >= 1) & (ix <= mx) & (iy >= 1) & (iy <= my)
        ni = int(inner.sum())
        jx = (2.0 * uniform(seed, STREAM_GENERAL, ni, ofs) - 1.0) * jitter
        jy = (2.0 * uniform(seed, STREAM_GENERAL, ni, ofs + ni) - 1.0) * jitter
        ofs += 2 * ni
        gx[inner] += jx
        gy[inner] += jy
        lidx = np.where(inner, (iy - 1) * mx + (ix - 1), -1)
        diag = uniform(seed, STREAM_GENERAL, ncell, ofs) < 0.5
        ofs += ncell
        u = uniform(seed, STREAM_GENERAL, 4 * ncell, ofs)
        ofs += 4 * ncell
        z = np.sqrt(-2.0 * np.log(1.0 - u[0::2])) * np.cos(2.0 * np.pi * u[1::2])  # 2 ncell normals
        cx = np.tile(np.arange(mx + 1), my + 1)
        cy = np.repeat(np.arange(my + 1), mx + 1)
        n00 = cy * ex + cx
        n10 = n00 + 1
        n01 = n00 + ex
        n11 = n01 + 1
        t1 = np.where(diag[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
        t2 = np.where(diag[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
        tri = np.concatenate([t1, t2])
        kt = float(T[f]) * np.exp(k_sigma * z)
        x = gx[tri]
        y = gy[tri]
        b = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], 1)
        c = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], 1)
        area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
        for aa in range(3):
            for bb in range(aa, 3):
                ka = kt * (b[:, aa] * b[:, bb] + c[:, aa] * c[:, bb]) / (4.0 * area)
                ga, gb = lidx[tri[:, aa]], lidx[tri[:, bb]]
                ok = (ga >= 0) & (gb >= 0)
                rows_l.append(o + np.maximum(ga[ok], gb[ok]))
                cols_l.append(o + np.minimum(ga[ok], gb[ok]))
                vals_l.append(ka[ok])
    n = int(offset[-1])
    rp, cc, vv = _coo_sum_to_csr(n, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(vals_l))
    rows = np.repeat(np.arange(n), np.diff(rp))
    strict = rows != cc
    rowptr, col, val = _coo_to_csr(n, np.concatenate([rows, cc[strict]]), np.concatenate([cc, rows[strict]]),
                                   np.concatenate([vv, vv[strict]]))
    return CSR(n, rowptr, col, val, {"kind": "dfn_A_p1"})


def _relabel_network(net: FractureNetwork, new: np.ndarray) -> FractureNetwork:
    """The same network with node i renamed new[i] (a permutation that maps
    every fracture's range onto itself): A, G^h rows and columns, the rows of
    C, B, the columns of C^T, B^T, q and the trace node lists."""
    n = net.n_h

    def rows_of(X):
        r = np.repeat(np.arange(X.nrows if hasattr(X, "nrows") else X.n), np.diff(X.rowptr))
        return r

    def sq(X, kind):
        r = rows_of(X)
        rp, cc, vv = _coo_to_csr(n, new[r], new[X.col], X.val)
        return CSR(n, rp, cc, vv, {"kind": kind})

    def rect_rows(X):
        r = rows_of(X)
        rp, cc, vv = _coo_to_csr(X.nrows, new[r], X.col.astype(np.int64), X.val)
        return RectCSR(X.nrows, X.ncols, rp, cc, vv)

    def rect_cols(X):
        r = rows_of(X)
        rp, cc, vv = _coo_to_csr(X.nrows, r, new[X.col], X.val)
        return RectCSR(X.nrows, X.ncols, rp, cc, vv)

    q = np.empty_like(net.q)
    q[new] = net.q
    return FractureNetwork(nx=net.nx, ny=net.ny, T=net.T, offset=net.offset, A=sq(net.A, net.A.meta.get("kind")),
                           C=rect_rows(net.C), B=rect_rows(net.B), CT=rect_cols(net.CT), BT=rect_cols(net.BT),
                           Gh=sq(net.Gh, "dfn_Gh"), Gu=net.Gu, q=q, alpha=net.alpha, own_node=new[net.own_node],
                           partner_node=new[net.partner_node], pair=net.pair, meta=dict(net.meta))


def general_fracture_network(net: FractureNetwork, jitter: float = 0.25, k_sigma: float = 1.0, seed: int = 11,
                             shuffle: bool = True) -> FractureNetwork:
    """The network `net` with fracture blocks of general form: A_f is the P1
    stiffness of a jittered, randomly split triangulation with lognormal
    coefficients (see _p1_blocks), and with shuffle the nodes of every
    fracture are renumbered by a seeded random permutation (so that the
    given numbering has no band structure).  Traces, C, B, G^h, G^u and q
    are those of `net`, carried along by the renumbering.  The rectangle
    metadata (nx, ny, T) no longer describes A; meta["general"] is set.
    """
    A = _p1_blocks(net.nx, net.ny, net.T, net.offset, jitter, k_sigma, seed)
    out = FractureNetwork(nx=net.nx, ny=net.ny, T=net.T, offset=net.offset, A=A, C=net.C, B=net.B, CT=net.CT,
                          BT=net.BT, Gh=net.Gh, Gu=net.Gu, q=net.q, alpha=net.alpha, own_node=net.own_node,
                          partner_node=net.partner_node, pair=net.pair, meta=dict(net.meta))
    if shuffle:
        u = uniform(seed, STREAM_GENERAL + 1, net.n_h)
        new = np.empty(net.n_h, dtype=np.int64)
        for f in range(net.n_f):
            o, e = int(net.offset[f]), int(net.offset[f + 1])
            new[o:e] = o + np.argsort(np.argsort(u[o:e], kind="stable"), kind="stable")
        out = _relabel_network(out, new)
    out.meta.update({"general": True, "jitter": jitter, "k_sigma": k_sigma, "general_seed": seed,
                     "shuffled": shuffle})
    return out


def with_dense_block(net: FractureNetwork, f: int, seed: int = 13) -> FractureNetwork:
    """The network with A_f replaced by the dense SPD block A_f + g g^T / n_f
    (g ~ N(0,1), seeded): a block whose band cannot be narrowed by any
    reordering.  meta["general"] is set."""
    o, e = int(net.offset[f]), int(net.offset[f + 1])
    nf = e - o
    D = net.A.to_dense()
    g = normal(seed, STREAM_GENERAL + 2, nf)
    blk = D[o:e, o:e] + np.outer(g, g) / nf
    D[o:e, o:e] = 0.5 * (blk + blk.T)
    mask = D != 0.0
    mask[o:e, o:e] = True
    rows, cols = np.nonzero(mask)
    rp, cc, vv = _coo_to_csr(net.n_h, rows, cols, D[rows, cols])
    A = CSR(net.n_h, rp, cc, vv, {"kind": "dfn_A_dense_block"})
    out = FractureNetwork(nx=net.nx, ny=net.ny, T=net.T, offset=net.offset, A=A, C=net.C, B=net.B, CT=net.CT,
                          BT=net.BT, Gh=net.Gh, Gu=net.Gu, q=net.q, alpha=net.alpha, own_node=net.own_node,
                          partner_node=net.partner_node, pair=net.pair, meta=dict(net.meta))
    out.meta.update({"general": True, "dense_block": f})
    return out


def tiny_fracture_network(seed: int = 7) -> FractureNetwork:
    """3 fractures of about 5 x 6 nodes and 3 traces, for dense checks."""
    return fracture_network(n_f=3, side_min=1.4, side_max=1.8, h=0.25, trace_min=0.75, trace_max=1.25,
                            trace_fraction=10.0, seed=seed, max_traces=3)


# ---------------------------------------------------------------------------
# Batched workload: many uneven diffusion instances with several RHS each
# ---------------------------------------------------------------------------


@dataclass
class BatchSpec:
    N: int
    sigma_ln: float
    nrhs: int
    seed: int


def batch_specs(count: int = 64, seed: int = 4, nmin: int = 48, nmax: int = 160, smin: float = 0.5,
                smax: float = 3.0, rmin: int = 1, rmax: int = 8) -> list:
    """Instance i: grid N ~ U{nmin..nmax}, lognormal sigma ~ U[smin, smax],
    nrhs ~ U{rmin..rmax}, matrix seed 1000*seed + i (stream STREAM_BATCH)."""
    u = uniform(seed, STREAM_BATCH + 10, 3 * count)
    out = []
    for i in range(count):
        N = nmin + min(int(u[3 * i] * (nmax - nmin + 1)), nmax - nmin)
        s = smin + (smax - smin) * u[3 * i + 1]
        r = rmin + min(int(u[3 * i + 2] * (rmax - rmin + 1)), rmax - rmin)
        out.append(BatchSpec(N, float(s), r, 1000 * seed + i))
    return out


def batch_instance(spec: BatchSpec) -> CSR:
    return diffusion3d(spec.N, spec.sigma_ln, seed=spec.seed)


def batch_rhs(spec: BatchSpec) -> np.ndarray:
    """N(0,1) right-hand sides, shape (n, nrhs), row-major [row][rhs]."""
    n = spec.N ** 3
    return normal(spec.seed, STREAM_RHS_NORMAL, n * spec.nrhs).reshape(n, spec.nrhs)
