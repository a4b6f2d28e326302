"""CPU FP64 oracle for the slab factor+solve path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and the two share no code: the only common
module is the seeded input generator, which holds none of the method's
arithmetic.

Contents
  * ``assemble`` / ``matvec`` / ``residual``: the five/seven-point operator
    (Sec. 2.1, eq. "discretiation", with the operator sign of eq. "var_helm")
    in CSR form, from the plain C library ``oracle.c``.
  * ``BandLU``: banded LU in the natural ordering (no pivoting for the SPD
    kinds, partial pivoting for Helmholtz) -- the plain definition u = A^-1 f.
  * ``dense_solve``: naive dense LU (separate C code), the brute-force check.
  * The slab method in the paper's own order and notation, in FP64 with
    library solves as steps: index sets I_1, I_2, ... (Sec. 2.2), the reduced
    blocks T (Sec. 3.1, eqs. T11-T35), the reduced load f~ (eqs. f1-f5), the
    sweeping build and solve (Sec. 4, Algorithms 1 and 2), the interior
    back-solve (eq. usol_even) and their composition (Algorithms 3 and 4).
  * ``schur_dense``: the exact Schur complement A_II - A_IJ A_JJ^-1 A_JI of the
    dense matrix, the invariant the assembled T must equal.
  * ``kappa_gradient``: dL/dkappa = -lam^T (dA/dkappa) u for the diffusion and convection kinds,
    lam solving A^T lam = dL/du (``adjoint_gradient``: a banded LU of the transposed matrix for
    the nonsymmetric convection kind).
  * ``boundary_lift``: non-zero Dirichlet data moved into the load of the interior system.
  * ``recovery`` (submodule): randomized recovery of a rank-structured block of T from products
    with it and its transpose (Sec. 3.3), as a HODLR matrix by the peeling scheme.

Readings of the paper used here (the paper is silent or garbled on these):
  b is the interface spacing (interfaces at x = q b, slab interiors b-1 wide);
  Dirichlet data are eliminated, so the interfaces are q = 1..n/b-1; the
  stencil is (A u)_P = h^-2 sum k_PQ (u_P - u_Q) + q_P u_P with k_PQ the mean
  of the two node values of kappa and q_P = -(omega/c_P)^2 for Helmholtz;
  eq. T31 is read as A31 - A32 A22^-1 A21 and eq. T35 as A35 - A34 A44^-1 A45;
  Algorithm 1's loop runs over every interface after the first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

POISSON, DIFFUSION, HELMHOLTZ, CONVECTION = 0, 1, 2, 3
PIVOTED_KINDS = (HELMHOLTZ, CONVECTION)     # banded LU with partial pivoting (indefinite / nonsymmetric)

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_nnz_bound.restype = _i64
            L.orc_nnz_bound.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_assemble.restype = _i64
            L.orc_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                       ctypes.c_double, _dp, _lp, _lp, _dp]
            L.orc_csr_matvec.restype = None
            L.orc_csr_matvec.argtypes = [_i64, _lp, _lp, _dp, ctypes.c_int, _dp, _dp]
            L.orc_band_ld.restype = _i64
            L.orc_band_ld.argtypes = [_i64, ctypes.c_int]
            L.orc_band_from_csr.restype = None
            L.orc_band_from_csr.argtypes = [_i64, _i64, ctypes.c_int, _lp, _lp, _dp, _dp]
            L.orc_band_lu.restype = ctypes.c_int
            L.orc_band_lu.argtypes = [_i64, _i64, ctypes.c_int, _dp, _lp]
            L.orc_band_solve.restype = None
            L.orc_band_solve.argtypes = [_i64, _i64, ctypes.c_int, _dp, _lp, ctypes.c_int, _dp]
            L.orc_dense_solve.restype = ctypes.c_int
            L.orc_dense_solve.argtypes = [_i64, _dp, ctypes.c_int, _dp]
            L.orc_kappa_gradient.restype = None
            L.orc_kappa_gradient.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.orc_boundary_lift.restype = None
            L.orc_boundary_lift.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                            ctypes.c_void_p, _dp]
            L.orc_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def threads() -> int:
    return int(lib().orc_threads())


# ----------------------------------------------------------------------------- operator

class CSR:
    """Assembled sparse matrix (rows sorted, FP64)."""

    def __init__(self, N, rowptr, col, val):
        self.N, self.rowptr, self.col, self.val = N, rowptr, col, val

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        y = np.empty_like(x)
        lib().orc_csr_matvec(self.N, _p(self.rowptr, _lp), _p(self.col, _lp), _p(self.val),
                             x.shape[0], _p(x), _p(y))
        return y

    def dense(self) -> np.ndarray:
        A = np.zeros((self.N, self.N))
        for i in range(self.N):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def submatrix(self, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
        """Dense A[rows][:, cols] (rows/cols are sorted index arrays)."""
        pos = -np.ones(self.N, dtype=np.int64)
        pos[cols] = np.arange(len(cols))
        out = np.zeros((len(rows), len(cols)))
        for a, i in enumerate(rows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            c = pos[self.col[s:e]]
            keep = c >= 0
            out[a, c[keep]] = self.val[s:e][keep]
        return out

    def transpose(self) -> "CSR":
        """A^T as CSR (rows sorted)."""
        rows = np.repeat(np.arange(self.N, dtype=np.int64), np.diff(self.rowptr))
        order = np.lexsort((rows, self.col))
        counts = np.bincount(self.col, minlength=self.N)
        rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return CSR(self.N, rp, rows[order].copy(), self.val[order].copy())

    def sub_csr(self, idx: np.ndarray) -> "CSR":
        """Principal submatrix A[idx][:, idx] as CSR, idx sorted."""
        pos = -np.ones(self.N, dtype=np.int64)
        pos[idx] = np.arange(len(idx))
        rp = [0]
        cols, vals = [], []
        for i in idx:
            s, e = self.rowptr[i], self.rowptr[i + 1]
            c = pos[self.col[s:e]]
            keep = c >= 0
            cols.append(c[keep])
            vals.append(self.val[s:e][keep])
            rp.append(rp[-1] + int(keep.sum()))
        return CSR(len(idx), np.asarray(rp, dtype=np.int64), np.concatenate(cols).astype(np.int64),
                   np.concatenate(vals).astype(np.float64))


def _node_arrays(dim, n, kind, kappa, c):
    nodes = (n + 1) ** dim
    kap = np.ones(nodes) if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    cc = np.ones(nodes) if c is None else np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
    assert kap.size == nodes and cc.size == nodes
    return kap, cc


def assemble(dim: int, n: int, kind: int, kappa=None, c=None, omega: float = 0.0, beta=None) -> CSR:
    """CSR assembly of the finite-difference matrix A (natural order, x fastest).  beta: the
    velocity components at the nodes, shape (dim, (n+1)^d), for the convection kind."""
    kap, cc = _node_arrays(dim, n, kind, kappa, c)
    nodes = (n + 1) ** dim
    if kind == CONVECTION:
        bet = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1)
        assert bet.size == dim * nodes
    else:
        bet = np.zeros(1)
    N = (n - 1) ** dim
    nb = int(lib().orc_nnz_bound(dim, n))
    rowptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(nb, dtype=np.int64)
    val = np.zeros(nb, dtype=np.float64)
    nnz = lib().orc_assemble(dim, n, kind, _p(kap), _p(cc), float(omega), _p(bet), _p(rowptr, _lp),
                             _p(col, _lp), _p(val))
    return CSR(N, rowptr, col[:nnz].copy(), val[:nnz].copy())


def boundary_lift(dim: int, n: int, kind: int, g: np.ndarray, f=None, kappa=None) -> np.ndarray:
    """Load of the interior system for Dirichlet data g (rows = right-hand sides, all (n+1)^d
    nodes): f + h^-2 sum over boundary neighbours Q of k_PQ g_Q (Sec. 1.1 with u = g on the
    boundary, the boundary unknowns eliminated from the interior rows)."""
    if kind == CONVECTION:
        raise NotImplementedError("boundary lift: symmetric kinds only")
    kap, _ = _node_arrays(dim, n, kind, kappa, None)
    G = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64)
    k = G.shape[0]
    assert G.shape[1] == (n + 1) ** dim
    out = np.empty((k, (n - 1) ** dim))
    F = None if f is None else np.ascontiguousarray(np.atleast_2d(f), dtype=np.float64)
    lib().orc_boundary_lift(dim, n, kind, _p(kap), k, _p(G), None if F is None else F.ctypes.data, _p(out))
    return out


def assemble_problem(p) -> CSR:
    return assemble(p.dim, p.n, p.kind, p.kappa, p.c, p.omega, getattr(p, "beta", None))


def residual(A: CSR, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """r = f - A u in FP64 (rows = right-hand sides)."""
    return np.atleast_2d(f) - A.matvec(u)


def relres(A: CSR, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """||A u - f||_2 / ||f||_2 per right-hand side (Sec. 6.1 relerr_res)."""
    r = residual(A, u, f)
    return np.linalg.norm(r, axis=1) / np.linalg.norm(np.atleast_2d(f), axis=1)


# ----------------------------------------------------------------------------- banded LU

class BandLU:
    """Banded LU of an assembled matrix in its own ordering.

    w is the half-bandwidth (for the natural ordering of the full grid,
    (n-1)^(d-1)); pivot selects partial pivoting.
    """

    def __init__(self, A: CSR, w: int, pivot: bool):
        self.N, self.w, self.pivot = A.N, int(w), int(bool(pivot))
        ld = int(lib().orc_band_ld(self.w, self.pivot))
        self.ab = np.empty(self.N * ld, dtype=np.float64)
        lib().orc_band_from_csr(self.N, self.w, self.pivot, _p(A.rowptr, _lp), _p(A.col, _lp),
                                _p(A.val), _p(self.ab))
        self.ipiv = np.zeros(self.N, dtype=np.int64)
        self.info = int(lib().orc_band_lu(self.N, self.w, self.pivot, _p(self.ab), _p(self.ipiv, _lp)))
        if self.info:
            raise np.linalg.LinAlgError(f"banded LU: zero pivot at column {self.info - 1}")

    def solve(self, F: np.ndarray) -> np.ndarray:
        X = np.array(np.atleast_2d(F), dtype=np.float64, order="C", copy=True)
        lib().orc_band_solve(self.N, self.w, self.pivot, _p(self.ab), _p(self.ipiv, _lp),
                             X.shape[0], _p(X))
        return X


def solve(p, f=None) -> np.ndarray:
    """u = A^-1 f by the banded LU of the whole grid (the plain definition)."""
    A = assemble_problem(p)
    lu = BandLU(A, (p.n - 1) ** (p.dim - 1), pivot=(p.kind in PIVOTED_KINDS))
    return lu.solve(p.f if f is None else f)


def solve_transposed(p, g) -> np.ndarray:
    """lam = A^-T g by the banded LU of the transposed matrix (the adjoint system)."""
    At = assemble_problem(p).transpose()
    return BandLU(At, (p.n - 1) ** (p.dim - 1), pivot=(p.kind in PIVOTED_KINDS)).solve(g)


def dense_solve(A: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Naive dense LU with partial pivoting (separate C code), k right-hand sides."""
    a = np.array(A, dtype=np.float64, order="C", copy=True)
    X = np.array(np.atleast_2d(F), dtype=np.float64, order="C", copy=True)
    info = lib().orc_dense_solve(a.shape[0], _p(a), X.shape[0], _p(X))
    if info:
        raise np.linalg.LinAlgError("dense LU: singular")
    return X


# ----------------------------------------------------------------------------- slab method

def index_sets(dim: int, n: int, b: int) -> List[np.ndarray]:
    """The paper's index vectors I_2, I_3, ..., I_{2 n/b} (Sec. 2.2, Fig. 1).

    Odd sets are interfaces (the grid planes x = q b, q = 1..n/b-1), even sets
    the slab interiors (x strictly between two interfaces).  I_1 and the last
    odd set lie on the Dirichlet boundary and are eliminated, so the list
    starts with I_2.  Each set is sorted in the natural order (x fastest), so
    an interface plane is ordered by y (then z).  Returned as
    [I_2, I_3, I_4, ...]: entry 2t is slab t, entry 2q-1 is interface q.
    """
    if b < 2 or n % b:
        raise ValueError("b must divide n and be >= 2")
    m = n - 1
    x = (np.arange((n - 1) ** dim) % m) + 1           # x coordinate of each unknown
    sets = []
    ns = n // b
    for t in range(ns):
        sets.append(np.nonzero((x > t * b) & (x < (t + 1) * b))[0])
        if t + 1 < ns:
            sets.append(np.nonzero(x == (t + 1) * b)[0])
    return sets


def _slab_solver(A: CSR, J: np.ndarray, dim: int, n: int, b: int, pivot: bool):
    """Factor of the slab-interior block A_JJ (banded in its natural order)."""
    width = (b - 1) * (n - 1) ** (dim - 2) if dim == 3 else (b - 1)
    return BandLU(A.sub_csr(J), width, pivot)


def reduced_system(A: CSR, dim: int, n: int, b: int, pivot: bool = False):
    """Blocks of the reduced matrix T (Sec. 3.1, eqs. T11-T35).

    Returns (Tdiag, Tsub, Tsup): Tdiag[q] = T_{2q+1,2q+1}, Tsub[q] = T_{2q+3,2q+1}
    and Tsup[q] = T_{2q+1,2q+3} for interfaces q = 0..N_I-1 (0-based), i.e.
      T_ii   = A_ii - A_{i,i-1} A_{i-1,i-1}^-1 A_{i-1,i} - A_{i,i+1} A_{i+1,i+1}^-1 A_{i+1,i},
      T_i,i+2 = A_{i,i+2} - A_{i,i+1} A_{i+1,i+1}^-1 A_{i+1,i+2},
    with i odd and the even blocks the slab interiors.
    """
    sets = index_sets(dim, n, b)
    ns = n // b
    ni = ns - 1
    slabs = [sets[2 * t] for t in range(ns)]
    ifaces = [sets[2 * q + 1] for q in range(ni)]
    Tdiag = [A.submatrix(I, I) for I in ifaces]
    Tsub, Tsup = [], []
    for q in range(ni - 1):
        Tsup.append(A.submatrix(ifaces[q], ifaces[q + 1]))
        Tsub.append(A.submatrix(ifaces[q + 1], ifaces[q]))
    for t in range(ns):
        J = slabs[t]
        nb = [q for q in (t - 1, t) if 0 <= q < ni]       # interfaces bordering slab t
        if not nb:
            continue
        lu = _slab_solver(A, J, dim, n, b, pivot)
        AJI = np.concatenate([A.submatrix(J, ifaces[q]) for q in nb], axis=1)
        X = lu.solve(AJI.T).T                               # A_JJ^-1 A_JI
        off = 0
        cols = {}
        for q in nb:
            cols[q] = slice(off, off + len(ifaces[q]))
            off += len(ifaces[q])
        for qa in nb:
            AIJ = A.submatrix(ifaces[qa], J)
            for qb in nb:
                blk = AIJ @ X[:, cols[qb]]
                if qa == qb:
                    Tdiag[qa] -= blk
                elif qb == qa + 1:
                    Tsup[qa] -= blk
                else:
                    Tsub[qb] -= blk
    return Tdiag, Tsub, Tsup


def reduced_rhs(A: CSR, f: np.ndarray, dim: int, n: int, b: int, pivot: bool = False) -> List[np.ndarray]:
    """Equivalent load on the interfaces (eqs. f1-f5): f~_i = f_i - sum A_{i,j} A_jj^-1 f_j.

    f has shape (k, N); returns one (k, |I_q|) array per interface.
    """
    sets = index_sets(dim, n, b)
    ns = n // b
    ni = ns - 1
    f = np.atleast_2d(f)
    ft = [f[:, sets[2 * q + 1]].copy() for q in range(ni)]
    for t in range(ns):
        J = sets[2 * t]
        lu = _slab_solver(A, J, dim, n, b, pivot)
        y = lu.solve(f[:, J])                               # A_JJ^-1 f_J, rows = rhs
        for q in (t - 1, t):
            if 0 <= q < ni:
                ft[q] -= (A.submatrix(sets[2 * q + 1], J) @ y.T).T
    return ft


def sweep_build(Tdiag, Tsub, Tsup) -> List[np.ndarray]:
    """Algorithm 1: S_1 = T_11, S_{j+1} = T_{j+1,j+1} - T_{j+1,j} S_j^-1 T_{j,j+1}; store S_j^-1."""
    Sinv = [np.linalg.inv(Tdiag[0])]
    for j in range(1, len(Tdiag)):
        S = Tdiag[j] - Tsub[j - 1] @ Sinv[j - 1] @ Tsup[j - 1]
        Sinv.append(np.linalg.inv(S))
    return Sinv


def sweep_solve(Tsub, Tsup, Sinv, ft: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Algorithm 2 on k right-hand sides (each ft[q] is (k, s)): returns u~ per interface."""
    x = [np.array(v, dtype=np.float64).T.copy() for v in ft]      # columns = rhs
    N = len(x)
    for j in range(N - 1):                                          # forward elimination
        x[j + 1] = x[j + 1] - Tsub[j] @ (Sinv[j] @ x[j])
    for j in range(N):                                              # block-diagonal solve
        x[j] = Sinv[j] @ x[j]
    for j in range(N - 2, -1, -1):                                  # back substitution
        x[j] = x[j] - Sinv[j] @ (Tsup[j] @ x[j + 1])
    return [v.T.copy() for v in x]


def interior_solve(A: CSR, f: np.ndarray, ut: Sequence[np.ndarray], dim: int, n: int, b: int,
                   pivot: bool = False) -> np.ndarray:
    """Eq. usol_even: u_i = A_ii^-1 (f_i - A_{i,i-1} u_{i-1} - A_{i,i+1} u_{i+1}) per slab."""
    sets = index_sets(dim, n, b)
    ns = n // b
    ni = ns - 1
    f = np.atleast_2d(f)
    u = np.zeros_like(f, dtype=np.float64)
    for q in range(ni):
        u[:, sets[2 * q + 1]] = ut[q]
    for t in range(ns):
        J = sets[2 * t]
        rhs = f[:, J].copy()
        for q in (t - 1, t):
            if 0 <= q < ni:
                rhs -= (A.submatrix(J, sets[2 * q + 1]) @ np.atleast_2d(ut[q]).T).T
        u[:, J] = _slab_solver(A, J, dim, n, b, pivot).solve(rhs)
    return u


def slab_solve(p, f=None) -> Tuple[np.ndarray, dict]:
    """Algorithms 3 and 4 with exact dense T: factor, then solve for p.f (or f)."""
    A = assemble_problem(p)
    piv = p.kind in PIVOTED_KINDS
    Td, Tl, Tu = reduced_system(A, p.dim, p.n, p.b, piv)
    Sinv = sweep_build(Td, Tl, Tu)
    f = p.f if f is None else f
    ft = reduced_rhs(A, f, p.dim, p.n, p.b, piv)
    ut = sweep_solve(Tl, Tu, Sinv, ft)
    u = interior_solve(A, f, ut, p.dim, p.n, p.b, piv)
    return u, dict(Tdiag=Td, Tsub=Tl, Tsup=Tu, Sinv=Sinv, ftilde=ft, utilde=ut)


def schur_dense(Ad: np.ndarray, I: np.ndarray, J: np.ndarray) -> np.ndarray:
    """Exact Schur complement A_II - A_IJ A_JJ^-1 A_JI of a dense matrix."""
    return Ad[np.ix_(I, I)] - Ad[np.ix_(I, J)] @ np.linalg.solve(Ad[np.ix_(J, J)], Ad[np.ix_(J, I)])


# ----------------------------------------------------------------------------- gradient

def kappa_gradient(dim: int, n: int, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/dkappa at the (n+1)^d nodes from the state u and adjoint lam (one pair)."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
    g = np.zeros((n + 1) ** dim)
    lib().orc_kappa_gradient(dim, n, _p(u), _p(lam), _p(g))
    return g.reshape((n + 1,) * dim)


def adjoint_gradient(p, u_target: np.ndarray):
    """Loss L = ||u - u_t||^2 for the diffusion or convection problem p: returns
    (L, u, lam, dL/dkappa), lam solving A^T lam = dL/du = 2 (u - u_t)."""
    A = assemble_problem(p)
    w = (p.n - 1) ** (p.dim - 1)
    piv = p.kind in PIVOTED_KINDS
    lu = BandLU(A, w, pivot=piv)
    u = lu.solve(p.f)
    r = u - np.atleast_2d(u_target)
    L = float(np.sum(r * r))
    if p.kind == CONVECTION:
        lam = BandLU(A.transpose(), w, pivot=piv).solve(2.0 * r)
    else:
        lam = lu.solve(2.0 * r)         # A is symmetric: A^T lam = dL/du
    return L, u, lam, kappa_gradient(p.dim, p.n, u, lam)
