"""Randomized recovery of a rank-structured block from matrix-vector products -- TEST
INFRASTRUCTURE ONLY (part of the CPU oracle; only tests/ may import it).

Sec. 3.3 of the paper forms each block of the reduced matrix T without ever writing it down:
it only applies T (and T^*) to random sketch matrices, Y = T Omega and Z = T^* Psi, and recovers a
hierarchical representation from the samples, which is exact because the blocks are rank
structured (Prop. 1: the coupling between a contiguous run of interface nodes and the rest of
the interface has rank at most 2 (b - 1) in this discretisation).  The paper cites an external
algorithm for the recovery; this module restates the published peeling scheme for hierarchically
off-diagonal low-rank (HODLR) matrices -- level by level from the root, sample the off-diagonal
blocks of the level with sketches supported on one child of every sibling pair, subtract what the
coarser levels already explain, take the range of the samples, then its coefficients from
products with the transpose; the leaves last, with identity sketches.  It uses only the two
products and plain numpy (SVD for the ranges), and reports how many products it spent.

The representation is exact up to rounding when every off-diagonal block of the tree has rank at
most `rank` (the oversampled sketch then spans its range with probability one).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Tuple

import numpy as np


def _boxes(n: int, leaf: int) -> List[List[Tuple[int, int]]]:
    """Contiguous index boxes per level: level 0 is [0, n), each box split into halves until the
    boxes are at most `leaf` long."""
    levels = [[(0, n)]]
    while max(e - s for s, e in levels[-1]) > leaf:
        nxt = []
        for s, e in levels[-1]:
            mid = (s + e) // 2
            nxt += [(s, mid), (mid, e)]
        levels.append(nxt)
    return levels


@dataclass
class HODLR:
    """Off-diagonal blocks M[rows, cols] = U V^T per level and sibling pair, dense leaves."""
    n: int
    levels: List[List[Tuple[int, int]]]
    offdiag: List[List[Tuple[Tuple[int, int], Tuple[int, int], np.ndarray, np.ndarray]]] = field(
        default_factory=list)
    leaves: Dict[Tuple[int, int], np.ndarray] = field(default_factory=dict)
    products: int = 0            # columns of M X plus columns of M^T X spent

    def apply_known(self, X: np.ndarray, upto: int, transpose: bool = False) -> np.ndarray:
        """(sum of the off-diagonal blocks of levels 1..upto-1) X, or its transpose applied."""
        out = np.zeros((self.n, X.shape[1]))
        for lvl in self.offdiag[:max(upto - 1, 0)]:
            for (r0, r1), (c0, c1), U, V in lvl:
                if transpose:
                    out[c0:c1] += V @ (U.T @ X[r0:r1])
                else:
                    out[r0:r1] += U @ (V.T @ X[c0:c1])
        return out

    def dense(self) -> np.ndarray:
        M = np.zeros((self.n, self.n))
        for lvl in self.offdiag:
            for (r0, r1), (c0, c1), U, V in lvl:
                M[r0:r1, c0:c1] = U @ V.T
        for (s, e), D in self.leaves.items():
            M[s:e, s:e] = D
        return M

    def stored_numbers(self) -> int:
        return (sum(U.size + V.size for lvl in self.offdiag for _, _, U, V in lvl)
                + sum(D.size for D in self.leaves.values()))


def _range(Y: np.ndarray, tol: float) -> np.ndarray:
    """Orthonormal basis of the numerical range of Y (SVD, relative tolerance tol)."""
    if Y.size == 0:
        return np.zeros((Y.shape[0], 0))
    Uy, sv, _ = np.linalg.svd(Y, full_matrices=False)
    if sv.size == 0 or sv[0] == 0.0:
        return np.zeros((Y.shape[0], 0))
    return Uy[:, : int(np.sum(sv > tol * sv[0]))]


def recover_hodlr(apply: Callable[[np.ndarray], np.ndarray], apply_t: Callable[[np.ndarray], np.ndarray],
                  n: int, rank: int, leaf: int, rng: np.random.Generator, oversample: int = 10,
                  tol: float = 1e-13) -> HODLR:
    """Recover an n x n matrix M from products X -> M X (apply) and X -> M^T X (apply_t)."""
    levels = _boxes(n, leaf)
    H = HODLR(n=n, levels=levels)
    k = rank + oversample
    for li in range(1, len(levels)):
        pairs = [(levels[li][2 * i], levels[li][2 * i + 1]) for i in range(len(levels[li]) // 2)]
        found = []
        for first in (0, 1):                      # 0: blocks M[right, left]; 1: M[left, right]
            G = rng.standard_normal((n, k))
            Om = np.zeros((n, k))
            for a, b in pairs:
                c0, c1 = (a, b)[first]
                Om[c0:c1] = G[c0:c1]
            Y = apply(Om) - H.apply_known(Om, li)
            H.products += k
            bases = []
            for a, b in pairs:
                r0, r1 = (b, a)[first]
                bases.append(_range(Y[r0:r1], tol))
            w = max(U.shape[1] for U in bases) if bases else 0
            Psi = np.zeros((n, w))
            for (a, b), U in zip(pairs, bases):
                r0, r1 = (b, a)[first]
                Psi[r0:r1, : U.shape[1]] = U
            Z = apply_t(Psi) - H.apply_known(Psi, li, transpose=True)
            H.products += w
            for (a, b), U in zip(pairs, bases):
                rows, cols = ((b, a), (a, b))[first]
                found.append((rows, cols, U, Z[cols[0]:cols[1], : U.shape[1]].copy()))
        H.offdiag.append(found)
    # leaves: identity sketches on every leaf at once; the off-diagonal part is all known now
    lv = levels[-1]
    w = max(e - s for s, e in lv)
    E = np.zeros((n, w))
    for s, e in lv:
        E[s:e, : e - s] = np.eye(e - s)
    Y = apply(E) - H.apply_known(E, len(levels))
    H.products += w
    for s, e in lv:
        H.leaves[(s, e)] = Y[s:e, : e - s].copy()
    return H
