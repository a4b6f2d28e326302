"""Pins of the oracle's randomized recovery of rank-structured blocks from products (Sec. 3.3).

The recovery sees a block only through X -> M X and X -> M^T X.  It is pinned to facts outside it:
on a matrix built with exact hierarchical off-diagonal ranks it must reproduce the matrix to
rounding with fewer products than the matrix has columns; on the reduced blocks T_qq, T_{q,q+1},
T_{q+1,q} of the slab method (Poisson, diffusion, and the nonsymmetric convection-diffusion,
whose transposed products differ) it must reproduce the exact blocks with the rank bound of
Prop. 1, 2 (b - 1); and two plausible mistakes -- too few samples for the true rank, or the
forward product where the transpose is needed -- must fail.
"""
import numpy as np
import pytest

from oracle.recovery import _boxes, recover_hodlr
from paper_2211_07572_gb300 import inputs


def _synthetic_hodlr(n, rank, leaf, rng):
    """Dense matrix whose off-diagonal blocks at every level of the box tree have rank `rank`."""
    levels = _boxes(n, leaf)
    M = np.zeros((n, n))
    for li in range(1, len(levels)):
        for i in range(len(levels[li]) // 2):
            (a0, a1), (b0, b1) = levels[li][2 * i], levels[li][2 * i + 1]
            M[b0:b1, a0:a1] = rng.standard_normal((b1 - b0, rank)) @ rng.standard_normal((rank, a1 - a0))
            M[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, rank)) @ rng.standard_normal((rank, b1 - b0))
    for s, e in levels[-1]:
        M[s:e, s:e] = rng.standard_normal((e - s, e - s))
    return M


def test_exact_on_a_synthetic_hodlr_matrix():
    rng = np.random.default_rng(1)
    n, rank, leaf = 1000, 5, 32
    M = _synthetic_hodlr(n, rank, leaf, rng)
    H = recover_hodlr(lambda X: M @ X, lambda X: M.T @ X, n, rank, leaf, np.random.default_rng(2))
    assert np.abs(H.dense() - M).max() <= 1e-11 * np.abs(M).max()
    assert H.products < n                      # cheaper than probing every column
    assert H.stored_numbers() < n * n / 3


def test_too_few_samples_fail():
    rng = np.random.default_rng(3)
    n, rank, leaf = 512, 6, 32
    M = _synthetic_hodlr(n, rank, leaf, rng)
    H = recover_hodlr(lambda X: M @ X, lambda X: M.T @ X, n, 2, leaf, np.random.default_rng(4), oversample=1)
    assert np.abs(H.dense() - M).max() > 1e-3 * np.abs(M).max()


def _blocks(kind, n, b):
    import oracle
    if kind == inputs.CONVECTION:
        p = inputs.convection(n, b, 1, field_seed=70, velocity_seeds=(71, 72, 73))
    elif kind == inputs.DIFFUSION:
        p = inputs.diffusion(n, b, 1, field_seed=74)
    else:
        p = inputs.Problem("p", 2, n, b, inputs.POISSON)
    A = oracle.assemble_problem(p)
    return oracle.reduced_system(A, 2, n, b, pivot=kind == inputs.CONVECTION)


@pytest.mark.parametrize("kind,n,b", [(inputs.POISSON, 128, 4), (inputs.DIFFUSION, 128, 8),
                                      (inputs.DIFFUSION, 256, 16), (inputs.CONVECTION, 128, 8)])
def test_recovers_the_reduced_blocks_at_the_rank_bound(kind, n, b):
    Td, Tl, Tu = _blocks(kind, n, b)
    rank = 2 * (b - 1)                          # Prop. 1
    for M in (Td[1], Tu[1], Tl[1]):
        H = recover_hodlr(lambda X: M @ X, lambda X: M.T @ X, M.shape[0], rank, 2 * rank,
                          np.random.default_rng(5))
        assert np.abs(H.dense() - M).max() <= 1e-11 * np.abs(M).max()


def test_transposed_products_are_needed_for_a_nonsymmetric_block():
    Td, Tl, Tu = _blocks(inputs.CONVECTION, 128, 8)
    M = Td[1]
    assert np.abs(M - M.T).max() > 1e-6 * np.abs(M).max()
    H = recover_hodlr(lambda X: M @ X, lambda X: M @ X, M.shape[0], 14, 28, np.random.default_rng(6))
    assert np.abs(H.dense() - M).max() > 1e-6 * np.abs(M).max()
