"""Three-dimensional slabs: parity of the CUDA path with the oracle (seven-point stencil).

The 3-D tree runs along z with sheets of m (n-1) unknowns per node; the interface planes are
(n-1)^2 nodes ordered y fastest, then z (the oracle's natural order restricted to a plane).
Inputs follow the 3-D diffusion workload's recipe (kappa = exp of a seeded 8-mode field,
N(0,1) loads) at sizes the banded-LU oracle finishes in seconds.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(p, precision, rtol=1e-12, max_refine=30, stage2="auto"):
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(3, p.n, p.b, p.kind, kappa=p.kappa, precision=precision, rtol=rtol,
                      max_refine=max_refine, stage2=stage2)


TOL = {"fp64": 1e-11, "fp32": 2e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", [(16, 4), (24, 6)])
def test_3d_T_blocks_match_oracle(n, b, precision):
    """Stage 1 + assembly in 3-D: every T block equals the oracle's Schur complement blocks."""
    p = inputs.diffusion(n, b, k=1, dim=3, n_modes=8, field_seed=4, rhs_seed=104)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 3, n, b)
    scale = max(np.abs(t).max() for t in Td)
    for q in range(len(Td)):
        assert np.abs(s.T_block(0, q) - Td[q]).max() <= TOL[precision] * scale, q
    for q in range(len(Tu)):
        assert np.abs(s.T_block(1, q) - Tu[q]).max() <= TOL[precision] * scale, q
    s.close()


@pytest.mark.parametrize("precision,stage2", [("fp64", "sweep"), ("fp32", "sweep"), ("fp32", "oddeven")])
@pytest.mark.parametrize("n,b", [(24, 6), (32, 8), (40, 8)])
def test_3d_solve_matches_oracle(n, b, precision, stage2):
    """End to end in 3-D (b = 8 is the 3-D workload's slab spacing; n = 40 has four interfaces)."""
    p = inputs.diffusion(n, b, k=3, dim=3, n_modes=8, field_seed=4, rhs_seed=104)
    s = _solver(p, precision, rtol=1e-13, stage2=stage2)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    r = s.residual(torch.from_numpy(u).cuda(), torch.from_numpy(p.f).cuda()).cpu().numpy()
    s.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    assert np.abs(r - oracle.residual(A, u, p.f)).max() <= 1e-12 * np.abs(p.f).max()
    err = np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert err.max() <= 1e-8, err


def test_3d_poisson_closed_form():
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z): the discrete solution is r3 sin sin sin exactly,
    r3 = 3 pi^2 / (3 * 4 sin^2(pi h / 2) / h^2)."""
    n, b = 32, 8
    p = inputs.poisson_sine(n, b, dim=3)
    s = _solver(p, "fp32", rtol=1e-13)
    u, rel, _ = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    s.close()
    h = 1.0 / n
    r3 = 3 * math.pi ** 2 / (3 * 4 * math.sin(math.pi * h / 2) ** 2 / h ** 2)
    exact = r3 * p.u_exact
    err = np.linalg.norm(u.cpu().numpy() - exact) / np.linalg.norm(exact)
    assert err <= 1e-10, err


def test_3d_phases_match_oracle():
    """Reduced load (eqs. f1-f5) and interior solve (eq. usol_even) in 3-D against the oracle."""
    n, b = 24, 6
    p = inputs.diffusion(n, b, k=2, dim=3, n_modes=8, field_seed=4, rhs_seed=105)
    s = _solver(p, "fp64")
    A = oracle.assemble_problem(p)
    ft = s.reduced_rhs(torch.from_numpy(p.f).cuda()).cpu().numpy()
    ft_o = np.concatenate(oracle.reduced_rhs(A, p.f, 3, n, b), axis=1)
    assert np.abs(ft - ft_o).max() <= 1e-10 * np.abs(ft_o).max()
    u_o = oracle.solve(p)
    sets = oracle.index_sets(3, n, b)
    ut = np.concatenate([u_o[:, sets[2 * q + 1]] for q in range(n // b - 1)], axis=1)
    u = s.interior_solve(torch.from_numpy(p.f).cuda(), torch.from_numpy(ut).cuda()).cpu().numpy()
    assert np.abs(u - u_o).max() <= 1e-10 * np.abs(u_o).max()
    s.close()
