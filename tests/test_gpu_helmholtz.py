"""Helmholtz (real indefinite) path: pivoted slab separators and pivoted Stage 2.

Inputs follow the Helmholtz workload recipe at sizes the oracle finishes in
seconds: c = 1 + 0.3 r (r a max-abs-normalised 8-mode field), omega giving 10 points
per wavelength at c = 1, point source or random right-hand sides.  The oracle is the
banded LU with partial pivoting.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(p, precision, rtol=1e-12, max_refine=30):
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(p.dim, p.n, p.b, p.kind, c=p.c, omega=p.omega, precision=precision, rtol=rtol,
                      max_refine=max_refine)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
@pytest.mark.parametrize("n,b", [(64, 8), (96, 16)])
def test_helmholtz_T_blocks_match_oracle(n, b, precision, tol):
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b, pivot=True)
    scale = max(np.abs(t).max() for t in Td)
    for q in range(len(Td)):
        assert np.abs(s.T_block(0, q) - Td[q]).max() <= tol * scale, q
    for q in range(len(Tu)):
        assert np.abs(s.T_block(1, q) - Tu[q]).max() <= tol * scale, q
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_helmholtz_solve_matches_oracle(precision):
    n, b = 128, 16
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    p.f = np.concatenate([p.f, inputs.normal_rhs(2, n, 2, 33)])      # point source + 2 random loads
    s = _solver(p, precision, rtol=1e-13)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    s.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    err = np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert err.max() <= 1e-8, err


def test_constant_helmholtz_matches_sine_transform():
    """c = 1: u = Q (Lam + q)^-1 Q f with the DST-I matrix Q, computed independently of the oracle."""
    n, b = 256, 16
    omega = 2 * math.pi * n / 10.0
    p = inputs.constant_helmholtz(n, b, omega, rhs_seed=41, k=2)
    s = _solver(p, "fp64", rtol=1e-13)
    u, rel, _ = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    s.close()
    h = 1.0 / n
    j = np.arange(1, n)
    Q = math.sqrt(2.0 / n) * np.sin(np.outer(j, j) * math.pi / n)
    mu = 4.0 * np.sin(j * math.pi * h / 2) ** 2 / h ** 2
    for r in range(2):
        F = p.f[r].reshape(n - 1, n - 1)
        U = Q @ ((Q @ F @ Q) / (mu[:, None] + mu[None, :] - omega ** 2)) @ Q
        assert np.linalg.norm(u[r].reshape(n - 1, n - 1) - U) <= 1e-9 * np.linalg.norm(U)


def test_helmholtz_point_source_residual():
    """Helmholtz workload shape (point source, 10 points per wavelength) at n = 512."""
    p = inputs.helmholtz(512, 32, n_modes=8, field_seed=3)
    s = _solver(p, "fp64", rtol=1e-12)
    u, rel, _ = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    s.close()
    A = oracle.assemble_problem(p)
    assert oracle.relres(A, u.cpu().numpy(), p.f).max() <= 1e-10
