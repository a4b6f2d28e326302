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


def _solver(p, precision, rtol=1e-12, max_refine=30, iprec=None, krylov=0):
    """precision "fp32" runs the FP32 slab trees with the FP64 interface system (the default for
    Helmholtz); iprec="fp32" forces the FP32 interface system as well; krylov=m refines by
    FP64 GMRES(m) preconditioned by the factor."""
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(p.dim, p.n, p.b, p.kind, c=p.c, omega=p.omega, precision=precision, rtol=rtol,
                      max_refine=max_refine, interface_precision=iprec, krylov=krylov)


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


@pytest.mark.parametrize("precision,iprec", [("fp64", None), ("fp32", None), ("fp32", "fp32")])
def test_helmholtz_solve_matches_oracle(precision, iprec):
    """n = 128: all three precision modes (FP64; FP32 trees + FP64 interface; all FP32)."""
    n, b = 128, 16
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    p.f = np.concatenate([p.f, inputs.normal_rhs(2, n, 2, 33)])      # point source + 2 random loads
    s = _solver(p, precision, rtol=1e-13, iprec=iprec)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    s.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    err = np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert err.max() <= 1e-8, err


def _block_tridiag(Td, Tl, Tu):
    NI, s = len(Td), Td[0].shape[0]
    T = np.zeros((NI * s, NI * s))
    for q in range(NI):
        T[q * s:(q + 1) * s, q * s:(q + 1) * s] = Td[q]
    for q in range(NI - 1):
        T[q * s:(q + 1) * s, (q + 1) * s:(q + 2) * s] = Tu[q]
        T[(q + 1) * s:(q + 2) * s, q * s:(q + 1) * s] = Tl[q]
    return T


@pytest.mark.parametrize("stage_prec,eps", [("fp64", 2.2e-16), ("fp32", 6e-8), ("fp64tc", 2.2e-16)])
@pytest.mark.parametrize("n,b", [(256, 16), (512, 32)])
def test_helmholtz_interface_solve_matches_oracle(n, b, stage_prec, eps):
    _interface_check(n, b, stage_prec, eps)


def _interface_check(n, b, stage_prec, eps):
    """Stage 2 alone (blocked Gauss-Jordan with tournament pivoting, Algorithm 2) on the oracle's
    reduced system: s_pad = 256 and 512 give 4 and 8 panels and one and two levels of tournament
    merges.  T is indefinite and ill-conditioned (cond ~ 3e5 and 1e8 here), so the main check is
    the normwise (infinity-norm) backward error ||T u - f|| / (||T|| ||u|| + ||f||); the forward
    error is compared with the oracle's own Algorithm 1/2.  Algorithm 1 applies explicit
    inverses S_j^{-1}; the residual of x = S^{-1} b is bounded by about cond(S) eps rather than
    eps (Gauss-Jordan / explicit-inverse residual bound), so the backward-error bound is
    10 max_j cond(S_j) eps (at most 1e-2); the forward error must agree with
    cond(T) times the two backward errors."""
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    p.f = np.concatenate([p.f, inputs.normal_rhs(2, n, 2, 35)])
    s = _solver(p, "fp64" if stage_prec == "fp64tc" else stage_prec, iprec=stage_prec)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b, pivot=True)
    ft = np.concatenate(oracle.reduced_rhs(A, p.f, 2, n, b, pivot=True), axis=1)
    Sinv = oracle.sweep_build(Td, Tl, Tu)
    ut_o = np.concatenate(oracle.sweep_solve(Tl, Tu, Sinv, np.split(ft, len(Td), axis=1)), axis=1)
    ut = s.interface_solve(torch.from_numpy(ft).cuda()).cpu().numpy()
    s.close()
    T = _block_tridiag(Td, Tl, Tu)
    tn = np.linalg.norm(T, np.inf)
    res = np.abs(ut @ T.T - ft).max(axis=1)
    berr = res / (tn * np.abs(ut).max(axis=1) + np.abs(ft).max(axis=1))
    # largest cond(S_j) of Algorithm 1, S_j = (S_j^{-1})^{-1} from the oracle
    condS = max(np.linalg.norm(np.linalg.inv(Si), np.inf) * np.linalg.norm(Si, np.inf) for Si in Sinv)
    assert berr.max() <= min(10 * condS * eps, 1e-2), (berr, condS)
    # forward error: both solutions lie within cond(T) x (their backward errors) of the exact one
    cond = tn * np.linalg.norm(np.linalg.inv(T), np.inf)
    res_o = np.abs(ut_o @ T.T - ft).max(axis=1)
    berr_o = res_o / (tn * np.abs(ut_o).max(axis=1) + np.abs(ft).max(axis=1))
    err = np.abs(ut - ut_o).max(axis=1) / np.abs(ut_o).max(axis=1)
    assert err.max() <= 4 * cond * (berr.max() + berr_o.max()), (err, cond, berr, berr_o)


@pytest.mark.parametrize("n,b,precision,iprec", [(256, 16, "fp64", None), (256, 16, "fp32", "fp32"),
                                                 (1024, 32, "fp64", None), (1024, 32, "fp32", None)])
def test_constant_helmholtz_matches_sine_transform(n, b, precision, iprec):
    """c = 1: u = Q (Lam + q)^-1 Q f with the DST-I matrix Q, computed independently of the oracle;
    n = 1024, b = 32 has the Helmholtz workload's slab width and points per wavelength.  There the
    Stage-2 block S_27 is the operator of the sub-box x < 28 b, whose smallest eigenvalue is
    1.2e-7 of the largest: numerically singular in FP32, so that size runs the interface system
    in FP64 (FP64, or FP32 slab trees with the FP64 interface)."""
    omega = 2 * math.pi * n / 10.0
    p = inputs.constant_helmholtz(n, b, omega, rhs_seed=41, k=2)
    s = _solver(p, precision, rtol=1e-13, max_refine=40, iprec=iprec)
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


@pytest.mark.parametrize("precision,iprec,krylov", [("fp64", None, 0), ("fp64", None, 10), ("fp64", "fp64tc", 0)])
def test_helmholtz_solve_matches_oracle_n512(precision, iprec, krylov):
    """End to end at n = 512, b = 32 (the Helmholtz workload's b and points per wavelength; eight
    Stage-2 panels with two tournament merge levels): refined solution vs the pivoted banded LU.
    FP64 factor, with plain refinement, with GMRES(10) refinement, and with the interface
    elimination's products FP64-accurate on the tensor cores ("fp64tc")."""
    n, b = 512, 32
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    s = _solver(p, precision, rtol=1e-12, max_refine=60, iprec=iprec, krylov=krylov)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    s.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    err = np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert err.max() <= 1e-8, err


@pytest.mark.parametrize("iprec,krylov", [(None, 0), ("fp32", 0), (None, 30)])
def test_helmholtz_fp32_factor_reports_noconv_n512(iprec, krylov):
    """At n = 512 and 10 points per wavelength an FP32 factor (FP32 slab trees with an FP64 or
    FP32 interface system) is too inaccurate for this indefinite operator: plain refinement
    diverges and GMRES preconditioned by it stagnates.  The solver must say so (ENOCONV, status
    4) rather than return the iterate as converged."""
    from paper_2211_07572_gb300 import SlabError
    n, b = 512, 32
    p = inputs.helmholtz(n, b, n_modes=8, field_seed=3)
    s = _solver(p, "fp32", rtol=1e-10, max_refine=20, iprec=iprec, krylov=krylov)
    with pytest.raises(SlabError) as ei:
        s.solve(torch.from_numpy(p.f).cuda())
    assert ei.value.status == 4
    s.close()
