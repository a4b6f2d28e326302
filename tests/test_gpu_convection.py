"""Nonsymmetric operator on the CUDA path: convection-diffusion -div(kappa grad u) + beta.grad u.

Parity with the CPU oracle through the C ABI, phase by phase (coefficients and stencil, the
reduced blocks T_qq, T_{q,q+1} and T_{q+1,q}, reduced load, interface solve, interior solve),
end to end with refinement, and for the adjoint: A^T lambda = dL/du solved transposed on the
same factors against the oracle's banded LU of A^T, the gradient against the oracle's and
against central differences of the loss.  Tolerances as in the symmetric parity tests: FP64
phases to rounding (1e-11 of the block scale), FP32 phases 2e-5 of the block scale (T) or
1e-3 relative (solves with cond(T) * eps32), refined solves relres <= 1e-10 and
||u - u_oracle|| / ||u_oracle|| <= 1e-8; gradients 1e-8 against the oracle's, 1e-6 against
central differences (step 1e-6).
"""
import numpy as np
import pytest
import torch

import oracle
from fdcheck import fd_operator_difference
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu
CONV = inputs.CONVECTION
TOL = {"fp64": 1e-11, "fp32": 2e-5}

# sizes spanning several 64-wide tiles with a ragged tail, the widest (b = 33) and narrowest
# (b = 2) slabs, and one odd interface count
CASES = [(64, 8), (96, 8), (66, 33), (40, 2), (130, 26)]


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()


def _problem(n, b, k=2, seed=0, speed=20.0):
    return inputs.convection(n, b, k, speed=speed, field_seed=60 + seed,
                             velocity_seeds=(61 + seed, 62 + seed, 63 + seed), rhs_seed=64 + seed)


def _solver(p, precision="fp64", rtol=1e-10, max_refine=30, iprec=None, pivot="tournament"):
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(2, p.n, p.b, CONV, kappa=p.kappa, beta=p.beta, precision=precision, rtol=rtol,
                      max_refine=max_refine, interface_precision=iprec, pivot=pivot)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_stencil_and_transpose_match_oracle():
    p = _problem(64, 8, k=3)
    s = _solver(p)
    A = oracle.assemble_problem(p)
    At = A.transpose()
    u = inputs.normal_rhs(2, p.n, 3, 77)
    scale = np.abs(A.matvec(u)).max()
    r = s.residual(_cuda(u), _cuda(p.f)).cpu().numpy()
    assert np.abs(r - oracle.residual(A, u, p.f)).max() <= 1e-13 * scale
    assert np.abs(s.apply(_cuda(u)).cpu().numpy() - A.matvec(u)).max() <= 1e-13 * scale
    yt = s.apply_transpose(_cuda(u)).cpu().numpy()
    assert np.abs(yt - At.matvec(u)).max() <= 1e-13 * scale
    assert np.abs(yt - A.matvec(u)).max() > 1e-3 * scale          # the operator is not symmetric


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", CASES)
def test_T_blocks_match_oracle(n, b, precision):
    """Stage 1 + assembly: T_qq, T_{q,q+1} and T_{q+1,q} equal eqs. T11-T35 of the oracle."""
    p = _problem(n, b)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b, pivot=True)
    scale = max(np.abs(t).max() for t in Td)
    for q in range(len(Td)):
        assert np.abs(s.T_block(0, q) - Td[q]).max() <= TOL[precision] * scale, q
    for q in range(len(Tu)):
        assert np.abs(s.T_block(1, q) - Tu[q]).max() <= TOL[precision] * scale, q
        assert np.abs(s.T_block(2, q) - Tl[q]).max() <= TOL[precision] * scale, q


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", CASES[:4])
def test_phases_match_oracle(n, b, precision):
    """Reduced load (eqs. f1-f5), Algorithms 1+2 on the oracle's f~, interior solve (eq. usol_even)."""
    p = _problem(n, b, k=3, seed=1)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    ft = oracle.reduced_rhs(A, p.f, 2, n, b, pivot=True)
    ftg = s.reduced_rhs(_cuda(p.f)).cpu().numpy()
    fto = np.concatenate(ft, axis=1)
    assert np.abs(ftg - fto).max() <= TOL[precision] * 50 * np.abs(fto).max()
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b, pivot=True)
    ut_o = np.concatenate(oracle.sweep_solve(Tl, Tu, oracle.sweep_build(Td, Tl, Tu), ft), axis=1)
    ut = s.interface_solve(_cuda(fto)).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert np.abs(ut - ut_o).max() <= tol * np.abs(ut_o).max()
    u_o = oracle.solve(p)
    sets = oracle.index_sets(2, n, b)
    uti = np.concatenate([u_o[:, sets[2 * q + 1]] for q in range(n // b - 1)], axis=1)
    u = s.interior_solve(_cuda(p.f), _cuda(uti)).cpu().numpy()
    assert np.abs(u - u_o).max() <= TOL[precision] * 50 * np.abs(u_o).max()


@pytest.mark.parametrize("precision,iprec", [("fp64", None), ("fp32", None), ("fp32", "fp64")])
@pytest.mark.parametrize("n,b", [(64, 8), (130, 26), (256, 16)])
def test_solve_matches_oracle(n, b, precision, iprec):
    p = _problem(n, b, k=3, seed=2)
    s = _solver(p, precision, iprec=iprec)
    u, rel, _ = s.solve(_cuda(p.f))
    u = u.cpu().numpy()
    A = oracle.assemble_problem(p)
    u_o = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    assert (np.linalg.norm(u - u_o, axis=1) / np.linalg.norm(u_o, axis=1)).max() <= 1e-8
    assert rel.max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", [(256, 16), (320, 32)])
def test_local_pivoting_matches_oracle(n, b, precision):
    """Pivot rows restricted to the diagonal 64-row blocks (no tournament): on a diffusion-dominated
    operator (cell Peclet number below 1) the factor, the solve and the transposed solve still meet
    the bounds of the pivoted path."""
    p = _problem(n, b, k=2, seed=7)
    s = _solver(p, precision, pivot="local")
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b, pivot=True)
    scale = max(np.abs(t).max() for t in Td)
    assert np.abs(s.T_block(2, 1) - Tl[1]).max() <= TOL[precision] * scale
    u, rel, _ = s.solve(_cuda(p.f))
    u_o = oracle.solve(p)
    assert rel.max() <= 1e-10
    assert (np.linalg.norm(u.cpu().numpy() - u_o, axis=1) / np.linalg.norm(u_o, axis=1)).max() <= 1e-8
    g = inputs.normal_rhs(2, n, 2, 95)
    lam, _ = s.adjoint(_cuda(g))
    lam_o = oracle.solve_transposed(p, g)
    assert (np.linalg.norm(lam.cpu().numpy() - lam_o, axis=1) / np.linalg.norm(lam_o, axis=1)).max() <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", [(64, 8), (130, 26)])
def test_adjoint_solve_is_transposed(n, b, precision):
    """slab_adjoint solves A^T lambda = g on the same factors (not A lambda = g)."""
    p = _problem(n, b, k=2, seed=3)
    s = _solver(p, precision)
    g = inputs.normal_rhs(2, n, 2, 91)
    lam, _ = s.adjoint(_cuda(g))
    lam = lam.cpu().numpy()
    lam_o = oracle.solve_transposed(p, g)
    At = oracle.assemble_problem(p).transpose()
    assert oracle.relres(At, lam, g).max() <= 1e-10
    assert (np.linalg.norm(lam - lam_o, axis=1) / np.linalg.norm(lam_o, axis=1)).max() <= 1e-8
    assert np.abs(lam - oracle.solve(p, g)).max() > 1e-3 * np.abs(lam_o).max()
    # the forward solve on the same handle is untouched by the transposed one
    u, rel, _ = s.solve(_cuda(p.f))
    assert rel.max() <= 1e-10
    assert np.abs(u.cpu().numpy() - oracle.solve(p)).max() <= 1e-8 * np.abs(oracle.solve(p)).max()


def test_adjoint_gradient_matches_oracle():
    p = _problem(96, 8, k=1, seed=4)
    ut = inputs.normal_rhs(2, p.n, 1, 92)
    L, u_o, lam_o, g_o = oracle.adjoint_gradient(p, ut)
    s = _solver(p, "fp32", rtol=1e-13, max_refine=40)
    u, _, _ = s.solve(_cuda(p.f), allow_noconv=True)
    lam, g = s.adjoint(2 * (u - _cuda(ut)), u, allow_noconv=True)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 1e-8
    assert (np.linalg.norm(lam.cpu().numpy() - lam_o) / np.linalg.norm(lam_o)) <= 1e-8


def test_adjoint_gradient_vs_central_differences():
    """32 probes, step 1e-6: the loss difference formed without cancellation (the kappa part of
    the operator difference in closed form; the first-order term does not depend on kappa)."""
    n, b, delta = 128, 16, 1e-6
    p = _problem(n, b, k=1, seed=5, speed=30.0)
    ut = _cuda(inputs.normal_rhs(2, n, 1, 93))
    f = _cuda(p.f)
    s = _solver(p, "fp32", rtol=1e-14, max_refine=40)
    u, _, _ = s.solve(f, allow_noconv=True)
    _, g = s.adjoint(2 * (u - ut), u, allow_noconv=True)
    g = g.cpu().numpy()
    s.close()
    rng = np.random.default_rng(94)
    fd, ad = [], []
    for (x, y) in rng.integers(1, n, size=(32, 2)):
        kp = p.kappa.copy(); kp[y, x] += delta
        km = p.kappa.copy(); km[y, x] -= delta
        pm = inputs.Problem("m", 2, n, b, CONV, kappa=km, beta=p.beta, f=p.f)
        pp = inputs.Problem("p", 2, n, b, CONV, kappa=kp, beta=p.beta, f=p.f)
        sm = _solver(pm, "fp32", rtol=1e-14, max_refine=40)
        um, _, _ = sm.solve(f, allow_noconv=True)
        sm.close()
        sp = _solver(pp, "fp32", rtol=1e-14, max_refine=40)
        dAu = _cuda(fd_operator_difference(um.cpu().numpy(), kp, km, x, y, n))
        du, _, _ = sp.solve(-dAu, allow_noconv=True)
        sp.close()
        fd.append(float((du * (2 * um + du - 2 * ut)).sum()) / (2 * delta))
        ad.append(g[y, x])
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) / np.linalg.norm(fd) <= 1e-6


def test_larger_grid_matches_oracle():
    """n = 512, b = 32, 4 loads: u against the oracle's pivoted banded LU."""
    p = _problem(512, 32, k=4, seed=6)
    s = _solver(p, "fp32")
    u, rel, _ = s.solve(_cuda(p.f))
    u = u.cpu().numpy()
    u_o = oracle.solve(p)
    assert rel.max() <= 1e-10
    assert oracle.relres(oracle.assemble_problem(p), u, p.f).max() <= 1e-10
    assert (np.linalg.norm(u - u_o, axis=1) / np.linalg.norm(u_o, axis=1)).max() <= 1e-8


def test_full_size_residuals_by_the_oracle():
    """The benchmark's configuration (n = 2048, b = 32, 16 loads), beyond the oracle's banded LU:
    the relative residuals of u (with A) and of the adjoint lambda (with A^T) on sampled loads,
    computed by the oracle's own CSR assembly, transpose and matvec, are <= 1e-10."""
    from paper_2211_07572_gb300.solver import SlabSolver
    n, b, k = 2048, 32, 16
    p = inputs.convection(n, b, k)
    ut = inputs.normal_rhs(2, n, k, 107)
    s = SlabSolver(2, n, b, CONV, kappa=p.kappa, beta=p.beta, rtol=1e-10, max_refine=40)
    u, rel, _ = s.solve(_cuda(p.f))
    g = 2 * (u - _cuda(ut))
    lam, _ = s.adjoint(g)
    s.close()
    idx = [0, k // 2, k - 1]
    us, ls, gs = u[idx].cpu().numpy(), lam[idx].cpu().numpy(), g[idx].cpu().numpy()
    del u, lam, g
    assert np.max(rel) <= 1e-10
    A = oracle.assemble_problem(p)
    assert oracle.relres(A, us, p.f[idx]).max() <= 1e-10
    assert oracle.relres(A.transpose(), ls, gs).max() <= 1e-10


def test_unsupported_and_invalid():
    from paper_2211_07572_gb300 import _lib
    from paper_2211_07572_gb300.solver import SlabSolver
    p = _problem(32, 8)
    with pytest.raises(_lib.SlabError) as e:
        SlabSolver(2, 32, 8, CONV, kappa=p.kappa, beta=None)          # no velocity field
    assert e.value.status == _lib.SLAB_EINVAL
    with pytest.raises(_lib.SlabError) as e:
        SlabSolver(2, 32, 8, CONV, kappa=p.kappa, beta=p.beta, stage2="oddeven")
    assert e.value.status == _lib.SLAB_EUNSUPPORTED
    q = inputs.convection(16, 4, 1, dim=3)
    with pytest.raises(_lib.SlabError) as e:
        SlabSolver(3, 16, 4, CONV, kappa=q.kappa, beta=q.beta)
    assert e.value.status == _lib.SLAB_EUNSUPPORTED
    s = _solver(p)
    with pytest.raises(_lib.SlabError) as e:
        s.boundary_lift(torch.zeros((1, 33 * 33), dtype=torch.float64, device="cuda"))
    assert e.value.status == _lib.SLAB_EUNSUPPORTED
