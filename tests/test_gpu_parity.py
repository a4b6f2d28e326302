"""Parity of the CUDA path with the CPU oracle, phase by phase and end to end.

Every test calls the library through the C ABI (via the thin Python binding)
and compares element by element with the oracle on the same seeded inputs.
Tolerances: FP64 factor paths must agree to rounding (1e-11 relative to the
block scale); FP32 factor phases to 2e-5 of the block scale (single-precision
unit roundoff 6e-8 times the growth of a few tree levels); solves with
refinement must reach relres <= 1e-10 and ||u - u_oracle|| / ||u_oracle|| <= 1e-8.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()


def _solver(p, precision="fp64", rtol=1e-10, max_refine=30, stage2="auto", iprec=None):
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(p.dim, p.n, p.b, p.kind, kappa=p.kappa, c=p.c, omega=p.omega, precision=precision,
                      rtol=rtol, max_refine=max_refine, stage2=stage2, interface_precision=iprec)


def _problem(n, b, kind, k=2, seed=0):
    kappa = np.exp(inputs.fourier_field(2, n, 8, seed=40 + seed)) if kind == inputs.DIFFUSION else None
    return inputs.Problem(f"t{n}", 2, n, b, kind, kappa=kappa, f=inputs.normal_rhs(2, n, k, 50 + seed))


TOL = {"fp64": 1e-11, "fp32": 2e-5}

CASES = [(64, 8, inputs.DIFFUSION), (96, 8, inputs.DIFFUSION), (48, 16, inputs.POISSON),
         (66, 33, inputs.DIFFUSION), (40, 2, inputs.DIFFUSION), (130, 26, inputs.DIFFUSION)]


def test_residual_matches_oracle():
    p = _problem(64, 8, inputs.DIFFUSION, k=3)
    s = _solver(p)
    u = inputs.normal_rhs(2, p.n, 3, 77)
    r = s.residual(torch.from_numpy(u).cuda(), torch.from_numpy(p.f).cuda()).cpu().numpy()
    A = oracle.assemble_problem(p)
    r_o = oracle.residual(A, u, p.f)
    scale = np.abs(A.matvec(u)).max()
    assert np.abs(r - r_o).max() <= 1e-13 * scale
    y = s.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert np.abs(y - A.matvec(u)).max() <= 1e-13 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b,kind", CASES)
def test_T_blocks_match_oracle(n, b, kind, precision):
    """Stage 1 + assembly (A0-A3): the GPU reduced matrix equals eqs. T11-T35 of the oracle."""
    p = _problem(n, b, kind)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b)
    scale = max(np.abs(t).max() for t in Td)
    for q in range(len(Td)):
        assert np.abs(s.T_block(0, q) - Td[q]).max() <= TOL[precision] * scale, q
    for q in range(len(Tu)):
        assert np.abs(s.T_block(1, q) - Tu[q]).max() <= TOL[precision] * scale, q


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b,kind", CASES[:4])
def test_reduced_rhs_matches_oracle(n, b, kind, precision):
    """A5: f~ = f_I - A_IJ A_JJ^-1 f_J (eqs. f1-f5)."""
    p = _problem(n, b, kind, k=3)
    s = _solver(p, precision)
    ft = s.reduced_rhs(torch.from_numpy(p.f).cuda()).cpu().numpy()
    A = oracle.assemble_problem(p)
    ft_o = np.concatenate(oracle.reduced_rhs(A, p.f, 2, n, b), axis=1)
    assert np.abs(ft - ft_o).max() <= TOL[precision] * 10 * np.abs(ft_o).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b,kind", CASES[:4])
def test_interface_solve_matches_oracle(n, b, kind, precision):
    """A4 + A6: Algorithm 1 factors, Algorithm 2 sweep, on the oracle's own f~."""
    p = _problem(n, b, kind, k=3)
    s = _solver(p, precision)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b)
    ft = oracle.reduced_rhs(A, p.f, 2, n, b)
    ut_o = np.concatenate(oracle.sweep_solve(Tl, Tu, oracle.sweep_build(Td, Tl, Tu), ft), axis=1)
    ut = s.interface_solve(torch.from_numpy(np.concatenate(ft, axis=1)).cuda()).cpu().numpy()
    # FP32 error bound: cond(T) * eps32 with cond(T) from the oracle's blocks
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert np.abs(ut - ut_o).max() <= tol * np.abs(ut_o).max()


@pytest.mark.parametrize("stage2", ["sweep", "oddeven"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b", [(48, 16), (64, 16), (96, 16), (96, 8), (40, 2)])
def test_stage2_orders_match_oracle(n, b, precision, stage2):
    """Both elimination orders of T (Algorithm 1's sweep and the odd-even order) give
    u~ = T^-1 f~ of the oracle; N_I = 2, 3, 5, 11, 19 covers levels with and without a
    right neighbour for the last eliminated block.  T itself is left intact by the factor."""
    p = _problem(n, b, inputs.DIFFUSION, k=3, seed=5)
    s = _solver(p, precision, stage2=stage2)
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, n, b)
    ft = oracle.reduced_rhs(A, p.f, 2, n, b)
    ut_o = np.concatenate(oracle.sweep_solve(Tl, Tu, oracle.sweep_build(Td, Tl, Tu), ft), axis=1)
    ut = s.interface_solve(torch.from_numpy(np.concatenate(ft, axis=1)).cuda()).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert np.abs(ut - ut_o).max() <= tol * np.abs(ut_o).max()
    scale = max(np.abs(t).max() for t in Td)
    last = len(Td) - 1
    assert np.abs(s.T_block(0, last) - Td[last]).max() <= TOL[precision] * scale
    if Tu:
        assert np.abs(s.T_block(1, 0) - Tu[0]).max() <= TOL[precision] * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,b,kind", CASES[:4])
def test_interior_solve_matches_oracle(n, b, kind, precision):
    """A7: eq. usol_even with the oracle's interface values."""
    p = _problem(n, b, kind, k=2)
    s = _solver(p, precision)
    u_o = oracle.solve(p)
    sets = oracle.index_sets(2, n, b)
    ut = np.concatenate([u_o[:, sets[2 * q + 1]] for q in range(n // b - 1)], axis=1)
    u = s.interior_solve(torch.from_numpy(p.f).cuda(), torch.from_numpy(ut).cuda()).cpu().numpy()
    assert np.abs(u - u_o).max() <= TOL[precision] * 50 * np.abs(u_o).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_poisson_sine_closed_form(precision):
    """Poisson n = 128, b = 16: the discrete solution is exactly r sin(pi x) sin(pi y)."""
    p = inputs.poisson_sine_128()
    s = _solver(p, precision, rtol=1e-13)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)   # 1e-13 is below the FP64 floor
    u = u.cpu().numpy()
    h = 1.0 / p.n
    r = 2 * math.pi ** 2 * h * h / (8 * math.sin(math.pi * h / 2) ** 2)
    exact = r * p.u_exact
    A = oracle.assemble_problem(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    assert np.linalg.norm(u - exact) / np.linalg.norm(exact) <= 1e-10
    assert np.linalg.norm(u - oracle.solve(p)) / np.linalg.norm(exact) <= 1e-10


@pytest.mark.parametrize("stage2", ["sweep", "oddeven"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diffusion_solve_matches_oracle(precision, stage2):
    """End to end (A0-A8) on a problem shaped like the n = 2048 diffusion workload at a size the oracle finishes in seconds."""
    p = inputs.diffusion(256, 16, k=4, n_modes=16, field_seed=2, rhs_seed=102)
    s = _solver(p, precision, rtol=1e-13, stage2=stage2)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    u = u.cpu().numpy()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u, p.f).max() <= 1e-10
    err = np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert err.max() <= 1e-8, err
    if precision == "fp32":
        assert 1 <= it <= 30


@pytest.mark.parametrize("stage2", ["sweep", "oddeven"])
def test_fp64tc_interface_matches_oracle(stage2):
    """FP64 slab trees, interface elimination with FP64-accurate tensor-core products."""
    p = inputs.diffusion(256, 16, k=2, n_modes=16, field_seed=2, rhs_seed=107)
    s = _solver(p, "fp64", rtol=1e-13, stage2=stage2, iprec="fp64tc")
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, p.n, p.b)
    ft = oracle.reduced_rhs(A, p.f, 2, p.n, p.b)
    ut_o = np.concatenate(oracle.sweep_solve(Tl, Tu, oracle.sweep_build(Td, Tl, Tu), ft), axis=1)
    ut = s.interface_solve(torch.from_numpy(np.concatenate(ft, axis=1)).cuda()).cpu().numpy()
    assert np.abs(ut - ut_o).max() <= 1e-10 * np.abs(ut_o).max()
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    uo = oracle.solve(p)
    assert oracle.relres(A, u.cpu().numpy(), p.f).max() <= 1e-12
    assert (np.linalg.norm(u.cpu().numpy() - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-10
    s.close()


@pytest.mark.parametrize("stage2", ["sweep", "oddeven"])
def test_mixed_precision_matches_oracle(stage2):
    """FP32 slab trees with the interface system in FP64 (both elimination orders): T blocks are
    the FP32 assembly widened, the refined solution matches the oracle."""
    p = inputs.diffusion(256, 16, k=2, n_modes=16, field_seed=2, rhs_seed=103)
    s = _solver(p, "fp32", rtol=1e-13, stage2=stage2, iprec="fp64")
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, 2, p.n, p.b)
    scale = max(np.abs(t).max() for t in Td)
    assert np.abs(s.T_block(0, 3) - Td[3]).max() <= TOL["fp32"] * scale
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    uo = oracle.solve(p)
    assert oracle.relres(A, u.cpu().numpy(), p.f).max() <= 1e-10
    assert (np.linalg.norm(u.cpu().numpy() - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-8
    s.close()
    with pytest.raises(Exception):
        _solver(p, "fp64", iprec="fp32")                    # an FP64 factor with an FP32 interface


def test_gmres_refinement_matches_oracle():
    """FP64 GMRES(8) preconditioned by the FP32 factor, three right-hand sides with separate Krylov
    spaces and a restart: same solution as the oracle, fewer preconditioner applications than
    plain refinement needs."""
    from paper_2211_07572_gb300.solver import SlabSolver
    p = inputs.diffusion(256, 16, k=3, n_modes=16, field_seed=2, rhs_seed=104)
    s = SlabSolver(2, p.n, p.b, p.kind, kappa=p.kappa, precision="fp32", rtol=1e-13, max_refine=40, krylov=8)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda())
    s.close()
    s0 = SlabSolver(2, p.n, p.b, p.kind, kappa=p.kappa, precision="fp32", rtol=1e-13, max_refine=40)
    _, rel0, it0 = s0.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    s0.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert rel.max() <= 1e-13 and oracle.relres(A, u.cpu().numpy(), p.f).max() <= 1e-12
    assert (np.linalg.norm(u.cpu().numpy() - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-10
    assert it <= it0 + 1, (it, it0)


@pytest.mark.parametrize("dim,n,b", [(2, 256, 16), (3, 32, 8)])
def test_tf32_factor_refines_to_oracle(dim, n, b):
    """Single-pass TF32 tensor products in the factor: the refined solution still matches the oracle."""
    from paper_2211_07572_gb300.solver import SlabSolver
    p = inputs.diffusion(n, b, k=2, dim=dim, n_modes=8, field_seed=4, rhs_seed=106)
    s = SlabSolver(dim, p.n, p.b, p.kind, kappa=p.kappa, precision="tf32", rtol=1e-12, max_refine=40)
    u, rel, it = s.solve(torch.from_numpy(p.f).cuda())
    s.close()
    A = oracle.assemble_problem(p)
    uo = oracle.solve(p)
    assert oracle.relres(A, u.cpu().numpy(), p.f).max() <= 1e-11
    assert (np.linalg.norm(u.cpu().numpy() - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-9


def test_many_rhs_chunks_and_empty():
    """k > 64 runs in several passes; k = 0 is a no-op."""
    p = _problem(64, 8, inputs.DIFFUSION, k=70, seed=3)
    s = _solver(p, "fp32", rtol=1e-12)
    u, rel, _ = s.solve(torch.from_numpy(p.f).cuda())
    uo = oracle.solve(p)
    assert rel.max() <= 1e-12
    assert np.abs(u.cpu().numpy() - uo).max() <= 1e-9 * np.abs(uo).max()
    empty = torch.empty((0, p.unknowns), dtype=torch.float64, device="cuda")
    u0, rel0, _ = s.solve(empty)
    assert u0.shape == (0, p.unknowns)


def test_adjoint_gradient_matches_oracle():
    """A9: lambda = A^-T dL/du and dL/dkappa = -lambda^T (dA/dkappa) u."""
    n, b = 32, 8
    p = inputs.Problem("g", 2, n, b, inputs.DIFFUSION, kappa=np.exp(inputs.fourier_field(2, n, 6, seed=61)),
                       f=inputs.normal_rhs(2, n, 1, 62))
    ut = inputs.normal_rhs(2, n, 1, 63)
    L, u_o, lam_o, g_o = oracle.adjoint_gradient(p, ut)
    s = _solver(p, "fp32", rtol=1e-13)
    u, _, _ = s.solve(torch.from_numpy(p.f).cuda(), allow_noconv=True)
    dLdu = 2 * (u - torch.from_numpy(ut).cuda())
    lam, g = s.adjoint(dLdu, u, allow_noconv=True)
    assert np.abs(lam.cpu().numpy() - lam_o).max() <= 1e-9 * np.abs(lam_o).max()
    assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-8 * np.abs(g_o).max()


def test_invalid_arguments_are_rejected():
    from paper_2211_07572_gb300 import SlabError
    p = _problem(64, 8, inputs.DIFFUSION)
    with pytest.raises(SlabError):
        _solver(inputs.Problem("x", 2, 64, 7, inputs.POISSON))
    with pytest.raises(SlabError):
        _solver(inputs.Problem("x", 2, 64, 64, inputs.POISSON))
    # a coefficient field with a non-positive region makes the operator indefinite
    bad = p.kappa.copy()
    bad[20:40, 20:40] = -1.0
    for stage2 in ("sweep", "oddeven"):
        with pytest.raises(SlabError) as ei:
            _solver(inputs.Problem("x", 2, 64, 8, inputs.DIFFUSION, kappa=bad), stage2=stage2)
        assert ei.value.status == 3
    # the odd-even order is Cholesky based: not offered for the indefinite kind
    hp = inputs.helmholtz(64, 8, n_modes=8, field_seed=3)
    with pytest.raises(SlabError) as ei:
        _solver(hp, stage2="oddeven")
    assert ei.value.status == 7


@pytest.mark.parametrize("dim,n,b,precision,tol", [(2, 64, 8, "fp64", 1e-11), (2, 64, 8, "fp32", 2e-5),
                                                   (3, 16, 4, "fp64", 1e-11)])
def test_matrix_free_T_sketch_matches_oracle(dim, n, b, precision, tol):
    """Y = T Omega for a Gaussian sketch Omega of 6 b columns (the sketch size the paper's recovery
    draws, Sec. 3.3), applied without forming T, against the oracle's reduced blocks (eqs. T11-T35)
    multiplied out block-tridiagonally."""
    from paper_2211_07572_gb300.solver import SlabSolver
    p = inputs.diffusion(n, b, k=0, dim=dim, n_modes=8, field_seed=51)
    s = SlabSolver(dim, n, b, inputs.DIFFUSION, kappa=p.kappa, precision=precision)
    si, NI = s.s, s.NI
    k = 6 * b
    Om = np.random.default_rng(52).standard_normal((k, NI * si))
    Y = s.apply_T(torch.from_numpy(Om).cuda()).cpu().numpy()
    s.close()
    A = oracle.assemble_problem(p)
    Td, Tl, Tu = oracle.reduced_system(A, dim, n, b)
    Yo = np.zeros_like(Om)
    for q in range(NI):
        acc = Om[:, q * si:(q + 1) * si] @ Td[q].T
        if q + 1 < NI:
            acc += Om[:, (q + 1) * si:(q + 2) * si] @ Tu[q].T
        if q > 0:
            acc += Om[:, (q - 1) * si:q * si] @ Tl[q - 1].T
        Yo[:, q * si:(q + 1) * si] = acc
    assert np.linalg.norm(Y - Yo) <= tol * np.linalg.norm(Yo)
