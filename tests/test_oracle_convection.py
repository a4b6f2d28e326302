"""Pins of the oracle's nonsymmetric (convection-diffusion) kind, CPU only.

The operator -div(kappa grad u) + beta.grad u is a second-order elliptic operator with a
first-order term (the operator class of Sec. 1.1, eq. "bvp"); its five-point matrix is not
symmetric, so the slab method's reduced blocks satisfy T_{q+1,q} != T_{q,q+1}^T and the adjoint
solves with A^T.  Each test ties the oracle to something outside it: hand-derived entries, the
O(h^2) convergence to a manufactured solution (which a wrong sign or a velocity taken at the
wrong node breaks), a separate dense LU and numpy, the exact dense Schur complement, and
central finite differences of the loss for the gradient through the transposed solve.
"""
import math
import os

import numpy as np
import pytest

from paper_2211_07572_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CONV = 3


def _load_matrix(name):
    rows = [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r] for r in rows])


def _problem(dim, n, b, k=2, speed=20.0, seed=40):
    return inputs.convection(n, b, k, dim=dim, speed=speed, field_seed=seed,
                             velocity_seeds=(seed + 1, seed + 2, seed + 3), rhs_seed=seed + 4)


def test_assembly_worked_example(oracle_mod):
    n = 3
    yy, xx = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    kappa = 1.0 + xx + 10.0 * yy
    beta = np.stack([2.0 * (1.0 + xx), -1.0 * yy])
    A = oracle_mod.assemble(2, n, CONV, kappa=kappa, beta=beta).dense()
    np.testing.assert_allclose(A, _load_matrix("assembly_n3_convection.txt"), rtol=0, atol=1e-12)


def test_transpose_is_the_dense_transpose(oracle_mod):
    p = _problem(2, 9, 3)
    A = oracle_mod.assemble_problem(p)
    np.testing.assert_array_equal(A.transpose().dense(), A.dense().T)
    # the convection term makes A nonsymmetric
    assert np.abs(A.dense() - A.dense().T).max() > 0.1 * np.abs(A.dense()).max() / 36


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_manufactured_solution_second_order(oracle_mod, sign):
    """u* = sin(pi x) sin(pi y), kappa = 1, beta = sign * (3 + x, -2 y): the discrete solution
    converges to u* at O(h^2).  f = 2 pi^2 u* + beta.grad u* pointwise."""
    errs = []
    for n in (16, 32, 64):
        t = np.arange(n + 1) / n
        Y, X = np.meshgrid(t, t, indexing="ij")
        bx, by = sign * (3.0 + X), sign * (-2.0 * Y)
        us = np.sin(math.pi * X) * np.sin(math.pi * Y)
        f = (2 * math.pi ** 2 * us + bx * math.pi * np.cos(math.pi * X) * np.sin(math.pi * Y)
             + by * math.pi * np.sin(math.pi * X) * np.cos(math.pi * Y))
        p = inputs.Problem("m", 2, n, 4, CONV, kappa=np.ones((n + 1, n + 1)), beta=np.stack([bx, by]),
                           f=f[1:n, 1:n].reshape(1, -1))
        u = oracle_mod.solve(p)
        errs.append(np.abs(u - us[1:n, 1:n].reshape(1, -1)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[2] < 2e-3
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


@pytest.mark.parametrize("dim,n", [(2, 7), (2, 10), (3, 5)])
def test_band_lu_vs_dense(oracle_mod, dim, n):
    p = _problem(dim, n, 2 if n % 2 == 0 else 1)
    A = oracle_mod.assemble_problem(p)
    F = np.random.default_rng(n).standard_normal((3, A.N))
    w = (n - 1) ** (dim - 1)
    u_band = oracle_mod.BandLU(A, w, pivot=True).solve(F)
    u_dense = oracle_mod.dense_solve(A.dense(), F)
    u_np = np.linalg.solve(A.dense(), F.T).T
    scale = np.abs(u_np).max()
    assert np.abs(u_band - u_dense).max() / scale < 1e-12
    assert np.abs(u_band - u_np).max() / scale < 1e-12
    lam = oracle_mod.BandLU(A.transpose(), w, pivot=True).solve(F)
    lam_np = np.linalg.solve(A.dense().T, F.T).T
    assert np.abs(lam - lam_np).max() / np.abs(lam_np).max() < 1e-12


@pytest.mark.parametrize("dim,n,b", [(2, 16, 4), (2, 24, 8), (3, 8, 4)])
def test_T_equals_exact_schur_complement(oracle_mod, dim, n, b):
    p = _problem(dim, n, b)
    A = oracle_mod.assemble_problem(p)
    Td, Tl, Tu = oracle_mod.reduced_system(A, dim, n, b, pivot=True)
    sets = oracle_mod.index_sets(dim, n, b)
    ifaces, slabs = sets[1::2], sets[0::2]
    I, J = np.concatenate(ifaces), np.concatenate(slabs)
    S = oracle_mod.schur_dense(A.dense(), I, J)
    s = len(ifaces[0])
    scale = np.abs(S).max()
    for q in range(len(ifaces)):
        assert np.abs(Td[q] - S[q * s:(q + 1) * s, q * s:(q + 1) * s]).max() < 1e-12 * scale
        if q + 1 < len(ifaces):
            assert np.abs(Tu[q] - S[q * s:(q + 1) * s, (q + 1) * s:(q + 2) * s]).max() < 1e-12 * scale
            assert np.abs(Tl[q] - S[(q + 1) * s:(q + 2) * s, q * s:(q + 1) * s]).max() < 1e-12 * scale
            # nonsymmetric: the sub-diagonal block is not the transpose of the super-diagonal one
            assert np.abs(Tl[q] - Tu[q].T).max() > 1e-4 * scale


@pytest.mark.parametrize("dim,n,b", [(2, 32, 8), (2, 24, 4), (3, 8, 4)])
def test_slab_method_equals_banded_lu(oracle_mod, dim, n, b):
    p = _problem(dim, n, b)
    u_slab, _ = oracle_mod.slab_solve(p)
    u_band = oracle_mod.solve(p)
    np.testing.assert_allclose(u_slab, u_band, rtol=0, atol=1e-10 * np.abs(u_band).max())
    assert oracle_mod.relres(oracle_mod.assemble_problem(p), u_slab, p.f).max() < 1e-11


def test_gradient_matches_central_differences(oracle_mod):
    """dL/dkappa through the transposed solve equals central differences of the loss; the
    untransposed solve does not (the test can tell the two apart)."""
    n = 8
    p = _problem(2, n, 4, k=1, speed=30.0, seed=50)
    ut = inputs.normal_rhs(2, n, 1, 55)
    L, u, lam, g = oracle_mod.adjoint_gradient(p, ut)
    A = oracle_mod.assemble_problem(p)
    assert oracle_mod.relres(A.transpose(), lam, 2 * (u - ut)).max() < 1e-12
    lam_wrong = oracle_mod.solve(p, 2 * (u - ut))            # A^-1 instead of A^-T
    g_wrong = oracle_mod.kappa_gradient(2, n, u, lam_wrong)
    delta = 1e-6
    rng = np.random.default_rng(56)
    nodes = [(0, 3), (n, 5), (2, 0)] + [tuple(v) for v in rng.integers(1, n, size=(6, 2))]
    fd, ad, wr = [], [], []
    for (x, y) in nodes:
        kp = p.kappa.copy(); kp[y, x] += delta
        km = p.kappa.copy(); km[y, x] -= delta
        up = oracle_mod.solve(inputs.Problem("g", 2, n, 4, CONV, kappa=kp, beta=p.beta, f=p.f))
        um = oracle_mod.solve(inputs.Problem("g", 2, n, 4, CONV, kappa=km, beta=p.beta, f=p.f))
        fd.append(np.sum((up - um) * (up + um - 2 * ut)) / (2 * delta))
        ad.append(g[y, x])
        wr.append(g_wrong[y, x])
    fd, ad, wr = np.array(fd), np.array(ad), np.array(wr)
    assert np.linalg.norm(fd - ad) / np.linalg.norm(fd) < 1e-6
    assert np.linalg.norm(fd - wr) / np.linalg.norm(fd) > 1e-3


def test_convection_inputs_follow_the_recipe():
    """Seeded: the same call twice gives the same fields; kappa = exp(unit-variance field) > 0;
    each velocity component reaches the stated speed in max-abs; loads have the stated shape."""
    p = inputs.convection(48, 8, 3, speed=20.0)
    q = inputs.convection(48, 8, 3, speed=20.0)
    np.testing.assert_array_equal(p.beta, q.beta)
    np.testing.assert_array_equal(p.kappa, q.kappa)
    np.testing.assert_array_equal(p.f, q.f)
    assert p.beta.shape == (2, 49, 49) and p.f.shape == (3, 47 * 47)
    assert (p.kappa > 0).all() and abs(np.log(p.kappa).std() - 1) < 1e-12
    for a in range(2):
        assert abs(np.abs(p.beta[a]).max() - 20.0) < 1e-12
    assert not np.array_equal(p.beta[0], p.beta[1])


def test_zero_velocity_is_the_diffusion_operator(oracle_mod):
    p = _problem(2, 12, 4)
    A0 = oracle_mod.assemble(2, 12, CONV, kappa=p.kappa, beta=np.zeros_like(p.beta)).dense()
    Ad = oracle_mod.assemble(2, 12, inputs.DIFFUSION, kappa=p.kappa).dense()
    np.testing.assert_array_equal(A0, Ad)


def test_constant_coefficients_are_a_kronecker_sum(oracle_mod):
    """kappa = 1, constant beta: A = I (x) T_x + T_y (x) I with the 1-D central-difference matrices
    T_a = h^-2 tridiag(-1 - beta_a h/2, 2, -1 + beta_a h/2) (sub, diagonal, super; x fastest)."""
    n, bx, by = 10, 7.0, -3.0
    h = 1.0 / n
    beta = np.stack([np.full((n + 1, n + 1), bx), np.full((n + 1, n + 1), by)])
    A = oracle_mod.assemble(2, n, CONV, kappa=np.ones((n + 1, n + 1)), beta=beta).dense()

    def t1(b):
        m = n - 1
        return (np.diag(np.full(m, 2.0)) + np.diag(np.full(m - 1, -1.0 + b * h / 2), 1)
                + np.diag(np.full(m - 1, -1.0 - b * h / 2), -1)) / h ** 2

    I = np.eye(n - 1)
    K = np.kron(I, t1(bx)) + np.kron(t1(by), I)
    np.testing.assert_allclose(A, K, rtol=0, atol=1e-12 * np.abs(K).max())
