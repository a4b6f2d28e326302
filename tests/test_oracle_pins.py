"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each test ties one oracle function to something the paper or mathematics fixes:
hand-derived stencil entries, closed-form discrete solutions, a separate dense
LU, the sine-transform diagonalisation of constant-coefficient operators, the
exact dense Schur complement, the rank property (Prop. 1), symmetry, and
central finite differences for the gradient.
"""
import math
import os

import numpy as np
import pytest

from paper_2211_07572_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load_matrix(name):
    rows = [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r] for r in rows])


def _sine_matrix(n):
    j = np.arange(1, n)
    return math.sqrt(2.0 / n) * np.sin(np.outer(j, j) * math.pi / n)   # symmetric, orthogonal


# --------------------------------------------------------------------------- assembly

def test_assembly_worked_example_diffusion(oracle_mod):
    n = 3
    yy, xx = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    kappa = 1.0 + xx + 10.0 * yy
    A = oracle_mod.assemble(2, n, oracle_mod.DIFFUSION, kappa=kappa).dense()
    np.testing.assert_allclose(A, _load_matrix("assembly_n3_diffusion.txt"), rtol=0, atol=1e-12)


def test_assembly_worked_example_helmholtz(oracle_mod):
    n = 3
    c = np.ones((n + 1, n + 1))
    c[1, 1] = 1.5
    A = oracle_mod.assemble(2, n, oracle_mod.HELMHOLTZ, c=c, omega=3.0).dense()
    np.testing.assert_allclose(A, _load_matrix("assembly_n3_helmholtz.txt"), rtol=0, atol=1e-12)


def test_assembly_3d_poisson_row(oracle_mod):
    # interior node of a 3-D grid: 6/h^2 on the diagonal, -1/h^2 to each of 6 neighbours
    n = 5
    A = oracle_mod.assemble(3, n, oracle_mod.POISSON)
    m = n - 1
    i = (1 * m + 1) * m + 1                       # node (2,2,2)
    s, e = A.rowptr[i], A.rowptr[i + 1]
    cols = A.col[s:e]
    np.testing.assert_array_equal(cols, sorted([i - m * m, i - m, i - 1, i, i + 1, i + m, i + m * m]))
    np.testing.assert_allclose(A.val[s:e], np.where(cols == i, 6.0 * n * n, -1.0 * n * n))


def test_diffusion_symmetric_and_row_sums(oracle_mod):
    n = 9
    kappa = np.exp(inputs.fourier_field(2, n, 4, seed=11))
    A = oracle_mod.assemble(2, n, oracle_mod.DIFFUSION, kappa=kappa).dense()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12)
    # A 1 = h^-2 * (sum of face coefficients to the Dirichlet boundary) at each node
    ones = A.sum(axis=1).reshape(n - 1, n - 1)
    exp = np.zeros((n - 1, n - 1))
    for y in range(1, n):
        for x in range(1, n):
            for (x2, y2) in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                if x2 in (0, n) or y2 in (0, n):
                    exp[y - 1, x - 1] += 0.5 * (kappa[y, x] + kappa[y2, x2]) * n * n
    np.testing.assert_allclose(ones, exp, rtol=1e-12, atol=1e-9)


# --------------------------------------------------------------------------- solves

def test_poisson_sine_closed_form_n128(oracle_mod):
    """Poisson n = 128: the discrete solution is exactly r sin sin, r from the golden file."""
    gold = {int(l.split()[0]): float(l.split()[1]) for l in open(os.path.join(GOLD, "poisson_sine.txt"))
            if l.strip() and not l.startswith("#")}
    p = inputs.poisson_sine_128()
    u = oracle_mod.solve(p)
    r = gold[128]
    err = np.abs(u - r * p.u_exact).max() / np.abs(r * p.u_exact).max()
    assert err < 1e-12, err
    assert abs(r - 1.0000502009159198) < 1e-15


def test_poisson_second_order_convergence(oracle_mod):
    errs = []
    for n in (16, 32, 64):
        p = inputs.poisson_sine(n, 4)
        u = oracle_mod.solve(p)
        errs.append(np.abs(u - p.u_exact).max())
        # error of the discrete solution is (r-1) sin sin with r - 1 ~ pi^2 h^2 / 12
        assert abs(errs[-1] / (math.pi ** 2 / (12 * n * n)) - 1.0) < 0.01
    assert 3.9 < errs[0] / errs[1] < 4.1 and 3.9 < errs[1] / errs[2] < 4.1


def test_poisson_3d_sine(oracle_mod):
    n = 12
    p = inputs.poisson_sine(n, 4, dim=3)
    u = oracle_mod.solve(p)
    h = 1.0 / n
    r = 3 * math.pi ** 2 * h * h / (12 * math.sin(math.pi * h / 2) ** 2)
    np.testing.assert_allclose(u, r * p.u_exact, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("dim,n,kind", [(2, 7, 1), (2, 8, 2), (3, 5, 1), (3, 4, 2), (2, 6, 0)])
def test_band_lu_vs_dense(oracle_mod, dim, n, kind):
    rng = np.random.default_rng(n * 10 + kind)
    kappa = np.exp(inputs.fourier_field(dim, n, 4, seed=5)) if kind == 1 else None
    c = 1.0 + 0.3 * inputs.fourier_field(dim, n, 3, seed=6, normalize="maxabs") if kind == 2 else None
    omega = 2 * math.pi * n / 3.0 if kind == 2 else 0.0
    A = oracle_mod.assemble(dim, n, kind, kappa=kappa, c=c, omega=omega)
    F = rng.standard_normal((3, A.N))
    lu = oracle_mod.BandLU(A, (n - 1) ** (dim - 1), pivot=(kind == 2))
    u_band = lu.solve(F)
    u_dense = oracle_mod.dense_solve(A.dense(), F)
    u_np = np.linalg.solve(A.dense(), F.T).T
    scale = np.abs(u_np).max()
    assert np.abs(u_band - u_dense).max() / scale < 1e-12
    assert np.abs(u_band - u_np).max() / scale < 1e-12
    assert oracle_mod.relres(A, u_band, F).max() < 1e-13


def test_pivoting_needed_and_used(oracle_mod):
    # Helmholtz with omega near a Dirichlet eigenvalue: the unpivoted banded LU
    # hits a tiny pivot, the pivoted one still matches the dense solve.
    n = 8
    lam11 = 8 * n * n * math.sin(math.pi / (2 * n)) ** 2
    omega = math.sqrt(lam11 * 1.7)
    A = oracle_mod.assemble(2, n, 2, c=np.ones((n + 1, n + 1)), omega=omega)
    F = np.random.default_rng(0).standard_normal((1, A.N))
    u = oracle_mod.BandLU(A, n - 1, pivot=True).solve(F)
    np.testing.assert_allclose(u, np.linalg.solve(A.dense(), F.T).T, rtol=1e-10, atol=1e-12)
    assert oracle_mod.BandLU(A, n - 1, pivot=True).ipiv.tolist() != list(range(A.N))


@pytest.mark.parametrize("kind", ["poisson", "helmholtz"])
def test_dst_constant_coefficient(oracle_mod, kind):
    """Constant coefficients: A = h^-2 (Q x Q) diag(lam_p + lam_q) (Q x Q) + q I with the DST-I matrix Q."""
    n = 48
    h = 1.0 / n
    Q = _sine_matrix(n)
    mu = 4.0 * np.sin(np.arange(1, n) * math.pi * h / 2) ** 2 / h ** 2
    if kind == "poisson":
        p = inputs.Problem("p", 2, n, 8, 0, f=inputs.normal_rhs(2, n, 2, 3))
        qv = 0.0
    else:
        omega = 2 * math.pi * n / 10.0
        p = inputs.constant_helmholtz(n, 8, omega, rhs_seed=4, k=2)
        qv = -omega ** 2
    u = oracle_mod.solve(p)
    for r in range(2):
        F = p.f[r].reshape(n - 1, n - 1)
        G = Q @ F @ Q                                   # coefficients in the sine basis
        U = Q @ (G / (mu[:, None] + mu[None, :] + qv)) @ Q
        np.testing.assert_allclose(u[r].reshape(n - 1, n - 1), U, rtol=0, atol=1e-10 * np.abs(U).max())


# --------------------------------------------------------------------------- reduced system T

def _interface_index(dim, n, b):
    sets = __import__("oracle").index_sets(dim, n, b)
    return sets[1::2], sets[0::2]


@pytest.mark.parametrize("dim,n,b,kind", [(2, 16, 4, 1), (2, 24, 8, 2), (2, 12, 3, 0), (3, 8, 4, 1)])
def test_T_equals_exact_schur_complement(oracle_mod, dim, n, b, kind):
    """The assembled reduced matrix equals A_II - A_IJ A_JJ^-1 A_JI of the dense A."""
    kappa = np.exp(inputs.fourier_field(dim, n, 5, seed=9)) if kind == 1 else None
    c = 1.0 + 0.3 * inputs.fourier_field(dim, n, 4, seed=8, normalize="maxabs") if kind == 2 else None
    omega = 2 * math.pi * n / 10 if kind == 2 else 0.0
    A = oracle_mod.assemble(dim, n, kind, kappa=kappa, c=c, omega=omega)
    Td, Tl, Tu = oracle_mod.reduced_system(A, dim, n, b, pivot=(kind == 2))
    ifaces, slabs = _interface_index(dim, n, b)
    I = np.concatenate(ifaces)
    J = np.concatenate(slabs)
    S = oracle_mod.schur_dense(A.dense(), I, J)
    s = len(ifaces[0])
    scale = np.abs(S).max()
    for q in range(len(ifaces)):
        blk = S[q * s:(q + 1) * s, q * s:(q + 1) * s]
        assert np.abs(Td[q] - blk).max() < 1e-12 * scale
        if q + 1 < len(ifaces):
            assert np.abs(Tu[q] - S[q * s:(q + 1) * s, (q + 1) * s:(q + 2) * s]).max() < 1e-12 * scale
            assert np.abs(Tl[q] - S[(q + 1) * s:(q + 2) * s, q * s:(q + 1) * s]).max() < 1e-12 * scale
        for q2 in range(q + 2, len(ifaces)):            # block tridiagonal: no fill beyond neighbours
            assert np.abs(S[q * s:(q + 1) * s, q2 * s:(q2 + 1) * s]).max() < 1e-12 * scale
        np.testing.assert_allclose(Td[q], Td[q].T, rtol=0, atol=1e-12 * scale)
    for q in range(len(Tu)):
        np.testing.assert_allclose(Tl[q], Tu[q].T, rtol=0, atol=1e-12 * scale)


def test_T_closed_form_poisson(oracle_mod):
    """Poisson: each sine mode p of an interface line sees 1-D chains of m = b-1 nodes.

    With 2 cosh(theta_p) = 2 + mu_p, mu_p = 4 sin^2(p pi h / 2), the Green's function of
    tridiag(-1, 2 cosh theta, -1) (size m) has end entries sinh(m theta)/sinh((m+1) theta)
    and sinh(theta)/sinh((m+1) theta), so (h^2-scaled)
      T_qq = Q diag(2 + mu - 2 sinh(m th)/sinh((m+1) th)) Q,  T_q,q+1 = Q diag(-sinh th / sinh((m+1) th)) Q.
    """
    n, b = 32, 8
    m = b - 1
    h = 1.0 / n
    A = oracle_mod.assemble(2, n, 0)
    Td, Tl, Tu = oracle_mod.reduced_system(A, 2, n, b)
    Q = _sine_matrix(n)
    mu = 4.0 * np.sin(np.arange(1, n) * math.pi * h / 2) ** 2
    th = np.arccosh(1.0 + mu / 2.0)
    dd = 2.0 + mu - 2.0 * np.sinh(m * th) / np.sinh((m + 1) * th)
    oo = -np.sinh(th) / np.sinh((m + 1) * th)
    Tdc = Q @ np.diag(dd) @ Q / h ** 2
    Toc = Q @ np.diag(oo) @ Q / h ** 2
    for q in range(len(Td)):
        np.testing.assert_allclose(Td[q], Tdc, rtol=0, atol=1e-9 * np.abs(Tdc).max())
    for q in range(len(Tu)):
        np.testing.assert_allclose(Tu[q], Toc, rtol=0, atol=1e-9 * np.abs(Tdc).max())


def test_rank_property(oracle_mod):
    """Prop. 1: off-diagonal blocks of a one-slab Schur complement have rank <= 2 x slab width."""
    n, b = 60, 6
    m = b - 1
    kappa = np.exp(inputs.fourier_field(2, n, 16, seed=21))
    A = oracle_mod.assemble(2, n, 1, kappa=kappa)
    ifaces, slabs = _interface_index(2, n, b)
    I, J = ifaces[2], slabs[2]                    # interface q=3 and the slab on its left
    X = A.submatrix(I, J) @ np.linalg.solve(A.submatrix(J, J), A.submatrix(J, I))
    Bsel = np.arange(12, 42)
    Fsel = np.setdiff1d(np.arange(len(I)), Bsel)
    sv = np.linalg.svd(X[np.ix_(Bsel, Fsel)], compute_uv=False)
    assert sv[2 * m] < 1e-10 * sv[0]              # numerical rank <= 2m
    assert sv[2 * m - 1] > 1e-14 * sv[0]          # and the bound is not vacuous
    # the full diagonal block (two slabs + the line operator) has rank <= 4m + 2
    Td, _, _ = oracle_mod.reduced_system(A, 2, n, b)
    sv2 = np.linalg.svd(Td[2][np.ix_(Bsel, Fsel)], compute_uv=False)
    assert sv2[4 * m + 2] < 1e-10 * sv2[0]


# --------------------------------------------------------------------------- sweep (Alg. 1/2)

def test_sweep_on_random_block_tridiagonal(oracle_mod):
    rng = np.random.default_rng(3)
    N, s = 6, 5
    Td = [rng.standard_normal((s, s)) + 6 * np.eye(s) for _ in range(N)]
    Tu = [rng.standard_normal((s, s)) for _ in range(N - 1)]
    Tl = [rng.standard_normal((s, s)) for _ in range(N - 1)]     # nonsymmetric on purpose
    Tfull = np.zeros((N * s, N * s))
    for j in range(N):
        Tfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = Td[j]
        if j + 1 < N:
            Tfull[j * s:(j + 1) * s, (j + 1) * s:(j + 2) * s] = Tu[j]
            Tfull[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Tl[j]
    F = rng.standard_normal((2, N * s))
    Sinv = oracle_mod.sweep_build(Td, Tl, Tu)
    ut = oracle_mod.sweep_solve(Tl, Tu, Sinv, [F[:, j * s:(j + 1) * s] for j in range(N)])
    np.testing.assert_allclose(np.concatenate(ut, axis=1), np.linalg.solve(Tfull, F.T).T, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("dim,n,b,kind", [(2, 32, 8, 1), (2, 24, 4, 2), (2, 16, 4, 0), (3, 8, 4, 1), (3, 8, 2, 2)])
def test_slab_method_equals_banded_lu(oracle_mod, dim, n, b, kind):
    """Algorithms 3+4 with exact T reproduce u = A^-1 f (the direct method is exact)."""
    kappa = np.exp(inputs.fourier_field(dim, n, 6, seed=12)) if kind == 1 else None
    c = 1.0 + 0.3 * inputs.fourier_field(dim, n, 5, seed=13, normalize="maxabs") if kind == 2 else None
    omega = 2 * math.pi * n / 10 if kind == 2 else 0.0
    p = inputs.Problem("t", dim, n, b, kind, kappa=kappa, c=c, omega=omega,
                       f=inputs.normal_rhs(dim, n, 2, 14))
    u_slab, parts = oracle_mod.slab_solve(p)
    u_band = oracle_mod.solve(p)
    np.testing.assert_allclose(u_slab, u_band, rtol=0, atol=1e-10 * np.abs(u_band).max())
    A = oracle_mod.assemble_problem(p)
    assert oracle_mod.relres(A, u_slab, p.f).max() < 1e-11


# --------------------------------------------------------------------------- gradient

def test_gradient_matches_central_differences(oracle_mod):
    n = 8
    kappa = np.exp(inputs.fourier_field(2, n, 4, seed=31))
    p = inputs.Problem("g", 2, n, 4, 1, kappa=kappa, f=inputs.normal_rhs(2, n, 1, 32))
    ut = inputs.normal_rhs(2, n, 1, 33)
    L, u, lam, g = oracle_mod.adjoint_gradient(p, ut)
    A = oracle_mod.assemble_problem(p)
    delta = 1e-6
    rng = np.random.default_rng(34)
    nodes = [(0, 3), (n, 5), (2, 0)] + [tuple(v) for v in rng.integers(1, n, size=(6, 2))]
    fd, ad = [], []
    for (x, y) in nodes:
        kp = kappa.copy(); kp[y, x] += delta
        km = kappa.copy(); km[y, x] -= delta
        up = oracle_mod.solve(inputs.Problem("g", 2, n, 4, 1, kappa=kp, f=p.f))
        um = oracle_mod.solve(inputs.Problem("g", 2, n, 4, 1, kappa=km, f=p.f))
        # L(k+d) - L(k-d) = sum (u+ - u-)(u+ + u- - 2 u_t), free of cancellation in the loss
        fd.append(np.sum((up - um) * (up + um - 2 * ut)) / (2 * delta))
        ad.append(g[y, x])
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) / np.linalg.norm(fd) < 1e-6
    # the adjoint solves the transposed system
    assert oracle_mod.relres(A, lam, 2 * (u - ut)).max() < 1e-12


# --------------------------------------------------------------------------- inputs

def test_input_generators_are_seeded():
    a = inputs.fourier_field(2, 64, 16, seed=2)
    b = inputs.fourier_field(2, 64, 16, seed=2)
    np.testing.assert_array_equal(a, b)
    assert abs(a.mean()) < 1e-12 and abs(a.std() - 1) < 1e-12
    r = inputs.fourier_field(3, 16, 8, seed=3, normalize="maxabs")
    assert abs(np.abs(r).max() - 1) < 1e-15
    f1 = inputs.normal_rhs(2, 32, 3, 9)
    np.testing.assert_array_equal(f1, inputs.normal_rhs(2, 32, 3, 9))
    assert f1.shape == (3, 31 * 31)
    ps = inputs.point_source(2, 8)
    assert ps.sum() == 64 and ps.reshape(7, 7)[3, 3] == 64


def _grid_nodes(dim, n):
    t = np.arange(n + 1) / n
    if dim == 2:
        Y, X = np.meshgrid(t, t, indexing="ij")
        return X.ravel(), Y.ravel(), None
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _interior(dim, n, v):
    if dim == 2:
        return v.reshape(n + 1, n + 1)[1:n, 1:n].ravel()
    return v.reshape(n + 1, n + 1, n + 1)[1:n, 1:n, 1:n].ravel()


@pytest.mark.parametrize("dim,n", [(2, 12), (2, 17), (3, 7)])
def test_boundary_lift_reproduces_the_full_stencil_on_cubics(oracle_mod, dim, n):
    """Sec. 1.1 with u = g on the boundary: for a cubic v the five/seven-point Laplacian is
    exact, so h^-2 sum_Q (v_P - v_Q) over all neighbours equals -Lap v.  Over the interior
    neighbours that sum is A v_I (oracle assembly, whose diagonal counts every face); the boundary
    neighbours add -h^-2 sum k g_Q = -lift.  Hence lift(v on the boundary) = A v_I + (Lap v)_I,
    which pins the lift's neighbours, sign and h^-2 scale."""
    X, Y, Z = _grid_nodes(dim, n)
    if dim == 2:
        v = X ** 3 - 2 * X * Y ** 2 + 0.5 * Y ** 3 + X * Y - 0.3 * X + 1.0
        lap = 6 * X - 4 * X + 3 * Y                     # v_xx + v_yy
    else:
        v = X ** 3 - 2 * X * Y ** 2 + 0.5 * Z ** 3 + X * Y * Z - Y * Z + 0.7
        lap = 6 * X - 4 * X + 3 * Z
    A = oracle_mod.assemble(dim, n, oracle_mod.POISSON)
    lifted = oracle_mod.boundary_lift(dim, n, oracle_mod.POISSON, v[None, :])
    expect = A.matvec(_interior(dim, n, v)[None, :]) + _interior(dim, n, lap)[None, :]
    assert np.abs(lifted - expect).max() <= 1e-9 * n * n * np.abs(v).max()


@pytest.mark.parametrize("dim,n,kind", [(2, 16, 1), (2, 9, 2), (3, 6, 1), (3, 5, 2)])
def test_boundary_lift_of_a_constant(oracle_mod, dim, n, kind):
    """For any coefficients the full operator maps the constant 1 to q (the face terms cancel),
    so A 1 - lift(1) = q: the lift uses the same face coefficients k_PQ as the assembled A."""
    rng = np.random.default_rng(n + 10 * kind)
    nodes = (n + 1) ** dim
    kappa = np.exp(rng.standard_normal(nodes)) if kind == 1 else None
    c = 1.0 + 0.2 * rng.random(nodes)
    omega = 3.0 if kind == 2 else 0.0
    A = oracle_mod.assemble(dim, n, kind, kappa=kappa, c=c, omega=omega)
    one = np.ones((1, nodes))
    lifted = oracle_mod.boundary_lift(dim, n, kind, one, kappa=kappa)
    q = -(omega / _interior(dim, n, c)) ** 2 if kind == 2 else np.zeros((n - 1) ** dim)
    got = A.matvec(np.ones((1, (n - 1) ** dim))) - lifted
    assert np.abs(got - q[None, :]).max() <= 1e-10 * n * n * (1.0 if kappa is None else kappa.max())


def test_boundary_lift_adds_to_the_load(oracle_mod):
    """f_out = f + lift(g), for several right-hand sides."""
    n = 10
    rng = np.random.default_rng(3)
    g = rng.standard_normal((3, (n + 1) ** 2))
    f = rng.standard_normal((3, (n - 1) ** 2))
    a = oracle_mod.boundary_lift(2, n, oracle_mod.POISSON, g, f=f)
    b = oracle_mod.boundary_lift(2, n, oracle_mod.POISSON, g) + f
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_bessel_j0_discrete_solution_converges_at_second_order(oracle_mod):
    """The J_0 benchmark (Sec. 6.1): the oracle's solution of the lifted interior system
    approaches u_true at O(h^2) at fixed wavenumber 27.1 (halving h divides the error by a factor
    approaching 4 from below as the pollution term settles: 3.26 from n = 128 to 256), which pins
    the Helmholtz sign, the h^-2 scale and the lift with non-zero boundary data; a wrong sign of
    the k^2 term or of the lift leaves no convergence at all."""
    errs = []
    for n in (128, 256):
        d = inputs.bessel_j0(n, 16)
        p = d["problem"]
        f = oracle_mod.boundary_lift(2, n, p.kind, d["g"])
        u = oracle_mod.solve(p, f)
        errs.append(np.linalg.norm(u - d["u_true"]) / np.linalg.norm(d["u_true"]))
    assert 3.0 <= errs[0] / errs[1] <= 4.3, errs
    assert errs[1] < 0.05, errs
