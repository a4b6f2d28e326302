"""Adjoint gradients (A9) on instances of the batched adjoint workload.

Each instance: -div(kappa grad u) = f on an n x n grid (n drawn from {256, 384, 512,
768, 1024}), b = 16, lognormal kappa from a seeded 16-mode field, f and the target
u_t ~ N(0,1), loss L = ||u - u_t||^2.  The gradient dL/dkappa from slab_adjoint is
checked against central finite differences (steps 1e-4 and 1e-6) on seeded interior
probe nodes (tolerance 1e-6 relative over the probes), against the oracle's adjoint
gradient (FP64 banded LU), and through the autograd Function.
"""
import numpy as np
import pytest
import torch

import oracle
from fdcheck import fd_operator_difference
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(n, b, kappa):
    from paper_2211_07572_gb300.solver import SlabSolver
    return SlabSolver(2, n, b, inputs.DIFFUSION, kappa=kappa, precision="fp32", rtol=1e-14, max_refine=40)


# Central differences L(k+d) - L(k-d) with the difference of the two forward solutions formed
# without cancellation:  u+ - u- = -A(k+d)^{-1} (A(k+d) - A(k-d)) u-, the operator difference
# applied in closed form (fd_operator_difference), and the loss difference
# sum (u+ - u-)(u+ + u- - 2 u_t), which has no cancellation either.  (u- is the exact solution for
# the load f - r-, r- its residual of relative size <= 1e-13; the gradient at that load differs
# from the one at f by that relative amount.)  The remaining FD error is the O(d^2) truncation,
# below 1e-8 relative at both steps for kappa >= 0.03.
@pytest.mark.parametrize("inst,delta,tol", [(0, 1e-4, 1e-6), (1, 1e-4, 1e-6), (0, 1e-6, 1e-6)])
def test_adjoint_gradient_vs_central_differences(inst, delta, tol):
    assert torch.cuda.is_available()
    sizes = inputs.adjoint_batch_sizes()
    n = int(min(sizes[inst], 384))               # the two smallest sizes keep the test short
    d = inputs.adjoint_instance(inst, n)
    kappa = d["kappa"]
    f = torch.from_numpy(d["f"]).cuda()
    ut = torch.from_numpy(d["u_target"]).cuda()
    s = _solver(n, d["b"], kappa)
    u, _, _ = s.solve(f, allow_noconv=True)
    lam, g = s.adjoint(2 * (u - ut), u, allow_noconv=True)
    g = g.cpu().numpy()
    s.close()
    fd, ad = [], []
    for (x, y) in d["probes"][:8]:
        kp = kappa.copy(); kp[y, x] += delta
        km = kappa.copy(); km[y, x] -= delta
        sm = _solver(n, d["b"], km)
        um, _, _ = sm.solve(f, allow_noconv=True)
        sm.close()
        sp = _solver(n, d["b"], kp)
        dAu = torch.from_numpy(fd_operator_difference(um.cpu().numpy(), kp, km, x, y, n)).cuda()
        du, _, _ = sp.solve(-dAu, allow_noconv=True)
        sp.close()
        fd.append(float((du * (2 * um + du - 2 * ut)).sum()) / (2 * delta))
        ad.append(g[y, x])
    fd, ad = np.array(fd), np.array(ad)
    rel = np.linalg.norm(fd - ad) / np.linalg.norm(fd)
    assert rel <= tol, (rel, fd, ad)


def test_adjoint_gradient_matches_oracle_on_instance():
    n = 256
    d = inputs.adjoint_instance(3, n)
    p = inputs.Problem("adjoint", 2, n, d["b"], inputs.DIFFUSION, kappa=d["kappa"], f=d["f"])
    L, u_o, lam_o, g_o = oracle.adjoint_gradient(p, d["u_target"])
    s = _solver(n, d["b"], d["kappa"])
    u, _, _ = s.solve(torch.from_numpy(d["f"]).cuda(), allow_noconv=True)
    lam, g = s.adjoint(2 * (u - torch.from_numpy(d["u_target"]).cuda()), u, allow_noconv=True)
    s.close()
    assert np.abs(u.cpu().numpy() - u_o).max() <= 1e-9 * np.abs(u_o).max()
    assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-8 * np.abs(g_o).max()


def test_autograd_function_backward_is_the_adjoint():
    from paper_2211_07572_gb300.solver import SlabSolveFunction
    n, b = 64, 16
    d = inputs.adjoint_instance(5, 256)
    kappa = torch.from_numpy(np.exp(inputs.fourier_field(2, n, 16, seed=1005))).cuda().requires_grad_(True)
    f = torch.from_numpy(inputs.normal_rhs(2, n, 1, 2005)).cuda().requires_grad_(True)
    ut = torch.from_numpy(inputs.normal_rhs(2, n, 1, 3005)).cuda()
    u = SlabSolveFunction.apply(kappa, f, n, b)
    loss = ((u - ut) ** 2).sum()
    gk, gf = torch.autograd.grad(loss, (kappa, f))
    p = inputs.Problem("a", 2, n, b, inputs.DIFFUSION, kappa=kappa.detach().cpu().numpy(),
                       f=f.detach().cpu().numpy())
    L, u_o, lam_o, g_o = oracle.adjoint_gradient(p, ut.cpu().numpy())
    assert abs(loss.item() - L) <= 1e-9 * L
    assert np.abs(gk.cpu().numpy() - g_o).max() <= 1e-8 * np.abs(g_o).max()
    assert np.abs(gf.cpu().numpy() - lam_o).max() <= 1e-8 * np.abs(lam_o).max()   # dL/df = lambda
    del d
