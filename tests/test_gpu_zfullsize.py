"""Full-size cases in the launch configuration the benchmark times (2-D diffusion n = 2048,
b = 32, 64 loads; 3-D diffusion n = 96, b = 8, 16 loads).  The oracle cannot factor these (a
137 GB / 124 GB band), so the pin is a property that holds at any size: the relative residual
||f - A u|| / ||f|| <= 1e-10, computed by the oracle's own CSR assembly and matvec (no code in
common with the CUDA residual kernel) on sampled right-hand sides of the library's solution.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,b,k,modes,field_seed,rhs_seed",
                         [(2, 2048, 32, 64, 16, 2, 102), (3, 96, 8, 16, 8, 4, 104)])
def test_full_size_residual_by_the_oracle(dim, n, b, k, modes, field_seed, rhs_seed):
    from paper_2211_07572_gb300.solver import SlabSolver
    p = inputs.diffusion(n, b, k=0, dim=dim, n_modes=modes, field_seed=field_seed, rhs_seed=rhs_seed)
    f = inputs.normal_rhs(dim, n, k, rhs_seed)
    s = SlabSolver(dim, n, b, inputs.DIFFUSION, kappa=p.kappa, rtol=1e-10, max_refine=40)
    u, rel, _ = s.solve(torch.from_numpy(f).cuda())
    s.close()
    idx = [0, k // 3, 2 * k // 3, k - 1]
    us = u[idx].cpu().numpy()
    del u
    assert np.max(rel) <= 1e-10
    A = oracle.assemble(dim, n, inputs.DIFFUSION, kappa=p.kappa)
    ro = oracle.relres(A, us, f[idx])
    assert ro.max() <= 1e-10, ro
