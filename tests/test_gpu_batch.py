"""Batches of independent problems (the batched adjoint workload): slab_factor_batched /
slab_solve_batched / slab_adjoint_batched against the single-problem path and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [64, 96, 128, 64, 160]


def _problems(sizes, b=16, base=0):
    probs, fs, uts = [], [], []
    for i, n in enumerate(sizes):
        d = inputs.adjoint_instance(base + i, n, b)
        probs.append(dict(dim=2, n=n, b=b, kind=inputs.DIFFUSION, kappa=d["kappa"]))
        fs.append(torch.from_numpy(d["f"]).cuda())
        uts.append(torch.from_numpy(d["u_target"]).cuda())
    return probs, fs, uts


def test_batch_matches_single_problem_path():
    from paper_2211_07572_gb300.solver import SlabSolver, batched_adjoint_gradients
    probs, fs, uts = _problems(SIZES)
    losses, grads = batched_adjoint_gradients(probs, fs, uts, wave=3, workers=4)
    for p, f, ut, L, g in zip(probs, fs, uts, losses, grads):
        s = SlabSolver(2, p["n"], p["b"], p["kind"], kappa=p["kappa"], precision="fp32", rtol=1e-12, max_refine=40,
                       stage2="sweep")
        u, _, _ = s.solve(f, allow_noconv=True)
        _, g1 = s.adjoint(2 * (u - ut), u, allow_noconv=True)
        s.close()
        assert abs(L - float(((u - ut) ** 2).sum())) <= 1e-12 * L
        assert torch.allclose(g, g1, rtol=0, atol=1e-12 * float(g1.abs().max()))


def test_batch_gradient_matches_oracle():
    from paper_2211_07572_gb300.solver import batched_adjoint_gradients
    probs, fs, uts = _problems([96, 128], base=7)
    losses, grads = batched_adjoint_gradients(probs, fs, uts, wave=2, workers=2)
    for p, f, ut, L, g in zip(probs, fs, uts, losses, grads):
        q = inputs.Problem("batch", 2, p["n"], p["b"], inputs.DIFFUSION, kappa=p["kappa"], f=f.cpu().numpy())
        L_o, u_o, lam_o, g_o = oracle.adjoint_gradient(q, ut.cpu().numpy())
        assert abs(L - L_o) <= 1e-9 * L_o
        assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-8 * np.abs(g_o).max()


def test_batch_reports_invalid_problem():
    from paper_2211_07572_gb300 import SlabError
    from paper_2211_07572_gb300.solver import SlabBatch
    probs, _, _ = _problems([64, 96])
    probs.append(dict(dim=2, n=100, b=16, kind=inputs.DIFFUSION, kappa=np.ones((101, 101))))   # 16 does not divide 100
    with pytest.raises(SlabError) as ei:
        SlabBatch(probs)
    assert ei.value.status == 1
