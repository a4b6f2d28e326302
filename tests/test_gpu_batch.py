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


# ----------------------------------------------------------------- CUDA-graph batch
def test_graph_batch_matches_handle_path_and_oracle():
    """slab_batch: three waves of uneven problems on two branches, two runs with different inputs
    (the replayed graphs read the current buffers); loss, u and dL/dkappa against the handle-based
    path (slab_factor / slab_solve / slab_adjoint) and the oracle's adjoint gradient."""
    from paper_2211_07572_gb300.solver import GraphBatch, SlabSolver
    sizes = [64, 96, 128, 64, 160]
    gb = GraphBatch(sizes, b=16, rtol=1e-12, steps=5, wave=2, branches=2)
    assert gb.device_bytes > 0
    for run in range(2):
        data = [inputs.adjoint_instance(10 * run + i, n, 16) for i, n in enumerate(sizes)]
        for i, d in enumerate(data):
            gb.set_inputs(i, torch.from_numpy(d["kappa"]).cuda(), torch.from_numpy(d["f"]).cuda(),
                          torch.from_numpy(d["u_target"]).cuda())
        gb.run()
        L, ru, rl = gb.results()
        assert ru.max() <= 1e-12 and rl.max() <= 1e-12, (ru, rl)
        for i, (n, d) in enumerate(zip(sizes, data)):
            u, lam, g = gb.outputs(i)
            s = SlabSolver(2, n, 16, inputs.DIFFUSION, kappa=d["kappa"], precision="fp32", rtol=1e-13, max_refine=40)
            f = torch.from_numpy(d["f"]).cuda()
            ut = torch.from_numpy(d["u_target"]).cuda()
            u1, _, _ = s.solve(f, allow_noconv=True)
            _, g1 = s.adjoint(2 * (u1 - ut), u1, allow_noconv=True)
            s.close()
            L1 = float(((u1 - ut) ** 2).sum())
            assert abs(L[i] - L1) <= 1e-10 * L1
            assert float((u - u1).abs().max()) <= 1e-9 * float(u1.abs().max())
            assert float((g - g1).abs().max()) <= 1e-8 * float(g1.abs().max())
        if run == 1:                                   # one problem against the oracle
            d = data[1]
            q = inputs.Problem("gb", 2, sizes[1], 16, inputs.DIFFUSION, kappa=d["kappa"], f=d["f"])
            L_o, u_o, lam_o, g_o = oracle.adjoint_gradient(q, d["u_target"])
            assert abs(L[1] - L_o) <= 1e-9 * L_o
            assert np.abs(gb.outputs(1)[2].cpu().numpy() - g_o).max() <= 1e-8 * np.abs(g_o).max()
    gb.close()


def test_graph_batch_reports_too_few_refinement_passes():
    """With no refinement pass an FP32 factor leaves a residual far above rtol = 1e-12: the results
    say so (ENOCONV) instead of passing the iterate off as converged."""
    from paper_2211_07572_gb300 import SlabError
    from paper_2211_07572_gb300.solver import GraphBatch
    gb = GraphBatch([64, 96], b=16, rtol=1e-12, steps=0, branches=2)
    for i, n in enumerate([64, 96]):
        d = inputs.adjoint_instance(i, n, 16)
        gb.set_inputs(i, d["kappa"], d["f"], d["u_target"])
    gb.run()
    with pytest.raises(SlabError) as ei:
        gb.results()
    assert ei.value.status == 4
    L, ru, rl = gb.results(allow_noconv=True)
    assert ru.max() > 1e-12 and np.all(L > 0)
    gb.close()


def test_graph_batch_rejects_bad_sizes():
    from paper_2211_07572_gb300 import SlabError
    from paper_2211_07572_gb300.solver import GraphBatch
    with pytest.raises(SlabError) as ei:
        GraphBatch([64, 100], b=16)
    assert ei.value.status == 1
