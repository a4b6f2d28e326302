"""The allocation-free residual entry point agrees with the handle-based one.

slab_residual_norms_noalloc is for callers that cannot call cudaMalloc (a stream
capture without allocation nodes, a device pool owned by another framework, a
real-time loop).  It keeps its reduction scratch in a fixed array inside the
library.  For each operator kind (Poisson, diffusion, Helmholtz) this test calls it
twice in a row through the C ABI with k = 11 loads -- two right-hand-side groups of
the reduction, the second one partial -- and compares the residual with
slab_apply_residual and the norms with the relative residual the handle-based solve
reports and with torch's norms of the same vectors, at the tolerance of the other
parity tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2211_07572_gb300 import inputs

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("kind", [inputs.POISSON, inputs.DIFFUSION, inputs.HELMHOLTZ])
def test_noalloc_residual_matches_handle_path_twice(kind):
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2211_07572_gb300 import _lib
    from paper_2211_07572_gb300.solver import SlabSolver
    lib = _lib.load()
    n, b, k = 128, 16, 11
    kappa = c = None
    omega = 0.0
    if kind == inputs.DIFFUSION:
        kappa = np.exp(inputs.fourier_field(2, n, 8, seed=91))
    elif kind == inputs.HELMHOLTZ:
        hp = inputs.helmholtz(n, b, dim=2, n_modes=8, field_seed=93)
        c, omega = hp.c, hp.omega
    f = torch.from_numpy(inputs.normal_rhs(2, n, k, 92)).cuda()
    s = SlabSolver(2, n, b, kind, kappa=kappa, c=c, omega=omega, precision="fp32", max_refine=0)
    u, relres, _ = s.solve(f, allow_noconv=True)      # one pass: the residual is far from zero
    kd = None if kappa is None else torch.from_numpy(kappa).cuda()
    cd = None if c is None else torch.from_numpy(c).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        uu = u if call == 0 else u * 0.5               # second call: different data, same scratch
        r = torch.empty_like(f)
        nr = torch.empty(k, dtype=torch.float64, device="cuda")
        nf = torch.empty(k, dtype=torch.float64, device="cuda")
        st = lib.slab_residual_norms_noalloc(n, kind, _p(kd), _p(cd), omega, _p(uu), _p(f), _p(r), k,
                                             _p(nr), _p(nf), ctypes.c_void_p(stream))
        assert st == 0, st
        r_ref = s.residual(uu, f)
        torch.cuda.synchronize()
        scale = float(s.apply(uu).abs().max())
        # the two residual kernels round differently, by up to about eps |A u| per entry
        assert float((r - r_ref).abs().max()) <= 1e-13 * scale
        rel = np.sqrt(nr.cpu().numpy() / nf.cpu().numpy())
        if call == 0:
            # per entry the residuals differ by up to 1e-13 |A u| while |r| ~ 1e-6 |A u| after one FP32
            # pass, so the two relative residuals agree to about 1e-7
            np.testing.assert_allclose(rel, relres, rtol=1e-7)
        # the reduction itself: the squared norms of the kernel's own residual and load
        np.testing.assert_allclose(nr.cpu().numpy(), (r * r).sum(dim=1).cpu().numpy(), rtol=1e-12)
        np.testing.assert_allclose(nf.cpu().numpy(), (f * f).sum(dim=1).cpu().numpy(), rtol=1e-12)
    # requests beyond the fixed scratch are rejected before any launch
    big = lib.slab_residual_norms_noalloc(4097, inputs.POISSON, None, None, 0.0, _p(u), _p(f), _p(r), 100000,
                                          _p(nr), _p(nf), None)
    assert big == _lib.SLAB_EINVAL
    s.close()
