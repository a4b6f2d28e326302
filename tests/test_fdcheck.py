"""The closed-form operator difference of the central-difference checks equals the difference of
the oracle's assembled operators (CPU)."""
import numpy as np

from fdcheck import fd_operator_difference
from paper_2211_07572_gb300 import inputs


def test_operator_difference_matches_assembled_matrices(oracle_mod):
    n, delta = 24, 1e-3
    kappa = np.exp(inputs.fourier_field(2, n, 8, seed=7))
    u = inputs.normal_rhs(2, n, 1, 8)[0]
    for (x, y) in ((1, 1), (5, 17), (n - 1, 3), (12, n - 1)):      # corners and edges included
        kp = kappa.copy(); kp[y, x] += delta
        km = kappa.copy(); km[y, x] -= delta
        Ap = oracle_mod.assemble(2, n, inputs.DIFFUSION, kappa=kp)
        Am = oracle_mod.assemble(2, n, inputs.DIFFUSION, kappa=km)
        ref = Ap.matvec(u) - Am.matvec(u)
        got = fd_operator_difference(u, kp, km, x, y, n)[0]
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
        assert np.count_nonzero(got) <= 5
