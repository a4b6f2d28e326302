"""Helper of the central-difference gradient checks (imported by the adjoint tests)."""
import numpy as np


def fd_operator_difference(u, kappa_plus, kappa_minus, x, y, n):
    """(A(kappa+) - A(kappa-)) u for kappas that differ only at the interior node (x, y), in closed
    form: only the four faces at that node change, each face coefficient (mean of its two node
    values) by dk = (kappa+_p - kappa-_p) / 2 (exact: the two values are within a factor 2), so
    row p gets n^2 dk (u_p - u_q) and row q gets n^2 dk (u_q - u_p) for each neighbour q (boundary
    values 0, boundary rows absent).  Subtracting two full stencil applies instead leaves rounding
    of size eps |A u| in the five changed rows, which is not small against a difference of size
    d |u_p - u_q| when the step d is 1e-6."""
    U = np.zeros((n + 1, n + 1))
    U[1:n, 1:n] = np.asarray(u, dtype=np.float64).reshape(n - 1, n - 1)
    dk = 0.5 * (kappa_plus[y, x] - kappa_minus[y, x])
    out = np.zeros((n + 1, n + 1))
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        qx, qy = x + dx, y + dy
        d = dk * (U[y, x] - U[qy, qx]) * float(n) * float(n)
        out[y, x] += d
        out[qy, qx] -= d
    return out[1:n, 1:n].reshape(1, -1)
