"""Seeded synthetic inputs for the slab solver workloads.

This module only draws numbers: smooth random coefficient fields, random
right-hand sides and point sources, each from an explicit seed.  It holds none
of the solver's arithmetic (no stencil, no elimination), so both the CUDA path
and the CPU oracle can be fed from it without sharing method code.

Conventions (shared by every consumer):
  * unit domain [0,1]^d, n grid intervals per side, h = 1/n;
  * node fields (kappa, c) are given at all (n+1)^d nodes including the
    boundary, C order [z][y][x] (x fastest);
  * vectors (f, u) live on the (n-1)^d interior nodes, C order [k][z][y][x].

The random field follows the workload recipe: g(x) = sum_q a_q cos(2 pi k_q.x +
phi_q) with integer wavenumbers k_q drawn uniformly from {1..kmax}^d, phases
uniform on [0, 2 pi), amplitudes standard normal; it is then normalised either
to zero sample mean and unit sample variance over the nodes ("var") or to
max |g| = 1 ("maxabs").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

POISSON, DIFFUSION, HELMHOLTZ, CONVECTION = 0, 1, 2, 3
KIND_NAMES = {POISSON: "poisson", DIFFUSION: "diffusion", HELMHOLTZ: "helmholtz", CONVECTION: "convection"}


def fourier_field(dim: int, n: int, n_modes: int, seed: int, kmax: int = 8,
                  normalize: str = "var") -> np.ndarray:
    """Smooth random field at the (n+1)^d nodes, shape (n+1,)*dim, float64."""
    rng = np.random.default_rng(seed)
    kq = rng.integers(1, kmax + 1, size=(n_modes, dim))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    amp = rng.standard_normal(n_modes)
    x = np.arange(n + 1, dtype=np.float64) / n
    g = np.zeros((n + 1,) * dim, dtype=np.float64)
    for q in range(n_modes):
        # cos(2 pi k.x + phi) as the real part of a separable product
        acc = np.exp(1j * phi[q]) * np.ones((1,) * dim, dtype=np.complex128)
        for ax in range(dim):
            e = np.exp(2j * math.pi * kq[q, ax] * x)
            shape = [1] * dim
            shape[dim - 1 - ax] = n + 1       # axis 0 of the node array is the slowest (z / y)
            acc = acc * e.reshape(shape)
        g += amp[q] * acc.real
    if normalize == "var":
        g = (g - g.mean()) / g.std()
    elif normalize == "maxabs":
        g = g / np.abs(g).max()
    else:
        raise ValueError(normalize)
    return g


def normal_rhs(dim: int, n: int, k: int, seed: int, dtype=np.float64) -> np.ndarray:
    """k i.i.d. N(0,1) right-hand sides on the interior nodes, shape (k, (n-1)^d)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, (n - 1) ** dim), dtype=dtype)


def sine_rhs(dim: int, n: int) -> np.ndarray:
    """f = d pi^2 prod sin(pi x_a) on the interior nodes (u = prod sin(pi x_a) solves -Lap u = f)."""
    x = np.arange(1, n, dtype=np.float64) / n
    s = np.sin(math.pi * x)
    v = s
    for _ in range(dim - 1):
        v = np.multiply.outer(s, v)
    return (dim * math.pi ** 2 * v).reshape(1, -1)


def sine_solution(dim: int, n: int) -> np.ndarray:
    """u = prod sin(pi x_a) on the interior nodes, shape (1, (n-1)^d)."""
    x = np.arange(1, n, dtype=np.float64) / n
    s = np.sin(math.pi * x)
    v = s
    for _ in range(dim - 1):
        v = np.multiply.outer(s, v)
    return v.reshape(1, -1)


def point_source(dim: int, n: int) -> np.ndarray:
    """f = h^-d at the centre node (n/2, ...), zero elsewhere; shape (1, (n-1)^d)."""
    f = np.zeros((n - 1,) * dim, dtype=np.float64)
    f[(n // 2 - 1,) * dim] = float(n) ** dim
    return f.reshape(1, -1)


@dataclass
class Problem:
    """One elliptic problem: operator data on the nodes plus right-hand sides."""
    name: str
    dim: int
    n: int
    b: int
    kind: int
    kappa: Optional[np.ndarray] = None      # (n+1)^d nodes, DIFFUSION and CONVECTION
    c: Optional[np.ndarray] = None          # (n+1)^d nodes, HELMHOLTZ only
    beta: Optional[np.ndarray] = None       # (d, (n+1)^d) velocity components x, y(, z), CONVECTION only
    omega: float = 0.0
    f: Optional[np.ndarray] = None          # (k, (n-1)^d)
    u_exact: Optional[np.ndarray] = None    # closed-form continuous solution where known
    meta: dict = field(default_factory=dict)

    @property
    def k(self) -> int:
        return 0 if self.f is None else self.f.shape[0]

    @property
    def unknowns(self) -> int:
        return (self.n - 1) ** self.dim


def poisson_sine(n: int = 128, b: int = 16, dim: int = 2) -> Problem:
    """-Lap u = f on the unit square/cube with u = prod sin(pi x_a) (Dirichlet 0)."""
    return Problem(name=f"poisson{dim}d_n{n}_b{b}", dim=dim, n=n, b=b, kind=POISSON,
                   f=sine_rhs(dim, n), u_exact=sine_solution(dim, n))


def diffusion(n: int, b: int, k: int, dim: int = 2, n_modes: int = 16,
              field_seed: int = 2, rhs_seed: int = 102) -> Problem:
    """-div(kappa grad u) = f with kappa = exp(g), g a unit-variance Fourier field."""
    g = fourier_field(dim, n, n_modes, field_seed, normalize="var")
    f = normal_rhs(dim, n, k, rhs_seed) if k > 0 else None
    return Problem(name=f"diffusion{dim}d_n{n}_b{b}_k{k}", dim=dim, n=n, b=b, kind=DIFFUSION,
                   kappa=np.exp(g), f=f, meta=dict(n_modes=n_modes, field_seed=field_seed,
                                                   rhs_seed=rhs_seed))


def helmholtz(n: int, b: int, dim: int = 2, n_modes: int = 8, field_seed: int = 3,
              ppw: float = 10.0, contrast: float = 0.3) -> Problem:
    """-Lap u - (omega/c)^2 u = f, c = 1 + contrast*r (r max-abs normalised), point source."""
    r = fourier_field(dim, n, n_modes, field_seed, normalize="maxabs")
    omega = 2.0 * math.pi * n / ppw
    return Problem(name=f"helmholtz{dim}d_n{n}_b{b}", dim=dim, n=n, b=b, kind=HELMHOLTZ,
                   c=1.0 + contrast * r, omega=omega, f=point_source(dim, n),
                   meta=dict(n_modes=n_modes, field_seed=field_seed, ppw=ppw))


def convection(n: int, b: int, k: int, dim: int = 2, speed: float = 20.0, n_modes: int = 16,
               field_seed: int = 6, velocity_seeds=(7, 8, 9), rhs_seed: int = 106) -> Problem:
    """-div(kappa grad u) + beta.grad u = f: kappa = exp(g) (g a unit-variance Fourier field, as the
    diffusion workload), velocity components beta_a = speed * r_a with r_a 8-mode fields normalised
    to max |r_a| = 1, f ~ N(0,1)."""
    g = fourier_field(dim, n, n_modes, field_seed, normalize="var")
    beta = np.stack([speed * fourier_field(dim, n, 8, velocity_seeds[a], normalize="maxabs")
                     for a in range(dim)])
    f = normal_rhs(dim, n, k, rhs_seed) if k > 0 else None
    return Problem(name=f"convection{dim}d_n{n}_b{b}_k{k}", dim=dim, n=n, b=b, kind=CONVECTION,
                   kappa=np.exp(g), beta=beta, f=f,
                   meta=dict(speed=speed, n_modes=n_modes, field_seed=field_seed, rhs_seed=rhs_seed))


def constant_helmholtz(n: int, b: int, omega: float, rhs_seed: int = 7, k: int = 1) -> Problem:
    """Constant-coefficient Helmholtz (c = 1) with random right-hand sides."""
    return Problem(name=f"helmholtz_const_n{n}_b{b}", dim=2, n=n, b=b, kind=HELMHOLTZ,
                   c=np.ones((n + 1, n + 1)), omega=omega, f=normal_rhs(2, n, k, rhs_seed))


def bessel_j0(n: int, b: int, wavenumber: float = 27.1, source=(-0.1, 0.5)) -> dict:
    """Constant-coefficient Helmholtz -Lap u - k^2 u = 0 on the unit square with Dirichlet data
    u = J_0(k |x - x_s|), x_s outside the domain (the paper's low-order benchmark PDE, Sec. 6.1,
    eq. "constant_coeff_helm").  Returns the problem (zero load), the data g on all (n+1)^2
    nodes (C order [y][x]) and the true solution at the interior nodes."""
    from scipy.special import j0
    t = np.arange(n + 1) / n
    Y, X = np.meshgrid(t, t, indexing="ij")
    u_nodes = j0(wavenumber * np.hypot(X - source[0], Y - source[1]))
    prob = Problem(name=f"helmholtz_j0_n{n}_b{b}", dim=2, n=n, b=b, kind=HELMHOLTZ, c=np.ones((n + 1, n + 1)),
                   omega=float(wavenumber), f=np.zeros((1, (n - 1) ** 2)),
                   meta=dict(wavenumber=wavenumber, source=tuple(source)))
    return dict(problem=prob, g=u_nodes.reshape(1, -1), u_true=u_nodes[1:n, 1:n].reshape(1, -1))


# The workloads, named by what they are (sizes and seeds fixed here).
def poisson_sine_128() -> Problem:
    """Poisson, n = 128, b = 16, manufactured sine solution."""
    return poisson_sine(128, 16)


def diffusion_2d_2048(k: int = 64, n: int = 2048, b: int = 32) -> Problem:
    """2-D variable-coefficient diffusion, n = 2048, b = 32, 64 random loads."""
    return diffusion(n, b, k, dim=2, n_modes=16, field_seed=2, rhs_seed=102)


def helmholtz_2d_4096(n: int = 4096, b: int = 32) -> Problem:
    """2-D variable-speed Helmholtz, n = 4096, b = 32, 10 points per wavelength, point source."""
    return helmholtz(n, b, dim=2, n_modes=8, field_seed=3)


def diffusion_3d_96(k: int = 16, n: int = 96, b: int = 8) -> Problem:
    """3-D variable-coefficient diffusion, n = 96, b = 8, 16 random loads."""
    return diffusion(n, b, k, dim=3, n_modes=8, field_seed=4, rhs_seed=104)


ADJOINT_BATCH_SIZES = (256, 384, 512, 768, 1024)


def adjoint_batch_sizes(count: int = 256, seed: int = 5) -> np.ndarray:
    """Grid sizes n of the batched adjoint workload's instances (uneven mix)."""
    rng = np.random.default_rng(seed)
    return np.asarray(ADJOINT_BATCH_SIZES)[rng.integers(0, len(ADJOINT_BATCH_SIZES), size=count)]


def adjoint_instance(i: int, n: int, b: int = 16) -> dict:
    """Instance i of the batched adjoint workload: kappa, f, u_target and 32 probe nodes."""
    g = fourier_field(2, n, 16, 1000 + i, normalize="var")
    f = normal_rhs(2, n, 1, 2000 + i)
    ut = normal_rhs(2, n, 1, 3000 + i)
    rng = np.random.default_rng(4000 + i)
    probes = rng.integers(1, n, size=(32, 2))      # interior node (x, y) indices
    return dict(n=n, b=b, kappa=np.exp(g), f=f, u_target=ut, probes=probes)
