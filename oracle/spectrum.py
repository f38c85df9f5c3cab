"""Closed-form spectrum of the Q1 discretisation of -Laplace on (0,1)^d, Dirichlet.

The 1D P1 pencil on a uniform mesh (h = 1/n, interior nodes) is
K1 = (1/h) tridiag(-1, 2, -1), M1 = (h/6) tridiag(1, 4, 1).  Both are diagonalised by
the discrete sines v_k(x_i) = sin(k pi x_i), k = 1..n-1, with eigenvalues
(2/h)(1 - cos k pi h) and (h/3)(2 + cos k pi h), so K1 v = mu_k M1 v with
mu_k = (6/h^2)(1 - cos k pi h)/(2 + cos k pi h).
The Q1 stiffness is sum_j (x)_i (K1 if i==j else M1) and the mass (x)_i M1, so the
tensor products of the sines are the eigenvectors of the d-dimensional pencil and
lambda_{k_1..k_d} = sum_j mu_{k_j}.  (This is the exact discrete spectrum of the
model problem of §2.1 / §6.1 on the uniform Q1 mesh.)
"""
import numpy as np


def mu_1d(n: int) -> np.ndarray:
    h = 1.0 / n
    k = np.arange(1, n)
    c = np.cos(k * np.pi * h)
    return (6.0 / h ** 2) * (1.0 - c) / (2.0 + c)


def q1_laplace_eigenvalues(d: int, n: int, count: int | None = None) -> np.ndarray:
    """All (or the `count` smallest) eigenvalues of the Q1 Laplace pencil, ascending."""
    mu = mu_1d(n)
    lam = mu
    for _ in range(d - 1):
        lam = (lam[..., None] + mu).reshape(-1)
    lam = np.sort(lam)
    return lam if count is None else lam[:count]


def q1_laplace_multiindices(d: int, n: int, count: int):
    """Multi-indices (k_1..k_d) of the `count` smallest eigenvalues (ties by index)."""
    mu = mu_1d(n)
    grids = np.meshgrid(*([np.arange(1, n)] * d), indexing="ij")
    lam = sum(mu[g - 1] for g in grids).reshape(-1)
    ks = np.stack([g.reshape(-1) for g in grids], axis=1)
    order = np.lexsort(tuple(ks[:, j] for j in reversed(range(d))) + (lam,))
    return lam[order[:count]], ks[order[:count]]
