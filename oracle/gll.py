"""Gauss-Lobatto-Legendre nodes, weights and derivative matrix (FP64).

Test infrastructure only (see the package docstring).

The SEM uses the local nodes of the element as its quadrature points
(Section 4.2, Eq. numerical_integ and the remark after Eq. dual_sys); for
tensor-product quads these are the GLL points of order p in each direction.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as _leg


def legendre_value(p: int, x):
    """P_p(x) by Bonnet's three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if p == 0:
        return p0
    p1 = x.copy()
    for k in range(1, p):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def gll_nodes(p: int) -> np.ndarray:
    """The p+1 GLL nodes on [-1, 1]: the endpoints and the roots of P_p'."""
    if p < 1:
        raise ValueError("order must be >= 1")
    dp = _leg.Legendre.basis(p).deriv()
    inner = np.sort(np.real(dp.roots())) if p > 1 else np.zeros(0)
    # polish the library roots with Newton on P_p' (P_p'' from the Legendre ODE)
    for _ in range(3):
        if inner.size == 0:
            break
        d1 = _leg.legval(inner, dp.coef)
        d2 = _leg.legval(inner, dp.deriv().coef)
        inner = inner - d1 / d2
    x = np.concatenate([[-1.0], inner, [1.0]])
    # exact symmetry: x_k = -x_{p-k}
    x = 0.5 * (x - x[::-1])
    return x


def gll_weights(p: int, x: np.ndarray | None = None) -> np.ndarray:
    """w_k = 2 / (p (p+1) P_p(x_k)^2)."""
    if x is None:
        x = gll_nodes(p)
    return 2.0 / (p * (p + 1) * legendre_value(p, x) ** 2)


def derivative_matrix(x: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(x_i) for the Lagrange basis on nodes x (barycentric form)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    bw = 1.0 / np.prod(diff, axis=1)            # barycentric weights
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (bw[j] / bw[i]) / (x[i] - x[j])
        D[i, i] = -sum(D[i, j] for j in range(n) if j != i)
    return D


def lagrange_values(x: np.ndarray, t) -> np.ndarray:
    """L[k, j] = l_j(t_k): the nodal basis on nodes x evaluated at points t."""
    x = np.asarray(x, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    L = np.ones((t.size, x.size))
    for j in range(x.size):
        for m in range(x.size):
            if m != j:
                L[:, j] *= (t - x[m]) / (x[j] - x[m])
    return L
