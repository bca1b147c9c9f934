"""1D nodal basis on Gauss-Legendre points (oracle; test infrastructure only).

The paper discretises with polynomials of degree k on quadrilaterals (Sec. 3.1,
spaces P^k).  The collocated nodal reading used here puts the (k+1)^d
tensor-product Gauss-Legendre points in the reference element [-1,1]^d and uses
the Lagrange polynomials through them as the basis.

Nodes are the roots of the Legendre polynomial P_n, found by Newton's method
on the three-term recurrence (Bonnet's formula); weights are
w_j = 2 / ((1 - x_j^2) P_n'(x_j)^2).  The derivative matrix
D[i, j] = l_j'(x_i) uses barycentric weights (Berrut & Trefethen 2004):
off-diagonal D[i, j] = (b_j / b_i) / (x_i - x_j), diagonal = minus the sum of
the off-diagonal row entries (so that D annihilates constants).
"""
import math

import numpy as np


def legendre_and_derivative(n, x):
    """P_n(x) and P_n'(x) by Bonnet's recurrence (k+1)P_{k+1} = (2k+1)x P_k - k P_{k-1}."""
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


def gauss_legendre(n):
    """n Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    # Chebyshev-type initial guesses, then Newton on P_n.
    x = np.array([-math.cos(math.pi * (j + 0.75) / (n + 0.5)) for j in range(n)])
    for _ in range(100):
        p, dp = legendre_and_derivative(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_lobatto_points(n):
    """The n Gauss-Lobatto points on [-1, 1] (ascending): the end points and
    the roots of P_{n-1}', here from numpy's Legendre-series routines."""
    if n == 2:
        return np.array([-1.0, 1.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def barycentric_weights(x):
    n = len(x)
    b = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                b[j] /= (x[j] - x[k])
    return b


def lagrange_eval(x, xe):
    """Matrix L[m, j] = l_j(xe_m) of the Lagrange basis through nodes x."""
    n = len(x)
    xe = np.atleast_1d(np.asarray(xe, dtype=np.float64))
    L = np.ones((len(xe), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                L[:, j] *= (xe - x[k]) / (x[j] - x[k])
    return L


def lagrange_derivative_at(x, e):
    """l_j'(e) for every j at a point e that is not a node:
    l_j'(e) = l_j(e) sum_{k != j} 1 / (e - x_k)."""
    n = len(x)
    L = lagrange_eval(x, e)[0]
    return np.array([L[j] * sum(1.0 / (e - x[k]) for k in range(n) if k != j) for j in range(n)])


def derivative_matrix(x):
    """D[i, j] = l_j'(x_i)."""
    n = len(x)
    b = barycentric_weights(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


class Basis1D:
    """Everything the collocated DG operator needs along one reference direction."""

    def __init__(self, p):
        self.p = p
        self.n = p + 1
        self.x, self.w = gauss_legendre(self.n)
        self.D = derivative_matrix(self.x)
        self.lm = lagrange_eval(self.x, -1.0)[0]   # l_j(-1)
        self.lp = lagrange_eval(self.x, +1.0)[0]   # l_j(+1)
        self.dlm = lagrange_derivative_at(self.x, -1.0)   # l_j'(-1)
        self.dlp = lagrange_derivative_at(self.x, +1.0)   # l_j'(+1)
