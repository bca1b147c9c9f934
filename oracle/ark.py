"""Explicit additive-Runge-Kutta stage and solution updates (oracle).

Test infrastructure only.  Follows Sec. 4.2 of the paper (ERK solution and
stage updates, Table of the padded ERK/DIRK tableaux) and Algorithm 1: with
f = -M^{-1} R^DG the explicit part of an (s+1)-stage scheme is

  y_1 = U_n,   y_i = U_n + dt sum_{j<i} a_ij f(y_j),
  U_{n+1} = U_n + dt sum_i b_i f(y_i)      (no FSAL shortcut: ARS is not FSAL).

The paper names the ARS family (Ascher, Ruuth & Spiteri 1997) without
printing coefficients; ``ars343`` is the explicit half of ARS(3,4,3) with the
ten-digit values published there, with b = (0, b2, b3, gamma) and
b2 = -3 gamma^2/2 + 4 gamma - 1/4, b3 = 3 gamma^2/2 - 5 gamma + 5/4.

The adjoint of one step (reverse stage recurrence), for a cotangent lam on
U_{n+1}:   mu_i = dt (b_i lam + sum_{j>i} a_ji nu_j),  nu_i = J(y_i)^T mu_i,
           lam_n = lam + sum_i nu_i,   processed for i = s+1 .. 1.
"""
import numpy as np

ARS343_GAMMA = 0.4358665215


def ars343():
    g = ARS343_GAMMA
    A = np.zeros((4, 4))
    A[1, 0] = g
    A[2, 0] = 0.3212788860
    A[2, 1] = 0.3966543747
    A[3, 0] = -0.105858296
    A[3, 1] = 0.5529291479
    A[3, 2] = 0.5529291479
    b = np.array([0.0, -1.5 * g * g + 4.0 * g - 0.25, 1.5 * g * g - 5.0 * g + 1.25, g])
    c = np.array([0.0, g, 0.5 * (1.0 + g), 1.0])
    return A, b, c


def forward_euler():
    return np.zeros((1, 1)), np.array([1.0]), np.array([0.0])


def heun2():
    """Two-stage second-order explicit RK (for temporal-order checks)."""
    A = np.array([[0.0, 0.0], [1.0, 0.0]])
    return A, np.array([0.5, 0.5]), np.array([0.0, 1.0])


def erk_step(f, U, dt, A, b, return_stages=False, t0=None, c=None):
    """One explicit step.  f(y) -- or f(y, t) with stage times t0 + c_i dt when
    ``t0`` is given (non-autonomous right-hand sides such as a manufactured
    source)."""
    s = len(b)
    ys, ks = [], []
    for i in range(s):
        y = U.clone() if hasattr(U, "clone") else U.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                y = y + dt * A[i, j] * ks[j]
        ys.append(y)
        ks.append(f(y) if t0 is None else f(y, t0 + c[i] * dt))
    Unew = U
    for i in range(s):
        if b[i] != 0.0:
            Unew = Unew + dt * b[i] * ks[i]
    return (Unew, ys, ks) if return_stages else Unew


def erk_adjoint_step(vjp, ys, lam, dt, A, b):
    """lam_n from lam_{n+1}; vjp(y, mu) = J(y)^T mu; ys = stage states of the step."""
    s = len(b)
    nu = [None] * s
    lam_n = lam
    for i in reversed(range(s)):
        mu = dt * b[i] * lam
        for j in range(i + 1, s):
            if A[j, i] != 0.0:
                mu = mu + dt * A[j, i] * nu[j]
        nu[i] = vjp(ys[i], mu)
        lam_n = lam_n + nu[i]
    return lam_n
