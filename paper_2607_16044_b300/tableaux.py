"""Explicit Butcher tableaux passed to dgx_set_tableau.

The paper advances the explicit region with the ERK half of an ARS-type
additive Runge-Kutta pair (Sec. 4.2, padded tableau with c_{i+1} = c_i of the
implicit half; Algorithm 1).  The coefficients are those Ascher, Ruuth and
Spiteri (1997) publish for ARS(3,4,3) (ten digits), gamma the root of
6 g^3 - 18 g^2 + 9 g - 1 in (0, 1); b = (0, b2, b3, gamma) with
b2 = -3 g^2/2 + 4 g - 1/4 and b3 = 3 g^2/2 - 5 g + 5/4 (not FSAL).
"""
import numpy as np

GAMMA_ARS343 = 0.4358665215


def ars343_explicit():
    g = GAMMA_ARS343
    A = np.array([[0.0, 0.0, 0.0, 0.0],
                  [g, 0.0, 0.0, 0.0],
                  [0.3212788860, 0.3966543747, 0.0, 0.0],
                  [-0.105858296, 0.5529291479, 0.5529291479, 0.0]])
    b = np.array([0.0, -1.5 * g * g + 4.0 * g - 0.25, 1.5 * g * g - 5.0 * g + 1.25, g])
    c = np.array([0.0, g, 0.5 * (1.0 + g), 1.0])
    return A, b, c


def forward_euler():
    return np.zeros((1, 1)), np.array([1.0]), np.array([0.0])
