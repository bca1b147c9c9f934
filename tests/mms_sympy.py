"""Symbolic restatement of the compressible Navier-Stokes operator (Sec. 2).

Used only to pin the oracle: sympy differentiates the continuous fluxes of
Sec. 2 (F^c with H = E + p/rho; tau with lambda = -2 mu/3; q = -kappa grad theta,
kappa = c_p mu / Pr) for a manufactured solution, so that the discrete operator
applied to that solution must approach -div(F^c - F^nu) as the mesh is refined.

The manufactured solution is the one of Sec. 5.1.1 (Gassner et al.):
rho = rho u = rho v = s + 4, rho E = (s + 4)^2, s = sin(pi (kx x + ky y) - omega pi t);
the 3D variant adds rho w = s + 4 and kz z.
"""
import functools

import numpy as np
import sympy as sp


@functools.lru_cache(maxsize=None)
def build(dim=2, gamma=1.4, mu=0.01, Pr=0.72, kx=2, ky=2, kz=2, omega=200):
    X = sp.symbols("x y z")[:dim]
    t = sp.Symbol("t")
    k = [kx, ky, kz][:dim]
    s = sp.sin(sp.pi * sum(ki * xi for ki, xi in zip(k, X)) - omega * sp.pi * t)
    rho = s + 4
    mom = [s + 4] * dim
    rE = (s + 4) ** 2
    U = [rho] + mom + [rE]
    u = [m / rho for m in mom]
    p = (gamma - 1) * (rE - sp.Rational(1, 2) * rho * sum(ui * ui for ui in u))
    H = (rE + p) / rho
    Fc = [[rho * u[i]] + [rho * u[i] * u[j] + (p if i == j else 0) for j in range(dim)] + [rho * u[i] * H]
          for i in range(dim)]
    # viscous: kappa grad theta = (gamma mu / Pr) grad e, e = E - |u|^2 / 2
    e = rE / rho - sp.Rational(1, 2) * sum(ui * ui for ui in u)
    lam = -sp.Rational(2, 3) * mu
    div = sum(sp.diff(u[i], X[i]) for i in range(dim))
    tau = [[mu * (sp.diff(u[j], X[i]) + sp.diff(u[i], X[j])) + (lam * div if i == j else 0)
            for j in range(dim)] for i in range(dim)]
    q = [-(gamma * mu / Pr) * sp.diff(e, X[i]) for i in range(dim)]
    Fv = [[0] + [tau[i][j] for j in range(dim)] + [sum(tau[i][j] * u[j] for j in range(dim)) - q[i]]
          for i in range(dim)]
    nf = dim + 2
    divF_c = [sum(sp.diff(Fc[i][f], X[i]) for i in range(dim)) for f in range(nf)]
    divF_v = [sum(sp.diff(Fv[i][f], X[i]) for i in range(dim)) for f in range(nf)]
    Ut = [sp.diff(Uf, t) for Uf in U]
    args = list(X) + [t]
    lamb = lambda exprs: [sp.lambdify(args, ex, "numpy") for ex in exprs]
    return {"U": lamb(U), "divFc": lamb(divF_c), "divFv": lamb(divF_v), "Ut": lamb(Ut)}


def evaluate(fns, xyz, t):
    """xyz[E][d][N] -> array[E][nf][N] for a list of lambdified component functions."""
    coords = [xyz[:, a, :] for a in range(xyz.shape[1])]
    out = []
    for fn in fns:
        v = fn(*coords, t)
        out.append(np.broadcast_to(np.asarray(v, dtype=np.float64), coords[0].shape))
    return np.stack(out, axis=1)
