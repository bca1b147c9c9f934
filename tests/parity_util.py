"""Shared helpers for the GPU-vs-oracle parity tests."""
import numpy as np
import torch

from oracle.physics import Gas
from oracle.residual import DGOperator, term_scale

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def gas_of(phys):
    return Gas(phys.gamma, Re=phys.Re if phys.viscous else 0.0, Pr=phys.Pr, viscous=phys.viscous)


def rel_err(got, ref):
    """max over fields of ||got - ref||_inf / ||ref||_inf (per field, all nodes)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    errs = []
    for f in range(ref.shape[1]):
        scale = np.abs(ref[:, f]).max()
        if scale == 0:
            scale = 1.0
        errs.append(np.abs(got[:, f] - ref[:, f]).max() / scale)
    return max(errs)


def oracle_rhs(mesh, phys, U, elems=None):
    op = DGOperator(mesh, gas_of(phys))
    return op.residual(torch.as_tensor(np.asarray(U, dtype=np.float64)), elems).numpy()


def quantize32(U):
    return np.asarray(U, dtype=np.float32).astype(np.float64)


def oracle_rhs_and_scale(mesh, phys, U, elems=None):
    op = DGOperator(mesh, gas_of(phys))
    Ut = torch.as_tensor(np.asarray(U, dtype=np.float64))
    f = op.residual(Ut, elems).numpy()
    T = term_scale(op, Ut, elems).numpy()
    return f, T


def scaled_err(got, ref, T):
    """max over fields of ||got - ref||_inf / ||T||_inf, T the term scale of the
    field (see oracle.residual.term_scale): agreement relative to the magnitude
    of what the residual sums, independent of how much those terms cancel."""
    got = np.asarray(got, dtype=np.float64)
    errs = []
    for f in range(ref.shape[1]):
        errs.append(np.abs(got[:, f] - ref[:, f]).max() / max(np.abs(T[:, f]).max(), 1e-300))
    return max(errs)


def record(name, **vals):
    """Append a parity measurement to $DGX_PARITY_LOG (JSON lines) if set."""
    import json
    import os
    path = os.environ.get("DGX_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"case": name, **{k: float(v) for k, v in vals.items()}}) + "\n")


def noise_floor(mesh, phys, U, eps, elems=None, trials=3, seed=0):
    """Sensitivity of the exact operator to rounding its input: the largest
    scaled change of f when U is perturbed by relative eps (uniform, i.i.d.).
    A backward-stable evaluation in a precision with unit roundoff eps lies
    within a small multiple of this of the exact result."""
    rng = np.random.default_rng(seed)
    f0, T = oracle_rhs_and_scale(mesh, phys, U, elems)
    worst = 0.0
    for _ in range(trials):
        Up = U * (1.0 + eps * rng.uniform(-1.0, 1.0, U.shape))
        fp = oracle_rhs(mesh, phys, Up, elems)
        worst = max(worst, scaled_err(fp, f0, T))
    return worst
