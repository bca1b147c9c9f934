"""Derivatives of the oracle residual (test infrastructure only).

* ``vjp``        -- g = (df/dU)^T lam by reverse-mode differentiation of the
                    oracle's own forward code (torch.autograd on float64).
* ``jvp_cs``     -- (df/dU) v by the complex step Im f(U + i h v) / h, h = 1e-30,
                    exact to rounding (no subtractive cancellation).
* ``jacobian_cs``-- dense Jacobian, one complex-step column per degree of freedom
                    (tiny meshes only).

The forward code branches on real parts at |.| and max (see ``physics``), so
both routes differentiate the same piecewise-analytic function.
"""
import torch


def vjp(op, U, lam, elems=None):
    Ut = torch.as_tensor(U, dtype=torch.float64).detach().clone().requires_grad_(True)
    f = op.residual(Ut, elems)
    lt = torch.as_tensor(lam, dtype=torch.float64)
    if elems is not None:
        lt = lt[torch.as_tensor(elems, dtype=torch.long)]
    (g,) = torch.autograd.grad(f, Ut, grad_outputs=lt)
    return g.detach()


def jvp_cs(op, U, v, h=1e-30):
    Uc = torch.as_tensor(U, dtype=torch.float64).to(torch.complex128) \
        + 1j * h * torch.as_tensor(v, dtype=torch.float64).to(torch.complex128)
    return op.residual(Uc).imag / h


def jacobian_cs(op, U, h=1e-30):
    U = torch.as_tensor(U, dtype=torch.float64)
    n = U.numel()
    cols = []
    for k in range(n):
        v = torch.zeros(n, dtype=torch.float64)
        v[k] = 1.0
        cols.append(jvp_cs(op, U, v.reshape(U.shape), h).reshape(-1))
    return torch.stack(cols, 1)


def vjp_rows(op, U, lam, rows):
    """Rows of g = (df/dU)^T lam for a few elements without a full-mesh pass.

    g_e collects lam_k (df_k/dU_e) over the elements k whose residual depends
    on U_e: the 1-ring (Euler) or 2-ring (BR1) of e.  Those residuals are
    evaluated on their own rings by ``DGOperator.residual(.., elems)``.
    """
    R = torch.as_tensor(rows, dtype=torch.long)
    K = op.ring(R)
    if op.gas.viscous:
        K = op.ring(K)
    Ut = torch.as_tensor(U, dtype=torch.float64).detach().clone().requires_grad_(True)
    f = op.residual(Ut, K)
    lt = torch.as_tensor(lam, dtype=torch.float64)[K]
    (g,) = torch.autograd.grad(f, Ut, grad_outputs=lt)
    return g[R].detach()
