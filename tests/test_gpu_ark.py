"""GPU parity of the fused explicit ARK step (dgx_ark_step) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.residual import DGOperator
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import gas_of, quantize32, rel_err


def increment_err(got, ref, U0, tol):
    """Per field: |got - ref| <= tol * max|ref - U0| + 8 eps * max|U0| (the
    increments are small differences of O(1) states, so the comparison itself
    carries the rounding of U)."""
    ok = True
    worst = 0.0
    for f in range(U0.shape[1]):
        inc = np.abs(ref[:, f] - U0[:, f]).max()
        bound = tol * inc + 8 * 2.2e-16 * np.abs(U0[:, f]).max()
        e = np.abs(got[:, f] - ref[:, f]).max()
        worst = max(worst, e / bound)
    return worst

pytestmark = pytest.mark.gpu


def _steps_gpu(mesh, phys, U0, prec, dt, nsteps, tableau):
    from paper_2607_16044_b300.dgx import Solver
    s = Solver(mesh, phys, prec)
    s.set_tableau(*tableau)
    U = torch.as_tensor(U0).cuda().contiguous()
    for _ in range(nsteps):
        s.ark_step(U, dt)
    s.check()
    return U.cpu().numpy()


def _steps_oracle(mesh, phys, U0, dt, nsteps, tableau):
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = tableau
    U = torch.as_tensor(U0)
    for _ in range(nsteps):
        U = ark.erk_step(op.residual, U, dt, A, b)
    return U.numpy()


@pytest.mark.parametrize("tableau", ["ars343", "forward_euler", "heun2"])
def test_ark_fp64_vortex(tableau):
    mesh, phys, U0 = I.vortex_workload(p=3, cells=8)
    tab = getattr(ark, tableau)()
    got = _steps_gpu(mesh, phys, U0, "fp64", 0.02, 3, tab)
    ref = _steps_oracle(mesh, phys, U0, 0.02, 3, tab)
    err = increment_err(got, ref, U0, 1e-12)
    assert err < 1.0, err


def test_ark_fp64_channel_walls():
    mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.3)], [True, False])
    phys = I.Physics(gamma=1.4, Re=200.0, Pr=0.72, Ma=0.3, viscous=True)
    U0 = I.channel_state(mesh, phys, 3)
    tab = ark.ars343()
    got = _steps_gpu(mesh, phys, U0, "fp64", 1e-5, 2, tab)
    ref = _steps_oracle(mesh, phys, U0, 1e-5, 2, tab)
    assert increment_err(got, ref, U0, 1e-12) < 1.0


def test_ark_fp32_vortex_stage_accumulation_in_fp64():
    """FP32 residuals on rounded stage states, FP64 accumulation into U_n."""
    mesh, phys, U0 = I.vortex_workload(p=3, cells=8)
    tab = ark.ars343()
    got = _steps_gpu(mesh, phys, U0, "fp32", 0.02, 3, tab)
    ref = _steps_oracle(mesh, phys, U0, 0.02, 3, tab)
    assert rel_err(got - U0, ref - U0) < 1e-5
    # the master state keeps more than FP32 precision: U0 + tiny increment survives
    U = U0.copy()
    got = _steps_gpu(mesh, phys, U, "fp32", 1e-9, 1, tab)
    ref = _steps_oracle(mesh, phys, U, 1e-9, 1, tab)
    assert rel_err(got - U0, ref - U0) < 1e-4
