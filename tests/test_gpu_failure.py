"""Failure detection on the GPU without a fault: a bounded device wait that
runs out is reported on the host and leaves the context usable.

The persistent TMA-fed element kernel waits on an mbarrier for each tile's
bulk copies.  With its poll bound set to 0 every CTA gives up at its first
wait, raises the timeout flag, waits (with the normal bound) for its own
copies still in flight and returns; dgx_check reports DGX_ETIMEOUT.  With the
bound restored the next residual is parity-green again."""
import numpy as np
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, oracle_rhs, quantize32, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bounded_wait_timeout_is_reported_and_recoverable(prec):
    from paper_2607_16044_b300.dgx import DGXError, Solver
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 24), I.wall_stretched_edges(8, 1.2)], [True, False])
    phys = I.Physics(gamma=1.4, Re=300.0, Pr=0.72, Ma=0.3, viscous=True)
    s = Solver(mesh, phys, prec)
    s.set_pipeline(True)
    U0 = I.random_state(mesh, 21)
    U = torch.as_tensor(U0).to("cuda", torch.float64 if prec == "fp64" else torch.float32).contiguous()
    s.rhs(U)
    s.check()                                              # clean start
    assert s.lib.dgx_set_wait_limit(s.h, 0) == 0
    s.rhs(U)
    with pytest.raises(DGXError) as ei:
        s.check()
    assert ei.value.code == 5                              # DGX_ETIMEOUT
    s.check()                                              # the flag was cleared
    assert s.lib.dgx_set_wait_limit(s.h, -1) == 0          # default bound again
    f = s.rhs(U).double().cpu().numpy()
    s.check()
    ref = oracle_rhs(mesh, phys, U0 if prec == "fp64" else quantize32(U0))
    assert rel_err(f, ref) < TOL[prec]
