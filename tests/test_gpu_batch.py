"""Batched ensemble (A12): grouped, concatenated instances, per-instance dt,
CUDA-graph step and tile autotuning -- checked against the single-instance path
(and, for one instance, against the oracle)."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.residual import DGOperator
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import gas_of, record, rel_err

pytestmark = pytest.mark.gpu


def _instances():
    specs = [{"cells": 6, "p": 2, "viscous": False}, {"cells": 5, "p": 3, "viscous": True},
             {"cells": 9, "p": 2, "viscous": False}, {"cells": 4, "p": 4, "viscous": True},
             {"cells": 7, "p": 3, "viscous": True}, {"cells": 3, "p": 5, "viscous": False}]
    out = []
    for k, sp in enumerate(specs):
        sp = dict(sp, dt=0.002 * (1 + k % 3))
        mesh, phys, U = I.ensemble_instance(sp)
        out.append((sp, mesh, phys, U))
    return out


def _solvers(insts, prec):
    from paper_2607_16044_b300.dgx import Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    sol = []
    for sp, mesh, phys, U in insts:
        s = Solver(mesh, phys, prec)
        s.set_tableau(*ars343_explicit())
        sol.append(s)
    return sol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single_instances(prec):
    from paper_2607_16044_b300.dgx import Batch
    insts = _instances()
    sol = _solvers(insts, prec)
    dts = [sp["dt"] for sp, *_ in insts]
    batch = Batch(sol, dts)
    assert batch.groups == 4           # distinct (p, physics) pairs among the six instances
    U = batch.pack([U0 for *_, U0 in insts])
    for _ in range(2):
        batch.step(U)
    refs = []
    for s, (sp, mesh, phys, U0), dt in zip(sol, insts, dts):
        Ui = torch.as_tensor(U0).cuda()
        for _ in range(2):
            s.ark_step(Ui, dt)
        refs.append(Ui)
    torch.cuda.synchronize()
    for got, ref in zip(batch.unpack(U), refs):
        assert torch.equal(got, ref)   # identical per-element arithmetic
    # graph replay continues bit-identically from the same state
    Ug, Ue = U.clone(), U.clone()
    for _ in range(3):
        batch.step(Ug, graph=True)
        batch.step(Ue)
    torch.cuda.synchronize()
    assert torch.equal(Ug, Ue)


def test_batch_instance_matches_oracle():
    from paper_2607_16044_b300.dgx import Batch
    insts = _instances()
    sol = _solvers(insts, "fp64")
    dts = [sp["dt"] for sp, *_ in insts]
    batch = Batch(sol, dts)
    U = batch.pack([U0 for *_, U0 in insts])
    batch.step(U)
    k = 3                               # the p = 4 NS instance
    sp, mesh, phys, U0 = insts[k]
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    ref = ark.erk_step(op.residual, torch.as_tensor(U0), dts[k], A, b).numpy()
    got = batch.unpack(U)[k].cpu().numpy()
    assert rel_err(got - U0, ref - U0) < 1e-11


def test_autotune_keeps_results():
    from paper_2607_16044_b300.dgx import Batch
    from paper_2607_16044_b300.tableaux import ars343_explicit
    insts = _instances()
    sol = _solvers(insts, "fp32")
    dts = [sp["dt"] for sp, *_ in insts]
    batch = Batch(sol, dts)
    U0 = batch.pack([U0 for *_, U0 in insts])
    U1 = U0.clone()
    batch.step(U1)
    batch.autotune(U0, reps=2)
    U2 = U0.clone()
    batch.step(U2)
    torch.cuda.synchronize()
    assert torch.equal(U1, U2)
    # single handle: every chosen variant is valid and results are unchanged
    mesh, phys, Uc = I.channel2d_workload(p=3, nx=32, n_half=8)
    from paper_2607_16044_b300.dgx import Solver
    s = Solver(mesh, phys, "fp32")
    s.set_tableau(*ars343_explicit())
    Ua = torch.as_tensor(Uc).cuda()
    f0 = s.rhs(Ua.float())
    v = s.autotune(Ua, reps=2)
    assert all(x in (0, 1, 2, 3) for x in v.values())
    f1 = s.rhs(Ua.float())
    assert torch.equal(f0, f1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_batch_bit_identical_to_groups(prec):
    """The persistent form (one launch per phase over every group's tiles)
    runs the groups' own tile arithmetic: identical states after eager and
    graph-replayed steps."""
    from paper_2607_16044_b300.dgx import Batch
    insts = _instances()
    dts = [sp["dt"] for sp, *_ in insts]
    states = [U0 for *_, U0 in insts]
    out = []
    for persistent in (False, True):
        b = Batch(_solvers(insts, prec), dts)
        b.set_persistent(persistent)
        U = b.pack(states)
        for _ in range(2):
            b.step(U)
        Ug = U.clone()
        for _ in range(2):
            b.step(Ug, graph=True)
        torch.cuda.synchronize()
        out.append((U, Ug))
    if prec == "fp64":
        assert torch.equal(out[0][0], out[1][0])
        assert torch.equal(out[0][1], out[1][1])
    else:
        # FP32: the same source inlined into another kernel may contract a
        # multiply-add differently, so the states agree to FP32 rounding
        for a, b in ((out[0][0], out[1][0]), (out[0][1], out[1][1])):
            dev = float(((a - b).abs().max() / a.abs().max()).item())
            record("persistent-batch-fp32-dev", rel=dev)
            assert dev < 1e-6, dev


def test_persistent_batch_ensemble_manifest():
    """The 64-instance seeded ensemble (8 groups): persistent form against the
    grouped form, one graph-replayed FP32 step."""
    from paper_2607_16044_b300.dgx import Batch, Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    specs = I.ensemble_manifest()
    res = []
    for persistent in (False, True):
        sol, states = [], []
        for sp in specs:
            mesh, phys, U0 = I.ensemble_instance(sp)
            so = Solver(mesh, phys, "fp32")
            so.set_tableau(*ars343_explicit())
            sol.append(so)
            states.append(U0)
        b = Batch(sol, [sp["dt"] for sp in specs])
        b.set_persistent(persistent)
        U = b.pack(states)
        b.step(U, graph=True)
        torch.cuda.synchronize()
        res.append(U)
    dev = float(((res[0] - res[1]).abs().max() / res[0].abs().max()).item())
    record("persistent-ensemble-fp32-dev", rel=dev)
    assert dev < 1e-6, dev
