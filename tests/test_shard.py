"""Multi-GPU decomposition logic on CPU ranks (gloo, world size 2): the
instance partition of an ensemble, and the element-slab partition whose halo
exchange (point-to-point through torch.distributed) lets each rank evaluate
the residual of its own elements on a local mesh -- the assembled rows equal
the single-mesh residual.  The residual on each rank is the oracle's here (no
GPU); on GPUs the same exchange feeds the library's residual."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2607_16044_b300 import inputs as I
from paper_2607_16044_b300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_balance_instances_covers_and_balances():
    specs = I.ensemble_manifest()
    costs = [(sp["cells"] ** 2) * (sp["p"] + 1) ** 2 * 4 for sp in specs]
    for world in (2, 3, 8):
        parts = shard.balance_instances(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(specs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)       # the greedy bound


def test_slab_owner_is_contiguous_and_even():
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 12), I.uniform_edges(0, 1, 5)], [True, True])
    owner = shard.slab_owner(mesh, 3, axis=0)
    counts = np.bincount(owner)
    assert counts.max() - counts.min() <= 1
    x = mesh.lo[:, 0]
    for r in range(2):                                     # slabs are ordered along x
        assert x[owner == r].max() <= x[owner == r + 1].min()


def _case(name):
    from oracle.physics import Gas
    from oracle.residual import DGOperator
    from oracle.sipg import SIPGOperator
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 8), I.wall_stretched_edges(2, 1.3)], [True, False])
    gas = Gas(1.4, Re=80.0, Pr=0.72, viscous=True)
    op_cls, rings = (DGOperator, 2) if name == "llf-br1" else (SIPGOperator, 1)
    return mesh, gas, op_cls, rings


def _worker(rank, world, port, name, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mesh, gas, op_cls, rings = _case(name)
        U = I.random_state(mesh, 5)
        owner = shard.slab_owner(mesh, world, axis=0)
        halo = shard.build_halo(mesh, owner, rank, rings)
        Ul = torch.zeros((halo.mesh.n_elem,) + U.shape[1:], dtype=torch.float64)
        Ul[:halo.n_owned] = torch.as_tensor(U[halo.glob[:halo.n_owned]])   # ghosts start empty
        halo.exchange(Ul)
        f = op_cls(halo.mesh, gas).residual(Ul)[:halo.n_owned].numpy()
        rows = [None] * world
        dist.all_gather_object(rows, (halo.glob[:halo.n_owned].tolist(), f))
        if rank == 0:
            full = np.zeros_like(U)
            for ids, fr in rows:
                full[ids] = fr
            out["assembled"] = full
            out["ghosts_filled"] = bool(np.allclose(Ul.numpy(), U[halo.glob]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["llf-br1", "dgip"])
def test_slab_halo_residual_matches_single_mesh(name):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, name, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    mesh, gas, op_cls, _ = _case(name)
    U = I.random_state(mesh, 5)
    ref = op_cls(mesh, gas).residual(torch.as_tensor(U)).numpy()
    assert res["ghosts_filled"]
    assert np.abs(res["assembled"] - ref).max() <= 1e-13 * np.abs(ref).max()
