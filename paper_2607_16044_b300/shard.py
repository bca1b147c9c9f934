"""Multi-GPU decomposition of the explicit DG operator (host logic).

Two ways to spread the work over ranks (one process per GPU):

* an ensemble by instance (``balance_instances``): each rank advances its own
  instances, no data exchange during a step; the partition balances the
  ranks' DOF counts (longest-processing-time greedy);
* one mesh by element slabs (``slab_owner``, ``build_halo``, ``Halo.exchange``):
  each rank owns a contiguous slab of elements along one axis and holds a
  halo of ghost elements around it; before each residual the ghost states are
  received from the ranks that own them (point-to-point send/recv through
  ``torch.distributed``: NCCL between GPUs, gloo on CPUs).  The residual of an
  owned element depends on its neighbours' traces (LLF, and DG-IP, whose
  face gradients are each element's own) or on their BR1 gradients too, so
  the halo is one ring of elements for Euler and DG-IP and two for BR1; the
  local mesh is the owned elements plus the halo, and faces leading out of
  it are closed on the element itself (only ghosts have them, and ghost
  residuals are discarded).

Nothing here computes any of the method's arithmetic: the residual itself is
the library's, on the local mesh.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence

import numpy as np


def balance_instances(costs: Sequence[float], world: int) -> List[List[int]]:
    """Instances (by index) per rank, balancing the summed cost (e.g. DOFs):
    largest first, each to the currently lightest rank."""
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def slab_owner(mesh, world: int, axis: int = 0) -> np.ndarray:
    """Owner rank of every element: contiguous slabs of equal element counts
    along ``axis`` (by the element's lower corner / first node coordinate)."""
    key = mesh.lo[:, axis] if mesh.lo is not None else mesh.xyz[:, axis, :].min(1)
    order = np.lexsort((np.arange(mesh.n_elem), key))
    owner = np.empty(mesh.n_elem, dtype=np.int64)
    for r, chunk in enumerate(np.array_split(order, world)):
        owner[chunk] = r
    return owner


@dataclasses.dataclass
class Halo:
    rank: int
    mesh: object                 # local mesh: owned elements, then ghosts
    glob: np.ndarray             # global id of every local element
    n_owned: int                 # the first n_owned local elements are owned
    send: Dict[int, np.ndarray]  # peer -> local ids of owned elements the peer needs
    recv: Dict[int, np.ndarray]  # peer -> local ids of ghosts the peer owns

    def exchange(self, U_local, group=None):
        """Fill the ghost rows of U_local ([E_local][nf][N], any torch device)
        with the owners' current states (point-to-point, deadlock free: every
        rank posts all sends and receives, then waits)."""
        import torch
        import torch.distributed as dist
        reqs, bufs = [], []
        for peer, idx in sorted(self.recv.items()):
            buf = torch.empty((len(idx),) + tuple(U_local.shape[1:]), dtype=U_local.dtype, device=U_local.device)
            bufs.append((idx, buf))
            reqs.append(dist.irecv(buf, src=peer, group=group))
        for peer, idx in sorted(self.send.items()):
            out = U_local[torch.as_tensor(idx, device=U_local.device)].contiguous()
            reqs.append(dist.isend(out, dst=peer, group=group))
        for r in reqs:
            r.wait()
        for idx, buf in bufs:
            U_local[torch.as_tensor(idx, device=U_local.device)] = buf
        return U_local


def _ring(mesh, elems: np.ndarray, rings: int) -> np.ndarray:
    keep = np.unique(elems)
    for _ in range(rings):
        nb = mesh.neighbor[keep].reshape(-1)
        keep = np.unique(np.concatenate([keep, nb[nb >= 0]]))
    return keep


def local_mesh(mesh, order: np.ndarray):
    """The elements ``order`` (global ids) as a mesh of their own; neighbours
    outside the set are replaced by the element itself across the opposite
    local face (a closed, valid connectivity)."""
    pos = np.full(mesh.n_elem, -1, dtype=np.int64)
    pos[order] = np.arange(len(order))
    nb = mesh.neighbor[order].astype(np.int64)
    inside = nb >= 0
    mapped = np.where(inside, pos[np.where(inside, nb, 0)], nb)
    outside = inside & (mapped < 0)
    self_ids = np.repeat(np.arange(len(order))[:, None], nb.shape[1], axis=1)
    faces = np.tile(np.arange(nb.shape[1]), (len(order), 1))
    nbf = np.where(outside, faces ^ 1, mesh.nbr_face[order])
    ori = np.where(outside, 0, mesh.orient[order])
    mapped = np.where(outside, self_ids, mapped)
    return dataclasses.replace(
        mesh, n_elem=len(order), xyz=mesh.xyz[order], neighbor=mapped.astype(np.int32),
        nbr_face=nbf.astype(np.int8), orient=ori.astype(np.int8),
        lo=None if mesh.lo is None else mesh.lo[order], size=None if mesh.size is None else mesh.size[order],
        shape=None)


def build_halo(mesh, owner: np.ndarray, rank: int, rings: int) -> Halo:
    """Local mesh and exchange lists of ``rank`` for a halo of ``rings``
    element rings (1: Euler / DG-IP, 2: BR1)."""
    owned = np.nonzero(owner == rank)[0]
    keep = _ring(mesh, owned, rings)
    ghosts = np.setdiff1d(keep, owned)
    order = np.concatenate([owned, ghosts])
    loc = local_mesh(mesh, order)
    recv: Dict[int, np.ndarray] = {}
    for peer in np.unique(owner[ghosts]):
        recv[int(peer)] = len(owned) + np.nonzero(owner[ghosts] == peer)[0]
    send: Dict[int, np.ndarray] = {}
    pos = np.full(mesh.n_elem, -1, dtype=np.int64)
    pos[owned] = np.arange(len(owned))
    for peer in np.unique(owner):
        peer = int(peer)
        if peer == rank:
            continue
        theirs = _ring(mesh, np.nonzero(owner == peer)[0], rings)
        need = np.intersect1d(theirs, owned)          # global ids, ascending = the peer's ghost order
        if len(need):
            send[peer] = pos[need]
    return Halo(rank, loc, order, len(owned), send, recv)
