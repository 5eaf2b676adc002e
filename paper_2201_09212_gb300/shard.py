"""One scene split by rows over several processes (one GPU each).

Only the product ``A v`` couples nodes (Sec. III.F): W, the surrogate step of
eq. (pgd1) and the one-shot contact solve of Alg. 2 are local to a row or a
contact's node(s).  So a scene splits into shards of contiguous node ranges --
on the lattices here, slabs of z-layers -- and one V-FPI sweep of the whole
scene is

1. every shard sweeps its own rows (``vfpi_shard_sweep``), reading the latest
   v of its halo: the other shards' nodes that its rows reference;
2. theta^2 of Alg. 1 is the sum of the shards' FP64 sums of squares, added in
   rank order on every rank (all take the same stop decision);
3. unless the stop test ends the solve, each shard sends the rows its
   neighbours need and sets the rows it receives as its halo.

Contacts must join nodes of one shard (an S-contact always does).  The solve
is plain Alg. 1 (the Chebyshev weights of Alg. 3 are not carried across the
per-sweep launches).  This module is the host side only: the partition, the
halo and send lists, the exchange over ``torch.distributed`` (NCCL between
GPUs, gloo on CPUs) or inside one process, and the loop; every step of the
sweep runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import vfpi

NOT_CONVERGED = vfpi.VFPI_NOT_CONVERGED


def partition(row_ptr, n_shards: int, align: int = 1) -> list[tuple[int, int]]:
    """Contiguous node ranges [n0, n1) with about the same number of blocks
    each (the sweep's work is its blocks), cut only at multiples of ``align``
    nodes (a lattice's layer ``nx * ny``: the shards are then z-slabs, and a
    27-point stencil's halo is one layer on each side)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = len(row_ptr) - 1
    if align < 1 or N % align:
        raise ValueError("align must divide n_nodes")
    units = N // align
    if not 1 <= n_shards <= units:
        raise ValueError("need 1 <= n_shards <= n_nodes / align")
    cuts = [0]
    for k in range(1, n_shards):
        c = int(np.searchsorted(row_ptr, row_ptr[-1] * k / n_shards))
        u = int(round(c / align))
        u = min(max(u, cuts[-1] // align + 1), units - (n_shards - k))
        cuts.append(u * align)
    cuts.append(N)
    return [(cuts[k], cuts[k + 1]) for k in range(n_shards)]


def halo_of(row_ptr, col_idx, n0: int, n1: int) -> np.ndarray:
    """Sorted global ids of the nodes outside [n0, n1) that rows n0..n1-1 reference."""
    cols = np.asarray(col_idx[row_ptr[n0]:row_ptr[n1]])
    return np.unique(cols[(cols < n0) | (cols >= n1)]).astype(np.int64)


@dataclasses.dataclass
class ShardPlan:
    """Everything one shard needs, in the shard's own numbering: own node
    g -> g - n0, halo node halo[k] -> (n1 - n0) + k."""
    rank: int
    ranges: list
    n0: int
    n1: int
    halo: np.ndarray                 # global ids, sorted
    row_ptr: np.ndarray              # [n_own + 1]
    col_idx: np.ndarray              # local numbering, the scene's column order
    blocks: slice                    # this shard's blocks in the scene's vals
    contacts: np.ndarray             # indices of this shard's contacts in the scene's list
    node_i: np.ndarray               # local
    node_j: np.ndarray               # local, -1 for S-contacts
    recv: dict                       # peer -> (first halo index, count)
    send: dict                       # peer -> local own ids the peer needs, in its halo order

    @property
    def n_own(self) -> int:
        return self.n1 - self.n0


def owner_of(ranges, g: np.ndarray) -> np.ndarray:
    starts = np.array([r[0] for r in ranges])
    return np.searchsorted(starts, g, side="right") - 1


def make_plan(row_ptr, col_idx, node_i, node_j, ranges, rank: int) -> ShardPlan:
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    node_i = np.asarray(node_i, dtype=np.int64)
    node_j = (np.full(len(node_i), -1, dtype=np.int64) if node_j is None
              else np.asarray(node_j, dtype=np.int64))
    n0, n1 = ranges[rank]
    halo = halo_of(row_ptr, col_idx, n0, n1)
    cols = col_idx[row_ptr[n0]:row_ptr[n1]]
    own = (cols >= n0) & (cols < n1)
    local = np.where(own, cols - n0, (n1 - n0) + np.searchsorted(halo, cols))
    mine = (node_i >= n0) & (node_i < n1)
    jm = node_j[mine]
    if ((jm >= 0) & ((jm < n0) | (jm >= n1))).any():
        raise ValueError("a contact joins nodes of two shards")
    if ((node_j >= n0) & (node_j < n1) & ~mine).any():
        raise ValueError("a contact joins nodes of two shards")
    recv = {}
    if len(halo):
        own_of = owner_of(ranges, halo)
        for p in np.unique(own_of):
            idx = np.nonzero(own_of == p)[0]
            recv[int(p)] = (int(idx[0]), int(len(idx)))
    send = {}
    for p, (a, b) in enumerate(ranges):
        if p == rank:
            continue
        h = halo_of(row_ptr, col_idx, a, b)
        need = h[(h >= n0) & (h < n1)]
        if len(need):
            send[p] = (need - n0).astype(np.int32)
    return ShardPlan(rank=rank, ranges=list(ranges), n0=n0, n1=n1, halo=halo,
                     row_ptr=(row_ptr[n0:n1 + 1] - row_ptr[n0]).astype(np.int32),
                     col_idx=local.astype(np.int32), blocks=slice(int(row_ptr[n0]), int(row_ptr[n1])),
                     contacts=np.nonzero(mine)[0], node_i=(node_i[mine] - n0).astype(np.int32),
                     node_j=np.where(jm >= 0, jm - n0, -1).astype(np.int32), recv=recv, send=send)


def shard_solver(scene, plan: ShardPlan, **kw) -> "vfpi.Solver":
    """The library context of one shard of ``scene`` (keyword arguments as for
    vfpi.Solver; theta_th and l_max there are unused by the sharded loop)."""
    c = plan.contacts
    return vfpi.Solver(plan.row_ptr, plan.col_idx, scene.vals[plan.blocks],
                       scene.b[3 * plan.n0:3 * plan.n1], plan.node_i, plan.node_j,
                       scene.R[c], scene.mu[c], scene.phi[c], h=scene.h,
                       n_halo=len(plan.halo), **kw)


# ----------------------------------------------------------------------------
# communication
# ----------------------------------------------------------------------------

class TorchComm:
    """Exchange through torch.distributed: point-to-point sends and receives of
    the boundary rows (NCCL on GPUs, gloo on CPUs) and an all-gather of the
    shards' sums of squares, added in rank order."""

    def __init__(self, dist, device):
        self.dist = dist
        self.device = device
        self.world = dist.get_world_size()

    def exchange(self, sends: dict, recv_shapes: dict, dtype):
        import torch
        ops, out = [], {}
        for p, n in recv_shapes.items():
            out[p] = torch.empty(n, dtype=dtype, device=self.device)
            ops.append(self.dist.P2POp(self.dist.irecv, out[p], p))
        for p, t in sends.items():
            ops.append(self.dist.P2POp(self.dist.isend, t, p))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        return out

    def sum_in_rank_order(self, x: float) -> float:
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t)
        tot = 0.0
        for q in parts:
            tot += float(q.item())
        return tot


class LocalComms:
    """All shards in one process (one GPU): a mailbox.  Each shard posts the
    rows it sends, then takes the rows addressed to it; the sweep loop runs the
    shards in lock step (see ``solve_local``)."""

    def __init__(self, world: int):
        self.world = world
        self.box = {}

    def post(self, src: int, sends: dict):
        for p, t in sends.items():
            self.box[(src, p)] = t.clone()

    def take(self, dst: int, recv_shapes: dict):
        return {p: self.box.pop((p, dst)) for p in recv_shapes}


# ----------------------------------------------------------------------------
# the sharded loop (Alg. 1 over shards)
# ----------------------------------------------------------------------------

def _sends(engine, plan, torch, dtype, device):
    out = {}
    for p, ids in plan.send.items():
        t = torch.empty(3 * len(ids), dtype=dtype, device=device)
        engine.get_nodes(ids, out=t)
        out[p] = t
    return out


def _set_halo(engine, plan, got):
    for p, (first, n) in plan.recv.items():
        engine.set_halo(first, got[p])


def _theta(s2: float, n_dof: int, norm: str) -> float:
    th = math.sqrt(s2)
    return th / math.sqrt(n_dof) if norm == "rms" else th


@dataclasses.dataclass
class ShardResult:
    v: object            # this shard's own rows (or every shard's, for solve_local)
    iters: int
    theta: float
    status: int


def solve(engine, plan: ShardPlan, comm: TorchComm, v0_own, *, n_dof: int, theta_th: float,
          l_max: int, norm: str = "abs", dtype=None, device=None) -> ShardResult:
    """Alg. 1 on one shard of a scene split over the ranks of ``comm``:
    ``engine`` is this shard's context (vfpi.Solver made with n_halo), ``n_dof``
    the whole scene's DOF count (for the rms norm).  Every rank calls it."""
    import torch
    dtype = dtype or torch.float32
    engine.set_velocity(v0_own)
    recv_shapes = {p: 3 * n for p, (_, n) in plan.recv.items()}
    _set_halo(engine, plan, comm.exchange(_sends(engine, plan, torch, dtype, device),
                                          recv_shapes, dtype))
    status = NOT_CONVERGED
    theta = float("nan")
    for l in range(1, l_max + 1):
        s2 = comm.sum_in_rank_order(engine.shard_sweep())
        theta = _theta(s2, n_dof, norm)
        if not math.isfinite(theta):
            raise vfpi.VfpiError(vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"], "non-finite residual")
        if theta < theta_th:
            status = vfpi.VFPI_OK
            break
        if l == l_max:
            break
        _set_halo(engine, plan, comm.exchange(_sends(engine, plan, torch, dtype, device),
                                              recv_shapes, dtype))
    return ShardResult(engine.get_velocity(), l, theta, status)


def solve_local(engines, plans, v0, *, n_dof: int, theta_th: float, l_max: int,
                norm: str = "abs", dtype=None, device=None) -> ShardResult:
    """The same loop with every shard in this process (one GPU): the shards
    sweep in turn, their sums are added in rank order, and the rows go through
    a mailbox.  ``v0`` is the whole scene's warm start; returns the whole v."""
    import torch
    dtype = dtype or torch.float32
    box = LocalComms(len(plans))

    def exchange():
        for e, pl in zip(engines, plans):
            box.post(pl.rank, _sends(e, pl, torch, dtype, device))
        for e, pl in zip(engines, plans):
            _set_halo(e, pl, box.take(pl.rank, pl.recv))

    for e, pl in zip(engines, plans):
        e.set_velocity(v0[3 * pl.n0:3 * pl.n1])
    exchange()
    status = NOT_CONVERGED
    theta = float("nan")
    for l in range(1, l_max + 1):
        s2 = 0.0
        for e in engines:
            s2 += e.shard_sweep()
        theta = _theta(s2, n_dof, norm)
        if not math.isfinite(theta):
            raise vfpi.VfpiError(vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"], "non-finite residual")
        if theta < theta_th:
            status = vfpi.VFPI_OK
            break
        if l == l_max:
            break
        exchange()
    v = np.concatenate([np.asarray(e.get_velocity()) for e in engines])
    return ShardResult(v, l, theta, status)
