"""One scene split by rows over several processes (one GPU each).

Only the product ``A v`` couples nodes (Sec. III.F): W, the surrogate step of
eq. (pgd1) and the one-shot contact solve of Alg. 2 are local to a row or a
contact's node(s).  So a scene splits into shards of contiguous node ranges --
on the lattices here, slabs of z-layers -- and one V-FPI sweep of the whole
scene is

1. every shard sweeps its own rows (``vfpi_shard_sweep``), reading the latest
   v of its halo: the other shards' nodes that its rows reference;
2. a D-contact whose nodes lie on two shards (a split contact) is held by
   both: each sends the other the v* of its endpoint, and both take the
   contact's step from the same inputs (``vfpi_finish_split``), each keeping
   its own endpoint's update; the contact belongs to (its lambda is reported
   by) the shard of its lower-numbered node;
3. theta^2 of Alg. 1 is the sum of the shards' FP64 sums of squares, added in
   rank order on every rank (all take the same stop decision);
4. unless the stop test ends the solve, each shard sends the rows its
   neighbours need and sets the rows it receives as its halo.

Before the first sweep the shards of each split contact also exchange the row
statistics the tied Frobenius W of its two nodes is formed from (Sec. IV.C).
After every sweep that goes on, each shard is given the scene's theta
(``vfpi_shard_set_theta``): with Alg. 3 (shards made with ``chebyshev_ls``)
the next sweep's weight comes from it.  This module is the host side only: the
partition, the halo, send and split lists, the exchange over
``torch.distributed`` (NCCL between GPUs, gloo on CPUs) or inside one process,
and the loop; every step of the sweep runs in the library's kernels.
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
    g -> g - n0, halo node halo[k] -> (n1 - n0) + k.  The halo is first the
    other shards' nodes that this shard's rows reference (sorted; exchanged
    every sweep), then the other endpoints of split contacts that no row
    references (sorted; only their v* is exchanged)."""
    rank: int
    ranges: list
    n0: int
    n1: int
    halo: np.ndarray                 # global ids
    n_halo_rows: int                 # the first part of the halo: referenced by rows
    row_ptr: np.ndarray              # [n_own + 1]
    col_idx: np.ndarray              # local numbering, the scene's column order
    blocks: slice                    # this shard's blocks in the scene's vals
    contacts: np.ndarray             # indices of this shard's contacts in the scene's list
    node_i: np.ndarray               # local
    node_j: np.ndarray               # local, -1 for S-contacts
    recv: dict                       # peer -> (first halo index, count)
    send: dict                       # peer -> local own ids the peer needs, in its halo order
    split: np.ndarray                # positions in ``contacts`` of the split contacts
    split_peer: dict                 # peer -> positions in ``split`` of the contacts shared with it
    owns: np.ndarray                 # [len(contacts)] this shard reports the contact's lambda

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
    inside = lambda g: (g >= n0) & (g < n1)                        # noqa: E731
    halo_rows = halo_of(row_ptr, col_idx, n0, n1)
    cols = col_idx[row_ptr[n0]:row_ptr[n1]]
    own = (cols >= n0) & (cols < n1)
    # this shard's contacts: every contact with a node here, in the scene's order
    contacts = np.nonzero(inside(node_i) | inside(node_j))[0]
    ci, cj = node_i[contacts], node_j[contacts]
    is_split = (cj >= 0) & (inside(ci) != inside(cj))
    other = np.where(inside(ci), cj, ci)[is_split]
    extra = np.setdiff1d(other, halo_rows)
    halo = np.concatenate([halo_rows, extra]).astype(np.int64)

    def local_of(g):
        """own g -> g - n0, halo g -> n_own + its halo position, -1 -> -1"""
        g = np.asarray(g, dtype=np.int64)
        if len(halo_rows):
            k = np.minimum(np.searchsorted(halo_rows, g), len(halo_rows) - 1)
            in_rows = halo_rows[k] == g
        else:
            k, in_rows = np.zeros(g.shape, np.int64), np.zeros(g.shape, bool)
        hpos = np.where(in_rows, k, len(halo_rows) + np.searchsorted(extra, g))
        out = np.where(inside(g), g - n0, (n1 - n0) + hpos)
        return np.where(g < 0, -1, out).astype(np.int32)

    local = np.where(own, cols - n0, (n1 - n0) + np.searchsorted(halo_rows, cols))
    split = np.nonzero(is_split)[0]
    split_peer = {}
    if len(split):
        peer_of = owner_of(ranges, other)
        for p in np.unique(peer_of):
            split_peer[int(p)] = np.nonzero(peer_of == p)[0]
    # the contact belongs to the shard of its lower-numbered node
    low = np.where(cj >= 0, np.minimum(ci, cj), ci)
    owns = inside(low)
    recv = {}
    if len(halo_rows):
        own_of = owner_of(ranges, halo_rows)
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
                     n_halo_rows=len(halo_rows),
                     row_ptr=(row_ptr[n0:n1 + 1] - row_ptr[n0]).astype(np.int32),
                     col_idx=local.astype(np.int32), blocks=slice(int(row_ptr[n0]), int(row_ptr[n1])),
                     contacts=contacts, node_i=local_of(ci), node_j=local_of(cj), recv=recv,
                     send=send, split=split, split_peer=split_peer, owns=owns)


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
        for p, t in sends.items():     # (fresh tensors: the sender keeps no reference)
            self.box[(src, p)] = t

    def take(self, dst: int, recv_shapes: dict):
        return {p: self.box.pop((p, dst)) for p in recv_shapes}


# ----------------------------------------------------------------------------
# the sharded loop (Alg. 1 over shards)
# ----------------------------------------------------------------------------

def _sends(engine, plan, torch, dtype, device):
    out = {}
    for p, ids in plan.send.items():   # (host lists: checked on the host, no wait for the GPU)
        t = torch.empty(3 * len(ids), dtype=dtype, device=device)
        engine.get_nodes(ids, out=t)
        out[p] = t
    return out


def _set_halo(engine, plan, got):
    for p, (first, n) in plan.recv.items():
        engine.set_halo(first, got[p])


def _split_sends(plan, vals, width):
    """Per peer: the rows (``width`` values each) of ``vals`` that belong to
    the split contacts shared with it, in the split order."""
    import torch
    v = vals.view(-1, width)
    return {p: v[torch.as_tensor(idx, device=v.device)].reshape(-1).contiguous()
            for p, idx in plan.split_peer.items()}


def _split_assemble(plan, got, width, like):
    """The other endpoints' rows received from each peer, in the split order."""
    import torch
    out = torch.empty_like(like)
    o = out.view(-1, width)
    for p, idx in plan.split_peer.items():
        o[torch.as_tensor(idx, device=o.device)] = got[p].view(-1, width)
    return out


def _split_shapes(plan, width):
    return {p: width * len(idx) for p, idx in plan.split_peer.items()}


def _theta(s2: float, n_dof: int, norm: str) -> float:
    """theta of Alg. 1 as the kernels form it (sqrt, times 1 / sqrt(n))."""
    th = math.sqrt(s2)
    return th * (1.0 / math.sqrt(n_dof)) if norm == "rms" else th


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
    n_split = len(plan.split)
    if n_split:    # the tied W of each split contact's two nodes
        st = engine.split_stats(out=torch.empty(6 * n_split, dtype=torch.float64, device=device))
        got = comm.exchange(_split_sends(plan, st, 6), _split_shapes(plan, 6), torch.float64)
        engine.set_split_stats(_split_assemble(plan, got, 6, st))
    _set_halo(engine, plan, comm.exchange(_sends(engine, plan, torch, dtype, device),
                                          recv_shapes, dtype))

    empty = torch.empty(0, dtype=dtype, device=device)

    def sweep():
        if not n_split:
            # the next sweep's halo rows go out behind this sweep on the stream,
            # before its sum is waited for (an exchange after the last sweep is
            # harmless: it writes halo rows only)
            engine.shard_sweep(sumsq=False)
            _set_halo(engine, plan, comm.exchange(_sends(engine, plan, torch, dtype, device),
                                                  recv_shapes, dtype))
            return engine.finish_split(empty)
        engine.shard_sweep(sumsq=False)
        vs = engine.split_vstar(out=torch.empty(3 * n_split, dtype=dtype, device=device))
        got = comm.exchange(_split_sends(plan, vs, 3), _split_shapes(plan, 3), dtype)
        return engine.finish_split(_split_assemble(plan, got, 3, vs))

    status = NOT_CONVERGED
    theta = float("nan")
    for l in range(1, l_max + 1):
        s2 = comm.sum_in_rank_order(sweep())
        theta = _theta(s2, n_dof, norm)
        if not math.isfinite(theta):
            raise vfpi.VfpiError(vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"], "non-finite residual")
        if theta < theta_th:
            status = vfpi.VFPI_OK
            break
        if l == l_max:
            break
        engine.shard_set_theta(theta)
        if n_split:   # (split contacts finish their rows after the v* exchange)
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

    def split_exchange(vals, width):
        for pl, x in zip(plans, vals):
            if len(pl.split):
                box.post(pl.rank, _split_sends(pl, x, width))
        return [_split_assemble(pl, box.take(pl.rank, pl.split_peer), width, x)
                if len(pl.split) else None for pl, x in zip(plans, vals)]

    split = any(len(pl.split) for pl in plans)
    for e, pl in zip(engines, plans):
        e.set_velocity(v0[3 * pl.n0:3 * pl.n1])
    if split:
        st = [e.split_stats(out=torch.empty(6 * len(pl.split), dtype=torch.float64, device=device))
              for e, pl in zip(engines, plans)]
        for e, x in zip(engines, split_exchange(st, 6)):
            if x is not None:
                e.set_split_stats(x)
    exchange()
    status = NOT_CONVERGED
    theta = float("nan")
    empty = torch.empty(0, dtype=dtype, device=device)
    for l in range(1, l_max + 1):
        # every shard's sweep launched before any sum is waited for
        for e in engines:
            e.shard_sweep(sumsq=False)
        if split:
            vs = [e.split_vstar(out=torch.empty(3 * len(pl.split), dtype=dtype, device=device))
                  for e, pl in zip(engines, plans)]
            parts = [e.finish_split(x if x is not None else empty)
                     for e, x in zip(engines, split_exchange(vs, 3))]
        else:
            exchange()     # queued behind the sweeps, before their sums are waited for
            parts = [e.finish_split(empty) for e in engines]
        s2 = 0.0
        for x in parts:
            s2 += x
        theta = _theta(s2, n_dof, norm)
        if not math.isfinite(theta):
            raise vfpi.VfpiError(vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"], "non-finite residual")
        if theta < theta_th:
            status = vfpi.VFPI_OK
            break
        if l == l_max:
            break
        for e in engines:
            e.shard_set_theta(theta)
        if split:
            exchange()
    v = np.concatenate([np.asarray(e.get_velocity()) for e in engines])
    return ShardResult(v, l, theta, status)
