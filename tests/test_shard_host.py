"""Host logic of the sharded scene (paper_2201_09212_gb300/shard.py) on the CPU:
the row partition, the halo and send lists, and the sweep loop with its
exchange and theta assembly, run over gloo ranks (world size 2 and 3) and in
one process.  The sweep itself is played by a stand-in engine that runs the
FP64 oracle's sweep (Alg. 1 + Alg. 2) on the whole scene's vector assembled
from the shard's own rows and halo: a shard's rows read only own and halo
columns, so its rows of that sweep are exactly the unsplit sweep's rows.  The
sharded solve must therefore reproduce the unsplit oracle solve bit for bit
(theta, summed per shard and then over shards, to rounding)."""
import math
import os
import socket

import numpy as np
import pytest
import torch

from oracle import vfpi as ov
from paper_2201_09212_gb300 import scenes, shard
from tests.conftest import oracle_problem

THETA = 1e-9
L_MAX = 400


def scene():
    # 12 x 10 x 6 nodes on the terrain (S-contacts on the bottom layer): z-slabs
    return scenes.terrain_lattice(np.float64, dims=(12, 10, 6))


class OracleShard:
    """Stand-in for a shard's library context: the oracle's sweep on the
    assembled vector, the shard's rows kept."""

    def __init__(self, P, w, plan):
        self.P, self.w, self.plan = P, w, plan
        self.own = slice(3 * plan.n0, 3 * plan.n1)
        self.halo_dofs = (3 * plan.halo[:, None] + np.arange(3)).ravel()
        self.h = np.zeros(3 * len(plan.halo))
        self.v = None

    def set_velocity(self, v):
        self.v = np.array(v, dtype=np.float64)

    def get_velocity(self):
        return self.v.copy()

    def get_nodes(self, ids, out):
        out.copy_(torch.from_numpy(self.v.reshape(-1, 3)[np.asarray(ids)].ravel()))
        return out

    def set_halo(self, first, vals):
        vals = np.asarray(vals.cpu() if hasattr(vals, "cpu") else vals, dtype=np.float64)
        self.h[3 * first:3 * first + len(vals)] = vals

    def shard_sweep(self):
        full = np.zeros(self.P.n)
        full[self.own] = self.v
        full[self.halo_dofs] = self.h
        new = ov.sweep(self.P, self.w, full).v_next[self.own]
        d = new - self.v
        self.v = new
        return math.fsum(d * d)


def test_partition_covers_every_node_with_balanced_blocks():
    sc = scenes.terrain_lattice(np.float32, dims=(16, 16, 12))
    for k in (1, 2, 3, 5):
        ranges = shard.partition(sc.row_ptr, k)
        assert ranges[0][0] == 0 and ranges[-1][1] == sc.n_nodes
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        blocks = [sc.row_ptr[b] - sc.row_ptr[a] for a, b in ranges]
        assert max(blocks) - min(blocks) <= 2 * np.diff(sc.row_ptr).max()
    with pytest.raises(ValueError):
        shard.partition(sc.row_ptr, 0)
    ranges = shard.partition(sc.row_ptr, 5, align=256)
    assert all(a % 256 == 0 for a, _ in ranges) and ranges[-1][1] == sc.n_nodes
    with pytest.raises(ValueError):
        shard.partition(sc.row_ptr, 2, align=7)


def test_plans_agree_on_what_each_pair_exchanges():
    """What shard p sends to q is q's halo segment owned by p, node for node,
    in q's halo order; local columns map back to the scene's columns."""
    sc = scene()
    ranges = shard.partition(sc.row_ptr, 3, align=12 * 10)
    assert ranges == [(0, 240), (240, 480), (480, 720)]
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(3)]
    for q in plans:
        for p, (first, n) in q.recv.items():
            sent = plans[p].send[q.rank] + plans[p].n0
            assert np.array_equal(sent, q.halo[first:first + n])
        glob = np.where(q.col_idx < q.n_own, q.col_idx + q.n0,
                        q.halo[np.maximum(q.col_idx - q.n_own, 0)])
        assert np.array_equal(glob, sc.col_idx[q.blocks])
        assert set(q.recv) == {p for p in range(3) if q.rank in plans[p].send}
    # z-slabs of a 27-point lattice: neighbours only, one layer each way
    assert set(plans[1].recv) == {0, 2} and set(plans[0].recv) == {1}
    assert len(plans[0].halo) == 12 * 10


def test_contacts_across_shards_are_refused():
    sc = scenes.random_problem(np.random.default_rng(3), 40, 6, d_contacts=6, density=0.2)
    ranges = shard.partition(sc.row_ptr, 2)
    cross = (sc.node_j >= 0) & ((sc.node_i < ranges[0][1]) != (sc.node_j < ranges[0][1]))
    if not cross.any():
        pytest.skip("seed gave no contact across the cut")
    with pytest.raises(ValueError):
        shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, 0)


def _unsplit(sc):
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    return P, w, ov.solve(P, w, sc.v0, theta_th=THETA, l_max=L_MAX, norm="rms")


def test_sharded_loop_in_one_process_reproduces_the_unsplit_solve():
    sc = scene()
    P, w, ref = _unsplit(sc)
    for k in (2, 3):
        ranges = shard.partition(sc.row_ptr, k)
        plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
                 for r in range(k)]
        engines = [OracleShard(P, w, pl) for pl in plans]
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=THETA, l_max=L_MAX,
                              norm="rms", dtype=torch.float64, device="cpu")
        assert r.iters == ref.iters and r.status == 0
        assert np.array_equal(r.v, ref.v)
        assert abs(r.theta - ref.theta) <= 1e-14 * ref.theta


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        sc = scene()
        P = oracle_problem(sc)
        w = ov.frobenius_w(P)
        ranges = shard.partition(sc.row_ptr, world)
        plan = shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, rank)
        eng = OracleShard(P, w, plan)
        r = shard.solve(eng, plan, shard.TorchComm(dist, "cpu"), sc.v0[3 * plan.n0:3 * plan.n1],
                        n_dof=sc.n, theta_th=THETA, l_max=L_MAX, norm="rms",
                        dtype=torch.float64, device="cpu")
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), v=r.v, iters=r.iters, theta=r.theta,
                 status=r.status)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_unsplit_solve(world, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    sc = scene()
    _, _, ref = _unsplit(sc)
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    assert all(int(g["iters"]) == ref.iters for g in got)
    assert all(float(g["theta"]) == float(got[0]["theta"]) for g in got)   # one decision
    assert abs(float(got[0]["theta"]) - ref.theta) <= 1e-14 * ref.theta
    assert np.array_equal(np.concatenate([g["v"] for g in got]), ref.v)
