"""Host logic of the sharded scene (paper_2201_09212_gb300/shard.py) on the CPU:
the row partition, the halo and send lists, and the sweep loop with its
exchange and theta assembly, run over gloo ranks (world size 2 and 3) and in
one process.  The sweep itself is played by a stand-in engine that runs the
FP64 oracle's sweep (Alg. 1 + Alg. 2) on the whole scene's vector assembled
from the shard's own rows and halo: a shard's rows read only own and halo
columns, so its rows of that sweep are exactly the unsplit sweep's rows.  A
D-contact across a cut (a split contact) takes its step in the stand-in's
second half-sweep from its own endpoint's v* and the other endpoint's v*
received through the loop's exchange.  The sharded solve must therefore
reproduce the unsplit oracle solve bit for bit (theta, summed per shard and
then over shards, to rounding)."""
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


def dofs(nodes):
    return (3 * np.asarray(nodes, dtype=np.int64)[:, None] + np.arange(3)).ravel()


def contact_stage(P, w, v_star):
    """Alg. 2 and eq. (vup) from a given v* (the second half of the oracle's sweep)."""
    eta = (P.Jc @ v_star).reshape(-1, 3)
    rhs = eta.copy()
    rhs[:, 0] += P.phi
    lam_star = -np.linalg.solve(ov.gamma_blocks(P, w), rhs[:, :, None])[:, :, 0]
    lam = ov.project_strict(lam_star, P.mu)
    return v_star + w * (P.Jc.T @ lam.ravel())


def row_stats(P, nodes):
    """[6 per node]: a_rr of the node's three rows, then their ||A_r*||^2."""
    A = P.A.tocsr()
    r = dofs(nodes).reshape(-1, 3)
    d = A.diagonal()[r]
    q = np.asarray(A.multiply(A).sum(axis=1)).ravel()[r]
    return np.concatenate([d, q], axis=1).ravel()


class OracleShard:
    """Stand-in for a shard's library context: the oracle's sweep on the
    assembled vector, the shard's rows kept; split contacts finish in a second
    half-sweep, as in the library.  cheb = (l_s, u): Alg. 3's combination on
    the shard's rows (the oracle's formula), with the weight that the scene's
    thetas give (shard_set_theta)."""

    def __init__(self, P, w, plan, cheb=None):
        self.P, self.w, self.plan, self.cheb = P, w, plan, cheb
        self.own = slice(3 * plan.n0, 3 * plan.n1)
        self.halo_dofs = (3 * plan.halo[:, None] + np.arange(3)).ravel()
        self.h = np.zeros(3 * len(plan.halo))
        self.v = None
        m = plan.contacts[plan.split]
        ni, nj = P.node_i[m], P.node_j[m]
        here = (ni >= plan.n0) & (ni < plan.n1)
        self.split_own = np.where(here, ni, nj)          # global endpoint nodes
        self.split_other = np.where(here, nj, ni)
        self.stats_set = len(m) == 0

    def set_velocity(self, v):
        self.v = np.array(v, dtype=np.float64)
        self.v_prev = self.v.copy()
        self.l, self.nu, self.rho, self.th1, self.th2 = 1, 1.0, 0.0, 0.0, 0.0

    def shard_set_theta(self, theta):
        if self.cheb:
            l_s = self.cheb[0]
            if self.l >= 3:
                self.rho = min(self.th1 / self.th2, 1.0) if self.th2 > 0 else 1.0
            self.th2, self.th1 = self.th1, theta
            self.nu = ov.chebyshev_nu(self.l + 1, l_s, self.rho, self.nu)
        self.l += 1

    def _combine(self, vss, v, v_prev):
        if not self.cheb:
            return vss
        u = self.cheb[1]
        return self.nu * (u * (vss - v) + v - v_prev) + v_prev

    def get_velocity(self):
        return self.v.copy()

    def get_nodes(self, ids, out):
        out.copy_(torch.from_numpy(self.v.reshape(-1, 3)[np.asarray(ids)].ravel()))
        return out

    def set_halo(self, first, vals):
        vals = np.asarray(vals.cpu() if hasattr(vals, "cpu") else vals, dtype=np.float64)
        self.h[3 * first:3 * first + len(vals)] = vals

    def shard_sweep(self, sumsq=True):
        full = np.zeros(self.P.n)
        full[self.own] = self.v
        full[self.halo_dofs] = self.h
        r = ov.sweep(self.P, self.w, full)
        new = self._combine(r.v_next[self.own], self.v, self.v_prev)
        loc = dofs(self.split_own) - 3 * self.plan.n0
        new[loc] = self.v[loc]                   # split endpoints: v^l until the second half
        self.split_prev = self.v_prev[loc].copy()
        self.vstar = r.v_star
        d = new - self.v
        self.v_prev = self.v
        self.v = new
        self.s2 = math.fsum(d * d)
        return self.s2 if sumsq else None

    def split_stats(self, out):
        out.copy_(torch.from_numpy(row_stats(self.P, self.split_own)))
        return out

    def set_split_stats(self, partner):
        # what arrives for each split contact is its other endpoint's statistics
        assert np.array_equal(np.asarray(partner), row_stats(self.P, self.split_other))
        self.stats_set = True

    def split_vstar(self, out):
        out.copy_(torch.from_numpy(self.vstar[dofs(self.split_own)]))
        return out

    def finish_split(self, partner):
        assert self.stats_set
        vs = self.vstar.copy()
        vs[dofs(self.split_other)] = np.asarray(partner)
        loc = dofs(self.split_own) - 3 * self.plan.n0
        new = self._combine(contact_stage(self.P, self.w, vs)[dofs(self.split_own)], self.v[loc],
                            self.split_prev)
        d = new - self.v[loc]
        self.v[loc] = new
        return self.s2 + math.fsum(d * d)


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


def split_scene(seed=3, n=60, d=14):
    """Random SPD problem with S- and D-contacts; D-contacts pair random nodes,
    so about half of them cross any cut."""
    return scenes.random_problem(np.random.default_rng(seed), n, 8, d_contacts=d, density=0.08,
                                 couple=0.4)


@pytest.mark.parametrize("k", [2, 3])
def test_split_contact_plans(k):
    """Every contact is held by the shards of its nodes and reported by the
    shard of its lower-numbered node; local node indices map back to the
    scene's; two shards list the split contacts they share in the same order."""
    sc = split_scene()
    ranges = shard.partition(sc.row_ptr, k)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    owner = shard.owner_of(ranges, np.arange(sc.n_nodes))
    n_split = 0
    for m in range(sc.n_c):
        i, j = sc.node_i[m], sc.node_j[m]
        holders = {int(owner[i])} | ({int(owner[j])} if j >= 0 else set())
        assert {pl.rank for pl in plans if m in pl.contacts} == holders
        low = i if j < 0 else min(i, j)
        assert [pl.rank for pl in plans if m in pl.contacts[pl.owns]] == [int(owner[low])]
        n_split += len(holders) == 2
    assert n_split >= 3
    for pl in plans:
        def glob(q):
            return np.where(q < pl.n_own, q + pl.n0, pl.halo[np.maximum(q - pl.n_own, 0)])
        assert np.array_equal(glob(pl.node_i), sc.node_i[pl.contacts])
        dj = pl.node_j >= 0
        assert np.array_equal(glob(pl.node_j[dj]), sc.node_j[pl.contacts][dj])
        assert (pl.node_j[~dj] == -1).all()
        # the rows' halo first (it alone is exchanged every sweep), then the other
        # endpoints of split contacts that no row references
        assert pl.n_halo_rows == len(shard.halo_of(sc.row_ptr, sc.col_idx, pl.n0, pl.n1))
        assert sum(n for _, n in pl.recv.values()) == pl.n_halo_rows
        for p, idx in pl.split_peer.items():
            q = plans[p]
            mine = pl.contacts[pl.split[idx]]
            assert np.array_equal(mine, q.contacts[q.split[q.split_peer[pl.rank]]])
            assert np.all(np.diff(mine) > 0)


@pytest.mark.parametrize("k", [2, 3])
def test_split_contacts_in_one_process_reproduce_the_unsplit_solve(k):
    sc = split_scene()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ranges = shard.partition(sc.row_ptr, k)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    assert all(len(pl.split) for pl in plans)
    for sweeps in (1, 2, 25):
        ref = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=sweeps)
        engines = [OracleShard(P, w, pl) for pl in plans]
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                              dtype=torch.float64, device="cpu")
        assert r.iters == sweeps
        assert np.array_equal(r.v, ref.v), sweeps
        assert abs(r.theta - ref.theta) <= 1e-13 * ref.theta


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


def _rank_main(rank, world, port, out_dir, kind="lattice"):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        sc = scene() if kind == "lattice" else split_scene()
        P = oracle_problem(sc)
        w = ov.frobenius_w(P)
        ranges = shard.partition(sc.row_ptr, world)
        plan = shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, rank)
        eng = OracleShard(P, w, plan, cheb=(5, 0.9) if kind == "split-cheb" else None)
        th, lm, norm = (THETA, L_MAX, "rms") if kind == "lattice" else (0.0, SPLIT_SWEEPS, "abs")
        r = shard.solve(eng, plan, shard.TorchComm(dist, "cpu"), sc.v0[3 * plan.n0:3 * plan.n1],
                        n_dof=sc.n, theta_th=th, l_max=lm, norm=norm,
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


SPLIT_SWEEPS = 20


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_with_split_contacts_reproduce_the_unsplit_solve(world, tmp_path):
    """D-contacts across the cuts: the split contacts' v* and row statistics
    travel point to point between the ranks that share them."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), "split"),
                       nprocs=world, start_method="spawn")
    sc = split_scene()
    P = oracle_problem(sc)
    ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=SPLIT_SWEEPS)
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    assert all(int(g["iters"]) == SPLIT_SWEEPS for g in got)
    assert all(float(g["theta"]) == float(got[0]["theta"]) for g in got)
    assert abs(float(got[0]["theta"]) - ref.theta) <= 1e-13 * ref.theta
    assert np.array_equal(np.concatenate([g["v"] for g in got]), ref.v)


@pytest.mark.parametrize("kind,k", [("lattice", 2), ("lattice", 3), ("split", 2), ("split", 3)])
def test_chebyshev_shards_in_one_process_match_the_oracle(kind, k):
    """Alg. 3 across shards: each shard is given the scene's theta after every
    sweep and forms the next weight from it; the split solve equals the
    oracle's Alg. 3 on the whole scene to rounding (theta is summed per shard
    first, so the weights can differ in their last bits)."""
    sc = scene() if kind == "lattice" else split_scene()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ranges = shard.partition(sc.row_ptr, k)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    for sweeps in (3, 8, 30):
        ref = ov.solve_chebyshev(P, w, sc.v0, theta_th=0.0, l_max=sweeps, l_s=5, u=0.9)
        engines = [OracleShard(P, w, pl, cheb=(5, 0.9)) for pl in plans]
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                              dtype=torch.float64, device="cpu")
        assert r.iters == sweeps
        assert np.linalg.norm(r.v - ref.v) <= 1e-12 * np.linalg.norm(ref.v), sweeps
        assert abs(r.theta - ref.theta) <= 1e-10 * ref.theta
    # mid-solve, Alg. 3's iterate is not the plain one
    plain = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=8)
    acc = ov.solve_chebyshev(P, w, sc.v0, theta_th=0.0, l_max=8, l_s=5, u=0.9)
    assert np.linalg.norm(plain.v - acc.v) > 1e-6 * np.linalg.norm(acc.v)


def test_gloo_ranks_with_chebyshev_and_split_contacts_match_the_oracle(tmp_path):
    """Alg. 3 over two gloo ranks with D-contacts across the cut: the scene's
    theta (all-gathered, summed in rank order) gives both ranks the same
    weights; the result is the oracle's Alg. 3 on the whole scene to rounding."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), "split-cheb"),
                       nprocs=2, start_method="spawn")
    sc = split_scene()
    P = oracle_problem(sc)
    ref = ov.solve_chebyshev(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=SPLIT_SWEEPS,
                             l_s=5, u=0.9)
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(2)]
    assert all(int(g["iters"]) == SPLIT_SWEEPS for g in got)
    assert float(got[0]["theta"]) == float(got[1]["theta"])
    v = np.concatenate([g["v"] for g in got])
    assert np.linalg.norm(v - ref.v) <= 1e-12 * np.linalg.norm(ref.v)
