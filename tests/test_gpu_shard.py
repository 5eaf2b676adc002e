"""Sharded scene on one GPU: a lattice split into z-slabs, each slab a library
context with a halo (vfpi_create with n_halo), swept in lock step in one
process with the boundary rows exchanged by the host loop of
shard.solve_local.  The shards keep the scene's column order, so every row's
sum, W and contact step are the unsplit solve's: after any number of sweeps
the iterate and the impulses equal the unsplit solve's bit for bit.  Also
against the FP64 oracle at the benchmark's stop test, and the shard entry
points' argument checks."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.checks import scc_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import shard, vfpi  # noqa: E402

DIMS = (40, 36, 12)


@pytest.fixture(scope="module")
def lattice():
    return scenes.terrain_lattice(dims=DIMS)


def make_shards(sc, k, **kw):
    ranges = shard.partition(sc.row_ptr, k, align=DIMS[0] * DIMS[1])
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    return plans, [shard.shard_solver(sc, pl, **kw) for pl in plans]


def lambdas(engines, plans, n_c):
    lam = np.full((n_c, 3), np.nan, dtype=np.float32)
    for e, pl in zip(engines, plans):
        lam[pl.contacts] = np.asarray(e.get_lambda()).reshape(-1, 3)
    return lam


@pytest.mark.parametrize("k", [2, 3])
def test_shards_equal_the_unsplit_solve_bitwise(lattice, k):
    sc = lattice
    plans, engines = make_shards(sc, k)
    try:
        assert all(len(pl.halo) > 0 for pl in plans)
        for sweeps in (1, 7, 30):
            with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps) as s:
                assert s.layout()["path"] == 1
                ref = s.solve(sc.v0)
            r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                                  norm="abs", device="cuda")
            assert r.iters == sweeps
            assert np.array_equal(r.v, ref.v), sweeps
            assert np.array_equal(lambdas(engines, plans, sc.n_c), np.asarray(ref.lam).reshape(-1, 3))
            # theta: the same squares, summed per shard then over shards
            assert abs(r.theta - ref.theta) <= 1e-12 * ref.theta
    finally:
        for e in engines:
            e.close()


def test_shards_converged_against_the_oracle(lattice):
    """At the benchmark's stop test (theta_rms < 1e-6) against the FP64
    oracle on the whole scene: relative error <= 1e-5, SCC residual <= 1e-6."""
    sc = lattice
    plans, engines = make_shards(sc, 2)
    try:
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=1e-6, l_max=200,
                              norm="rms", device="cuda")
        lam = lambdas(engines, plans, sc.n_c)
    finally:
        for e in engines:
            e.close()
    assert r.status == vfpi.VFPI_OK
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, np.asarray(sc.v0, float), theta_th=1e-6, l_max=200, norm="rms")
    assert abs(r.iters - ref.iters) <= 1
    if r.iters != ref.iters:
        ref = ov.solve(P, w, np.asarray(sc.v0, float), theta_th=0.0, l_max=r.iters)
    v = np.asarray(r.v, float)
    assert np.linalg.norm(v - ref.v) <= 1e-5 * np.linalg.norm(ref.v)
    assert np.abs(v - ref.v).max() <= 1e-5 * np.abs(ref.v).max()
    assert scc_residual(P, v, lam.astype(float)) <= 1e-6


def test_shard_entry_points_check_their_arguments(lattice):
    sc = lattice
    plans, engines = make_shards(sc, 2)
    e, pl = engines[0], plans[0]
    code = vfpi.STATUS_CODES
    try:
        with pytest.raises(vfpi.VfpiError) as x:
            e.get_nodes(np.array([0, pl.n_own], dtype=np.int32))
        assert x.value.status == code["VFPI_ERR_INVALID_ARG"]
        with pytest.raises(vfpi.VfpiError) as x:
            e.set_halo(len(pl.halo) - 1, np.zeros(6, np.float32))
        assert x.value.status == code["VFPI_ERR_INVALID_ARG"]
        for call in (lambda: e.solve(sc.v0[:3 * pl.n_own]), lambda: e.set_chebyshev(5),
                     lambda: e.matvec(np.zeros(3 * pl.n_own, np.float32)),
                     lambda: e.adjoint(np.zeros(3 * pl.n_own, np.float32))):
            with pytest.raises(vfpi.VfpiError) as x:
                call()
            assert x.value.status == code["VFPI_ERR_UNSUPPORTED"]
        # the halo values are what the row products read: a halo row moved by
        # hand changes the next sweep of the rows next to it, and only those
        e.set_velocity(sc.v0[:3 * pl.n_own])
        e.set_halo(0, np.zeros(3 * len(pl.halo), np.float32))
        e.shard_sweep()
        a = np.asarray(e.get_velocity())
        e.set_velocity(sc.v0[:3 * pl.n_own])
        e.set_halo(0, np.full(3 * len(pl.halo), 0.5, np.float32))
        e.shard_sweep()
        b = np.asarray(e.get_velocity())
        moved = np.unique(np.nonzero(a != b)[0] // 3)
        layer = DIMS[0] * DIMS[1]
        assert len(moved) and moved.min() >= pl.n_own - layer      # the slab's top layer
    finally:
        for x in engines:
            x.close()
    # a shard's pattern: a repeated column, a column past the halo, Chebyshev
    bad = plans[0].col_idx.copy()
    bad[1] = bad[0]
    with pytest.raises(vfpi.VfpiError):
        vfpi.Solver(pl.row_ptr, bad, sc.vals[pl.blocks], sc.b[:3 * pl.n_own], pl.node_i,
                    pl.node_j, sc.R[pl.contacts], sc.mu[pl.contacts], sc.phi[pl.contacts],
                    n_halo=len(pl.halo))
    bad = plans[0].col_idx.copy()
    bad[-1] = pl.n_own + len(pl.halo)
    with pytest.raises(vfpi.VfpiError):
        vfpi.Solver(pl.row_ptr, bad, sc.vals[pl.blocks], sc.b[:3 * pl.n_own], pl.node_i,
                    pl.node_j, sc.R[pl.contacts], sc.mu[pl.contacts], sc.phi[pl.contacts],
                    n_halo=len(pl.halo))
    with pytest.raises(vfpi.VfpiError) as x:
        shard.shard_solver(sc, pl, chebyshev_ls=5)
    assert x.value.status == code["VFPI_ERR_UNSUPPORTED"]


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, sweeps):
    """One rank: its shard's library context on the GPU, the boundary rows
    moved through host tensors over gloo (no kernel waits on another rank:
    every exchange goes through the host between launches)."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        sc = scenes.terrain_lattice(dims=DIMS)
        ranges = shard.partition(sc.row_ptr, world, align=DIMS[0] * DIMS[1])
        plan = shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, rank)
        with shard.shard_solver(sc, plan) as eng:
            r = shard.solve(eng, plan, shard.TorchComm(dist, "cpu"),
                            sc.v0[3 * plan.n0:3 * plan.n1], n_dof=sc.n, theta_th=0.0,
                            l_max=sweeps, norm="abs", device="cpu")
            lam = np.asarray(eng.get_lambda())
        np.savez(f"{out_dir}/r{rank}.npz", v=np.asarray(r.v), lam=lam, iters=r.iters,
                 theta=r.theta, contacts=plan.contacts)
    finally:
        dist.destroy_process_group()


def test_two_processes_over_gloo_equal_the_unsplit_solve(lattice, tmp_path):
    """shard.solve over torch.distributed with the library's shard contexts:
    two ranks (processes) on this GPU, the unsplit solve's iterate and
    impulses bit for bit after 12 sweeps."""
    import torch.multiprocessing as mp
    sweeps = 12
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), sweeps), nprocs=2,
                       start_method="spawn")
    sc = lattice
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps) as s:
        ref = s.solve(sc.v0)
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(2)]
    assert all(int(g["iters"]) == sweeps for g in got)
    assert float(got[0]["theta"]) == float(got[1]["theta"])
    assert np.array_equal(np.concatenate([g["v"] for g in got]), ref.v)
    lam = np.full((sc.n_c, 3), np.nan, dtype=np.float32)
    for g in got:
        lam[g["contacts"]] = g["lam"].reshape(-1, 3)
    assert np.array_equal(lam, np.asarray(ref.lam).reshape(-1, 3))


def test_shards_with_d_contacts_in_fp64_equal_the_unsplit_solve():
    """FP64, a random SPD problem with S- and D-contacts (the D-contact phase
    and its mid-sweep barrier run on every shard), each D-contact inside one
    shard: bitwise the unsplit solve after 1 and 9 sweeps, and at convergence
    within FP64 rounding of the oracle."""
    import dataclasses
    rng = np.random.default_rng(7)
    sc = scenes.random_problem(rng, 300, 40, d_contacts=40, density=0.03, couple=0.4)
    ranges = shard.partition(sc.row_ptr, 2)
    cut = ranges[0][1]
    keep = (sc.node_j < 0) | ((sc.node_i < cut) == (sc.node_j < cut))
    sc = dataclasses.replace(sc, node_i=sc.node_i[keep], node_j=sc.node_j[keep], R=sc.R[keep],
                             mu=sc.mu[keep], phi=sc.phi[keep])
    assert (sc.node_j >= 0).sum() >= 10
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(2)]
    assert all((pl.node_j >= 0).any() for pl in plans)
    engines = [shard.shard_solver(sc, pl, dtype="f64") for pl in plans]
    try:
        for sweeps in (1, 9):
            with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps, force_path=1) as s:
                ref = s.solve(sc.v0)
            r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                                  dtype=torch.float64, device="cuda")
            assert np.array_equal(r.v, ref.v), sweeps
            lam = np.full((sc.n_c, 3), np.nan)
            for e, pl in zip(engines, plans):
                lam[pl.contacts] = np.asarray(e.get_lambda()).reshape(-1, 3)
            assert np.array_equal(lam, np.asarray(ref.lam).reshape(-1, 3)), sweeps
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=1e-12, l_max=20000,
                              dtype=torch.float64, device="cuda")
    finally:
        for e in engines:
            e.close()
    assert r.status == vfpi.VFPI_OK
    P = oracle_problem(sc)
    ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=200000)
    assert np.linalg.norm(r.v - ref.v) <= 1e-9 * np.linalg.norm(ref.v)
