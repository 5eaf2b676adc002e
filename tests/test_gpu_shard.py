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


def lambdas(engines, plans, n_c, dtype=np.float32):
    """The scene's lambda, each contact from the shard that owns it; a split
    contact's other shard must hold the same lambda bit for bit."""
    lam = np.full((n_c, 3), np.nan, dtype=dtype)
    for e, pl in zip(engines, plans):
        lam[pl.contacts[pl.owns]] = np.asarray(e.get_lambda()).reshape(-1, 3)[pl.owns]
    for e, pl in zip(engines, plans):
        mine = np.asarray(e.get_lambda()).reshape(-1, 3)
        assert np.array_equal(mine, lam[pl.contacts])
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
        for call in (lambda: e.solve(sc.v0[:3 * pl.n_own]), lambda: e.set_adjoint_chebyshev(5),
                     lambda: e.matvec(np.zeros(3 * pl.n_own, np.float32)),
                     lambda: e.adjoint(np.zeros(3 * pl.n_own, np.float32))):
            with pytest.raises(vfpi.VfpiError) as x:
                call()
            assert x.value.status == code["VFPI_ERR_UNSUPPORTED"]
        for th in (-1.0, float("nan")):
            with pytest.raises(vfpi.VfpiError) as x:
                e.shard_set_theta(th)
            assert x.value.status == code["VFPI_ERR_NONFINITE"]
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
    # a shard's pattern: a repeated column, a column past the halo; a whole
    # scene takes no shard step
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
    with vfpi.Solver.from_scene(sc) as whole:
        with pytest.raises(vfpi.VfpiError) as x:
            whole.shard_set_theta(1.0)
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


def with_split_d_contacts(sc, ranges, n_per_cut=40, seed=11):
    """The lattice plus D-contacts across each cut: node a within three layers
    below the cut, node b within three layers above (some pairs coupled in A,
    most not, so the other endpoint is a row-halo node or an extra halo node),
    no node in two contacts, none on the contact layer."""
    import dataclasses
    rng = np.random.default_rng(seed)
    layer = DIMS[0] * DIMS[1]
    used = set(int(x) for x in sc.node_i)
    ni, nj = [], []
    for c in (r[0] for r in ranges[1:]):
        k = 0
        while k < n_per_cut:
            a = int(rng.integers(max(c - 3 * layer, layer), c))
            b = int(rng.integers(c, min(c + 3 * layer, sc.n_nodes)))
            if a in used or b in used:
                continue
            used.update((a, b))
            # half of them with the lower node as node j
            ni.append(a if k % 2 else b)
            nj.append(b if k % 2 else a)
            k += 1
    m = len(ni)
    R = scenes.random_rotations(rng, m).astype(sc.R.dtype)
    return dataclasses.replace(
        sc, node_i=np.concatenate([sc.node_i, ni]).astype(np.int32),
        node_j=np.concatenate([sc.node_j, nj]).astype(np.int32),
        R=np.concatenate([sc.R, R]), mu=np.concatenate([sc.mu, rng.uniform(0.2, 0.8, m)]).astype(sc.mu.dtype),
        phi=np.concatenate([sc.phi, rng.uniform(-0.05, 0.02, m)]).astype(sc.phi.dtype))


@pytest.mark.parametrize("k", [2, 3])
def test_split_d_contacts_equal_the_unsplit_solve_bitwise(lattice, k):
    """FP32 lattice with D-contacts across the cuts (v* exchanged mid-sweep,
    row statistics before the first): iterate and impulses bit for bit the
    unsplit solve's after 1, 7 and 30 sweeps."""
    ranges = shard.partition(lattice.row_ptr, k, align=DIMS[0] * DIMS[1])
    sc = with_split_d_contacts(lattice, ranges)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    engines = [shard.shard_solver(sc, pl) for pl in plans]
    try:
        for e, pl in zip(engines, plans):
            assert e.shard_info() == (len(pl.halo), len(pl.split)) and len(pl.split) >= 40
            assert len(pl.halo) > pl.n_halo_rows          # endpoints no row references
        for sweeps in (1, 7, 30):
            with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps, force_path=1) as s:
                ref = s.solve(sc.v0)
            r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                                  device="cuda")
            assert np.array_equal(r.v, ref.v), sweeps
            assert np.array_equal(lambdas(engines, plans, sc.n_c), np.asarray(ref.lam).reshape(-1, 3))
            assert abs(r.theta - ref.theta) <= 1e-12 * ref.theta
    finally:
        for e in engines:
            e.close()


@pytest.mark.parametrize("k", [2, 3])
def test_split_d_contacts_in_fp64_against_the_oracle(k):
    """FP64, a random SPD problem whose D-contacts pair random nodes (about
    half cross a cut): bitwise the unsplit solve after 1 and 9 sweeps, and at
    convergence within FP64 rounding of the oracle."""
    rng = np.random.default_rng(7)
    sc = scenes.random_problem(rng, 300, 40, d_contacts=40, density=0.03, couple=0.4)
    ranges = shard.partition(sc.row_ptr, k)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    assert all(len(pl.split) >= 5 for pl in plans)
    engines = [shard.shard_solver(sc, pl, dtype="f64") for pl in plans]
    try:
        for sweeps in (1, 9):
            with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps, force_path=1) as s:
                ref = s.solve(sc.v0)
            r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                                  dtype=torch.float64, device="cuda")
            assert np.array_equal(r.v, ref.v), sweeps
            lam = lambdas(engines, plans, sc.n_c, np.float64)
            assert np.array_equal(lam, np.asarray(ref.lam).reshape(-1, 3)), sweeps
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=1e-12, l_max=20000,
                              dtype=torch.float64, device="cuda")
        lam = lambdas(engines, plans, sc.n_c, np.float64)
    finally:
        for e in engines:
            e.close()
    assert r.status == vfpi.VFPI_OK
    P = oracle_problem(sc)
    ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=200000)
    assert np.linalg.norm(r.v - ref.v) <= 1e-9 * np.linalg.norm(ref.v)
    assert scc_residual(P, r.v, lam) <= 1e-9


def test_split_contact_calls_check_their_arguments():
    rng = np.random.default_rng(7)
    sc = scenes.random_problem(rng, 120, 10, d_contacts=20, density=0.05, couple=0.4)
    ranges = shard.partition(sc.row_ptr, 2)
    pl = shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, 0)
    code = vfpi.STATUS_CODES
    n_split = len(pl.split)
    assert n_split > 0
    with shard.shard_solver(sc, pl, dtype="f64") as e:
        # the tied W needs the other endpoints' statistics before a sweep
        with pytest.raises(vfpi.VfpiError) as x:
            e.shard_sweep()
        assert x.value.status == code["VFPI_ERR_INVALID_ARG"]
        bad = np.ones(6 * n_split)
        bad[3] = np.inf
        with pytest.raises(vfpi.VfpiError) as x:
            e.set_split_stats(bad)
        assert x.value.status == code["VFPI_ERR_NONFINITE"]
        st = e.split_stats()
        assert st.shape == (6 * n_split,) and (st[0::6] > 0).all()
        e.set_split_stats(st)                     # any finite statistics are taken
        e.set_velocity(sc.v0[3 * pl.n0:3 * pl.n1])
        e.shard_sweep()
        # the own endpoints stay at v^l until the second half of the sweep
        own = np.where(pl.node_i[pl.split] < pl.n_own, pl.node_i[pl.split], pl.node_j[pl.split])
        v = np.asarray(e.get_velocity()).reshape(-1, 3)
        assert np.array_equal(v[own], sc.v0.reshape(-1, 3)[pl.n0 + own])
        assert e.split_vstar().shape == (3 * n_split,)
        e.finish_split(e.split_vstar())
        assert not np.array_equal(np.asarray(e.get_velocity()).reshape(-1, 3)[own],
                                  sc.v0.reshape(-1, 3)[pl.n0 + own])
    # an S-contact on a halo node, a D-contact between two halo nodes
    for ni, nj in ((pl.n_own, -1), (pl.n_own, pl.n_own + 1)):
        with pytest.raises(vfpi.VfpiError) as x:
            vfpi.Solver(pl.row_ptr, pl.col_idx, sc.vals[pl.blocks], sc.b[3 * pl.n0:3 * pl.n1],
                        np.array([ni], np.int32), np.array([nj], np.int32), sc.R[:1], sc.mu[:1],
                        sc.phi[:1], dtype="f64", n_halo=len(pl.halo))
        assert x.value.status == code["VFPI_ERR_INVALID_ARG"]


@pytest.mark.parametrize("k", [2, 3])
def test_chebyshev_shards_with_split_contacts_equal_the_unsplit_solve(lattice, k):
    """Alg. 3 (l_s = 5, u = 1) on the FP32 lattice with D-contacts across the
    cuts: each shard gets the scene's theta after every sweep and forms the
    weight from it.  theta is summed per shard first, so the weights can
    differ from the unsplit solve's in their last bits (FP64); the iterates
    agree to FP32 rounding after 1, 7 and 30 sweeps, and at the benchmark's
    stop test with the oracle's Alg. 3."""
    ranges = shard.partition(lattice.row_ptr, k, align=DIMS[0] * DIMS[1])
    sc = with_split_d_contacts(lattice, ranges)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(k)]
    engines = [shard.shard_solver(sc, pl, chebyshev_ls=5, chebyshev_u=1.0) for pl in plans]
    try:
        for sweeps in (1, 7, 30):
            with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=sweeps, force_path=1,
                                        chebyshev_ls=5, chebyshev_u=1.0) as s:
                ref = s.solve(sc.v0)
            r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=sweeps,
                                  device="cuda")
            assert np.linalg.norm(r.v - ref.v) <= 1e-6 * np.linalg.norm(ref.v), sweeps
            lam = lambdas(engines, plans, sc.n_c)
            ref_lam = np.asarray(ref.lam).reshape(-1, 3)
            assert np.linalg.norm(lam - ref_lam) <= 1e-5 * np.linalg.norm(ref_lam), sweeps
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=1e-6, l_max=200,
                              norm="rms", device="cuda")
        lam = lambdas(engines, plans, sc.n_c)
    finally:
        for e in engines:
            e.close()
    assert r.status == vfpi.VFPI_OK
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve_chebyshev(P, w, np.asarray(sc.v0, float), theta_th=1e-6, l_max=200,
                             l_s=5, u=1.0, norm="rms")
    assert abs(r.iters - ref.iters) <= 1
    if r.iters != ref.iters:
        ref = ov.solve_chebyshev(P, w, np.asarray(sc.v0, float), theta_th=0.0, l_max=r.iters,
                                 l_s=5, u=1.0)
    v = np.asarray(r.v, float)
    assert np.linalg.norm(v - ref.v) <= 1e-5 * np.linalg.norm(ref.v)
    assert scc_residual(P, v, lam.astype(float)) <= 1e-6


def test_chebyshev_shards_in_fp64_against_the_unsplit_solve_and_the_oracle():
    rng = np.random.default_rng(7)
    sc = scenes.random_problem(rng, 300, 40, d_contacts=40, density=0.03, couple=0.4)
    ranges = shard.partition(sc.row_ptr, 2)
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(2)]
    engines = [shard.shard_solver(sc, pl, dtype="f64", chebyshev_ls=5, chebyshev_u=0.9)
               for pl in plans]
    try:
        with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=12, force_path=1, chebyshev_ls=5,
                                    chebyshev_u=0.9) as s:
            ref = s.solve(sc.v0)
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=0.0, l_max=12,
                              dtype=torch.float64, device="cuda")
        assert np.linalg.norm(r.v - ref.v) <= 1e-12 * np.linalg.norm(ref.v)
        r = shard.solve_local(engines, plans, sc.v0, n_dof=sc.n, theta_th=1e-12, l_max=20000,
                              dtype=torch.float64, device="cuda")
    finally:
        for e in engines:
            e.close()
    assert r.status == vfpi.VFPI_OK
    P = oracle_problem(sc)
    ref = ov.solve_chebyshev(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=200000, l_s=5,
                             u=0.9)
    assert np.linalg.norm(r.v - ref.v) <= 1e-9 * np.linalg.norm(ref.v)
