"""The seeded input generators against the recipe they are quoted with: block
counts from closed forms of the coupling patterns, contact counts, friction
and side distributions, symmetry and positive definiteness of A (CPU, small
copies)."""
import numpy as np
import pytest

from paper_2201_09212_gb300 import scenes


def kuhn_blocks(cx, cy, cz):
    """Blocks of A for a Kuhn-split cell grid: one per node plus two per edge
    (axis edges, one diagonal per cell face, one body diagonal per cell)."""
    nx, ny, nz = cx + 1, cy + 1, cz + 1
    axis = cx * ny * nz + nx * cy * nz + nx * ny * cz
    face = cx * cy * nz + cx * ny * cz + nx * cy * cz
    body = cx * cy * cz
    return nx * ny * nz + 2 * (axis + face + body)


def test_fem_block_pattern():
    assert kuhn_blocks(64, 64, 16) == 1_026_481          # the full-size block's count
    sc = scenes.fem_block(cells=(5, 4, 3))
    assert sc.n_nodes == 6 * 5 * 4 and sc.nnzb == kuhn_blocks(5, 4, 3)
    assert sc.n_c == 6 * 5 and np.allclose(sc.mu, 0.4)
    A = sc.dense_A().astype(np.float64)
    assert np.allclose(A, A.T, rtol=1e-6, atol=0)
    assert np.linalg.eigvalsh(A).min() > 0


def test_small_lattice_recipe():
    sc = scenes.small_lattice()
    assert (sc.n_nodes, sc.n, sc.nnzb, sc.n_c) == (216, 648, (3 * 6 - 2) ** 3, 36)
    assert np.all(sc.mu == 0.5) and np.all(sc.phi == 0.0) and np.all(sc.node_j == -1)
    A = sc.dense_A()
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > 0
    # warm start: -0.1 e_z plus small noise
    v = sc.v0.reshape(-1, 3)
    assert abs(v[:, 2].mean() + 0.1) < 1e-3 and abs(v[:, :2].mean()) < 1e-3


def test_terrain_lattice_recipe():
    sc = scenes.terrain_lattice(dims=(12, 10, 4))
    assert sc.nnzb == 34 * 28 * 10 and sc.n_c == 12 * 10
    assert sc.mu.min() >= 0.2 and sc.mu.max() <= 0.8
    R = sc.R.astype(np.float64)
    assert np.allclose(R @ R.transpose(0, 2, 1), np.eye(3), atol=1e-6)
    assert (R[:, 0, 2] > 0.9).all()                        # normals close to e_z


@pytest.mark.parametrize("side_range", [(4, 12), (4, 6)])
def test_batched_lattices_recipe(side_range):
    b = scenes.lattice_batch(64, seed=scenes.SEED_BASE + 4, side_range=side_range)
    k = np.asarray(b.meta["sides"])
    assert k.min() >= side_range[0] and k.max() <= side_range[1] and len(np.unique(k)) > 1
    stiff = np.asarray(b.meta["k"]) / 1e3                   # spring stiffness x U[0.5, 2]
    assert stiff.min() >= 0.5 and stiff.max() <= 2.0
    g = np.asarray(b.meta["gravity"], float)
    tilt = np.degrees(np.arccos(-g[:, 2] / np.linalg.norm(g, axis=1)))
    assert tilt.max() <= 30.0 + 1e-9 and np.allclose(np.linalg.norm(g, axis=1), scenes.GRAVITY)
    assert b.n_nodes == int((k ** 3).sum()) and b.n_c == int((k ** 2).sum())
    assert b.nnzb == int(((3 * k - 2) ** 3).sum())
    assert b.mu.min() >= 0.2 and b.mu.max() <= 0.8
    sp = np.asarray(b.scene_ptr)
    assert sp[0] == 0 and sp[-1] == b.n_nodes and np.array_equal(np.diff(sp), k ** 3)
