"""Seeded synthetic scene generators.

This module produces the *inputs* of the velocity fixed-point iteration:
the SPD system matrix ``A`` in 3x3 block-sparse row (BSR) form, the right-hand
side ``b``, the nodal contact records (node indices, contact frame ``R``,
friction ``mu``, penetration term ``phi``) and the warm-start velocity.  It is
harness code (the paper's "dynamics construction" and "collision detection",
Sec. II.A and Sec. III.A) and holds none of the solver's arithmetic, so both
the CUDA path and the CPU oracle consume its output.

Dynamics are backward Euler with linear springs / linear tetrahedra,
``A = M + h D + h^2 K`` and ``b = M v + h (f_ext + f_el(x))`` (a form the
paper allows, Sec. II.A, eq. (lindyn)/(newton)); springs use the Gauss-Newton
block ``k d d^T`` of eq. (hess_psi).  Contact frames are rotation matrices whose
rows are ``[n; t1; t2]`` (eq. (jcnode)); ``t1 = normalize(n x e)`` with
``e = e_x`` unless ``|n_x| > 0.9`` (then ``e_y``) and ``t2 = n x t1``.
``phi = d / h`` with ``d`` the signed gap along the normal (eq. (scc) leaves
the form of ``phi`` open).

Node order in every lattice is ``i = ix + nx * (iy + ny * iz)``; the bottom
layer (``iz = 0``) therefore holds the first ``nx * ny`` nodes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2201_09212
GRAVITY = 9.81


@dataclasses.dataclass
class Scene:
    """One linear contact problem ``A v = b + J_c^T lambda`` plus warm start."""

    n_nodes: int
    row_ptr: np.ndarray          # int32 [N+1]
    col_idx: np.ndarray          # int32 [nnzb], sorted per row, diagonal present
    vals: np.ndarray             # float [nnzb, 3, 3], row-major blocks
    b: np.ndarray                # float [3N]
    node_i: np.ndarray           # int32 [n_c]
    node_j: np.ndarray           # int32 [n_c], -1 for an S-contact
    R: np.ndarray                # float [n_c, 3, 3], rows n, t1, t2
    mu: np.ndarray               # float [n_c]
    phi: np.ndarray              # float [n_c]
    v0: np.ndarray               # float [3N] warm start
    h: float = 1e-3
    x0: np.ndarray | None = None     # float64 [3N] positions
    mass: np.ndarray | None = None   # float64 [3N] lumped mass per DOF
    scene_ptr: np.ndarray | None = None  # int32 [S+1] node offsets (batched)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return 3 * self.n_nodes

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_c(self) -> int:
        return int(self.node_i.shape[0])

    def rounded(self, dtype) -> "Scene":
        """Copy whose float arrays are rounded to ``dtype`` and kept in that dtype."""
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=dtype)
        return dataclasses.replace(
            self, vals=f(self.vals), b=f(self.b), R=f(self.R), mu=f(self.mu),
            phi=f(self.phi), v0=f(self.v0), meta=dict(self.meta))

    def as_f64(self) -> "Scene":
        """Copy with every float array promoted (exactly) to float64."""
        return self.rounded(np.float64)

    def dense_A(self) -> np.ndarray:
        n = self.n
        A = np.zeros((n, n), dtype=np.float64)
        for i in range(self.n_nodes):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                j = self.col_idx[p]
                A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = self.vals[p]
        return A


# ----------------------------------------------------------------------------
# contact frames
# ----------------------------------------------------------------------------

def contact_frames(normals: np.ndarray) -> np.ndarray:
    """Rotation matrices with rows ``[n; t1; t2]`` for unit normals ``[m, 3]``."""
    n = np.asarray(normals, dtype=np.float64)
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    e = np.zeros_like(n)
    use_y = np.abs(n[:, 0]) > 0.9
    e[~use_y, 0] = 1.0
    e[use_y, 1] = 1.0
    t1 = np.cross(n, e)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(n, t1)
    return np.stack([n, t1, t2], axis=1)


def random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """``m`` random proper rotations (QR of Gaussian matrices, det fixed to +1)."""
    g = rng.standard_normal((m, 3, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    det = np.linalg.det(q)
    q[det < 0, :, 2] *= -1.0
    return q


# ----------------------------------------------------------------------------
# structured BSR assembly (a regular grid of nodes, 27 possible neighbours)
# ----------------------------------------------------------------------------

def _offsets(nx: int, ny: int):
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    offs.sort(key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    return offs


def _grid_index(nx, ny, nz):
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ix.ravel(), iy.ravel(), iz.ravel()


def _compress(nx, ny, nz, diag, off, present, dtype):
    """Build sorted-column BSR from per-offset block arrays.

    ``off[k]`` is ``[N, 3, 3]`` for the k-th sorted offset (``None`` for the
    diagonal slot) and ``present[k]`` the boolean mask of rows holding it.
    """
    N = nx * ny * nz
    offs = _offsets(nx, ny)
    counts = np.zeros(N, dtype=np.int64)
    for k in range(27):
        counts += present[k]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnzb = int(row_ptr[-1])
    col = np.empty(nnzb, dtype=np.int32)
    vals = np.empty((nnzb, 3, 3), dtype=dtype)
    fill = row_ptr[:-1].copy()
    rows = np.arange(N, dtype=np.int64)
    for k, (dx, dy, dz) in enumerate(offs):
        m = present[k]
        if not m.any():
            continue
        r = rows[m]
        pos = fill[m]
        col[pos] = (r + dx + nx * (dy + ny * dz)).astype(np.int32)
        if dx == 0 and dy == 0 and dz == 0:
            vals[pos] = diag[m].astype(dtype)
        else:
            vals[pos] = off[k][m].astype(dtype)
        fill[m] += 1
    return row_ptr.astype(np.int32), col, vals


# ----------------------------------------------------------------------------
# mass-spring lattice (configs 1, 3, 4, 5)
# ----------------------------------------------------------------------------

def lattice_system(nx, ny, nz, x, rest, v, *, mass=1e-3, k=1e3, c=0.1, h=1e-3,
                   gravity=(0.0, 0.0, -GRAVITY), dtype=np.float64):
    """``A = M + h D + h^2 K`` and ``b = M v + h (m g + f_el)`` of a 26-neighbour lattice.

    ``x``/``rest`` are positions ``[N, 3]`` (current / rest); springs connect
    every node to its 26 grid neighbours with Gauss-Newton stiffness
    ``k d d^T`` and a dashpot ``c d d^T`` along the current direction ``d``.
    """
    N = nx * ny * nz
    ix, iy, iz = _grid_index(nx, ny, nz)
    offs = _offsets(nx, ny)
    x = np.asarray(x, dtype=np.float64).reshape(N, 3)
    rest = np.asarray(rest, dtype=np.float64).reshape(N, 3)
    coef = h * c + h * h * k
    diag = np.zeros((N, 3, 3), dtype=np.float64)
    diag[:, 0, 0] = diag[:, 1, 1] = diag[:, 2, 2] = mass
    f_el = np.zeros((N, 3), dtype=np.float64)
    off, present = [], []
    rows = np.arange(N)
    for (dx, dy, dz) in offs:
        m = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
             & (iz + dz >= 0) & (iz + dz < nz))
        present.append(m)
        if dx == 0 and dy == 0 and dz == 0:
            off.append(None)
            continue
        i = rows[m]
        j = i + dx + nx * (dy + ny * dz)
        dvec = x[j] - x[i]
        length = np.linalg.norm(dvec, axis=1)
        d = dvec / length[:, None]
        L0 = np.linalg.norm(rest[j] - rest[i], axis=1)
        ddt = d[:, :, None] * d[:, None, :]
        blk = np.zeros((N, 3, 3), dtype=dtype)
        blk[m] = (-coef * ddt).astype(dtype)
        off.append(blk)
        diag[m] += coef * ddt
        f_el[m] += (k * (length - L0))[:, None] * d
    row_ptr, col, vals = _compress(nx, ny, nz, diag, off, present, dtype)
    g = np.asarray(gravity, dtype=np.float64)
    b = (mass * np.asarray(v, dtype=np.float64).reshape(N, 3)
         + h * (mass * g[None, :] + f_el)).ravel()
    return row_ptr, col, vals, b


def heightfield(rng, nx, ny, spacing=0.01, amp=5e-3, period=0.32, noise=0.5e-3):
    """Sinusoid + uniform noise heightfield sampled on the lattice grid.

    Returns ``(H, S, normals)`` on ``[ny, nx]``: total height, its smooth part
    and unit normals from the central-difference gradient of ``H``.
    """
    xs = np.arange(nx) * spacing
    ys = np.arange(ny) * spacing
    S = amp * np.sin(2 * np.pi * xs[None, :] / period) * np.sin(2 * np.pi * ys[:, None] / period)
    H = S + rng.uniform(-noise, noise, size=S.shape)
    gy, gx = np.gradient(H, spacing, spacing)
    nrm = np.stack([-gx, -gy, np.ones_like(H)], axis=-1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    return H, S, nrm


def lattice_scene(nx, ny, nz, *, seed, spacing=0.01, mass=1e-3, k=1e3, c=0.1,
                  h=1e-3, v_down=0.1, v_sigma=1e-3, mu=0.5, terrain=False,
                  gravity=(0.0, 0.0, -GRAVITY), dtype=np.float64, mu_range=None):
    """A lattice resting with its bottom layer in contact.

    ``terrain=False``: flat ground ``z = 0``, bottom layer at ``z = 0``.
    ``terrain=True``: sinusoid+noise heightfield; the lattice is draped on the
    smooth part of the terrain (columns shifted by it), so each bottom node's
    gap is minus the local noise, up to +-0.5 mm.
    """
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    ix, iy, iz = _grid_index(nx, ny, nz)
    x = np.stack([ix * spacing, iy * spacing, iz * spacing], axis=1).astype(np.float64)
    nb = nx * ny
    if terrain:
        H, S, nrm = heightfield(rng, nx, ny, spacing)
        x[:, 2] += S[iy, ix]
        normals = nrm[iy[:nb], ix[:nb]]
        gap = (x[:nb, 2] - H[iy[:nb], ix[:nb]]) * normals[:, 2]
    else:
        normals = np.tile(np.array([0.0, 0.0, 1.0]), (nb, 1))
        gap = x[:nb, 2].copy()
    v = np.zeros((N, 3))
    v[:, 2] = -v_down
    v += rng.normal(0.0, v_sigma, size=(N, 3))
    row_ptr, col, vals, b = lattice_system(nx, ny, nz, x, x, v, mass=mass, k=k, c=c,
                                           h=h, gravity=gravity, dtype=dtype)
    if mu_range is not None:
        mus = rng.uniform(mu_range[0], mu_range[1], size=nb)
    else:
        mus = np.full(nb, mu)
    return Scene(
        n_nodes=N, row_ptr=row_ptr, col_idx=col, vals=vals, b=b.astype(dtype),
        node_i=np.arange(nb, dtype=np.int32), node_j=np.full(nb, -1, dtype=np.int32),
        R=contact_frames(normals).astype(dtype), mu=mus.astype(dtype),
        phi=(gap / h).astype(dtype), v0=v.ravel().astype(dtype), h=h,
        x0=x.ravel(), mass=np.full(3 * N, mass),
        meta=dict(kind="lattice", dims=(nx, ny, nz), spacing=spacing, k=k, c=c,
                  node_mass=mass, gravity=tuple(gravity), terrain=terrain, seed=seed))


# ----------------------------------------------------------------------------
# linear tetrahedral FEM block (config 2)
# ----------------------------------------------------------------------------

def _kuhn_tets():
    """The six tetrahedra of the Kuhn split of the unit cube (corner bit-vectors)."""
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c = np.zeros(3, dtype=np.int64)
        verts = [c.copy()]
        for a in perm:
            c[a] += 1
            verts.append(c.copy())
        tets.append(np.array(verts))
    return tets


def _tet_stiffness(X, E, nu):
    """12x12 linear-elastic stiffness ``V B^T C B`` of a tetrahedron with vertices ``X``."""
    Dm = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    V = abs(np.linalg.det(Dm)) / 6.0
    G = np.linalg.inv(Dm).T           # rows: gradients of N1..N3 are columns of inv(Dm)^T
    grads = np.zeros((4, 3))
    grads[1:] = G.T
    grads[0] = -grads[1:].sum(axis=0)
    B = np.zeros((6, 12))
    for a in range(4):
        gx, gy, gz = grads[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1] = gz
        B[3, 3 * a + 2] = gy
        B[4, 3 * a + 0] = gz
        B[4, 3 * a + 2] = gx
        B[5, 3 * a + 0] = gy
        B[5, 3 * a + 1] = gx
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu_ = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu_
    C[3, 3] = C[4, 4] = C[5, 5] = mu_
    return V * B.T @ C @ B, V


def fem_block_scene(cx=64, cy=64, cz=16, *, seed, spacing=0.01, E=1e5, nu=0.3,
                    rho=1000.0, h=1e-3, mu=0.4, v_sigma=1e-2,
                    gravity=(0.0, 0.0, -GRAVITY), dtype=np.float64):
    """Linear-tet FEM block on the ground plane, ``A = M + h^2 K`` (lumped M)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = cx + 1, cy + 1, cz + 1
    N = nx * ny * nz
    ix, iy, iz = _grid_index(nx, ny, nz)
    offs = _offsets(nx, ny)
    okey = {o: kk for kk, o in enumerate(offs)}
    kz, ky, kx = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    cell_node = (kx + nx * (ky + ny * kz)).ravel()
    diag = np.zeros((N, 3, 3))
    off = [None if o == (0, 0, 0) else np.zeros((N, 3, 3)) for o in offs]
    present = [np.zeros(N, dtype=bool) for _ in offs]
    mass = np.zeros(N)
    for tv in _kuhn_tets():
        Ke, V = _tet_stiffness(tv.astype(np.float64) * spacing, E, nu)
        Ke = h * h * Ke
        for a in range(4):
            ra = cell_node + tv[a][0] + nx * (tv[a][1] + ny * tv[a][2])
            mass[ra] += rho * V / 4.0
            for bb in range(4):
                o = tuple(int(t) for t in (tv[bb] - tv[a]))
                blk = Ke[3 * a:3 * a + 3, 3 * bb:3 * bb + 3]
                if o == (0, 0, 0):
                    diag[ra] += blk
                else:
                    off[okey[o]][ra] += blk
                present[okey[o]][ra] = True
    present[okey[(0, 0, 0)]][:] = True
    diag[:, 0, 0] += mass
    diag[:, 1, 1] += mass
    diag[:, 2, 2] += mass
    row_ptr, col, vals = _compress(nx, ny, nz, diag, off, present, dtype)
    x = np.stack([ix * spacing, iy * spacing, iz * spacing], axis=1).astype(np.float64)
    v = rng.normal(0.0, v_sigma, size=(N, 3))
    g = np.asarray(gravity)
    b = (mass[:, None] * v + h * mass[:, None] * g[None, :]).ravel()
    nb = nx * ny
    normals = np.tile(np.array([0.0, 0.0, 1.0]), (nb, 1))
    return Scene(
        n_nodes=N, row_ptr=row_ptr, col_idx=col, vals=vals, b=b.astype(dtype),
        node_i=np.arange(nb, dtype=np.int32), node_j=np.full(nb, -1, dtype=np.int32),
        R=contact_frames(normals).astype(dtype), mu=np.full(nb, mu, dtype=dtype),
        phi=np.zeros(nb, dtype=dtype), v0=v.ravel().astype(dtype), h=h,
        x0=x.ravel(), mass=np.repeat(mass, 3),
        meta=dict(kind="fem", cells=(cx, cy, cz), E=E, nu=nu, rho=rho, seed=seed))


# ----------------------------------------------------------------------------
# batches of independent scenes (configs 4, 5)
# ----------------------------------------------------------------------------

def tilted_gravity(rng) -> np.ndarray:
    """Gravity tilted by U[0, 30] degrees about a random horizontal axis."""
    tilt = math.radians(rng.uniform(0.0, 30.0))
    az = rng.uniform(0.0, 2 * math.pi)
    axis = np.array([math.cos(az), math.sin(az), 0.0])
    g = np.array([0.0, 0.0, -GRAVITY])
    # Rodrigues rotation of g about the horizontal axis
    return (g * math.cos(tilt) + np.cross(axis, g) * math.sin(tilt)
            + axis * axis.dot(g) * (1 - math.cos(tilt)))


def concat_scenes(scenes, dtype=None) -> Scene:
    """Block-diagonal concatenation of independent scenes (one batched problem)."""
    dtype = dtype or scenes[0].vals.dtype
    node_off = np.zeros(len(scenes) + 1, dtype=np.int64)
    node_off[1:] = np.cumsum([s.n_nodes for s in scenes])
    blk_off = np.zeros(len(scenes) + 1, dtype=np.int64)
    blk_off[1:] = np.cumsum([s.nnzb for s in scenes])
    row_ptr = np.concatenate([s.row_ptr[:-1].astype(np.int64) + blk_off[q]
                              for q, s in enumerate(scenes)] + [blk_off[-1:]])
    col = np.concatenate([s.col_idx.astype(np.int64) + node_off[q] for q, s in enumerate(scenes)])
    cat = lambda name: np.concatenate([getattr(s, name) for s in scenes]).astype(dtype)
    node_i = np.concatenate([s.node_i.astype(np.int64) + node_off[q] for q, s in enumerate(scenes)])
    node_j = np.concatenate([np.where(s.node_j >= 0, s.node_j.astype(np.int64) + node_off[q], -1)
                             for q, s in enumerate(scenes)])
    return Scene(
        n_nodes=int(node_off[-1]), row_ptr=row_ptr.astype(np.int32), col_idx=col.astype(np.int32),
        vals=np.concatenate([s.vals for s in scenes]).astype(dtype), b=cat("b"),
        node_i=node_i.astype(np.int32), node_j=node_j.astype(np.int32), R=cat("R"),
        mu=cat("mu"), phi=cat("phi"), v0=cat("v0"), h=scenes[0].h,
        x0=(np.concatenate([s.x0 for s in scenes])
            if all(s.x0 is not None for s in scenes) else None),
        mass=(np.concatenate([s.mass for s in scenes])
              if all(s.mass is not None for s in scenes) else None),
        scene_ptr=node_off.astype(np.int32),
        meta=dict(kind="batch", n_scenes=len(scenes)))


def batched_lattices(n_scenes, *, seed, side_range=(4, 12), dtype=np.float32,
                     k_scale_range=(0.5, 2.0)):
    """Independent cubic lattices on the ground plane, each with its own side,
    spring stiffness scale, per-contact friction and tilted gravity."""
    rng = np.random.default_rng(seed)
    scenes = []
    for q in range(n_scenes):
        s = int(rng.integers(side_range[0], side_range[1] + 1))
        kscale = float(rng.uniform(*k_scale_range))
        scenes.append(lattice_scene(
            s, s, s, seed=int(rng.integers(0, 2**62)), k=1e3 * kscale,
            gravity=tuple(tilted_gravity(rng)), mu_range=(0.2, 0.8), dtype=dtype))
    return scenes


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def small_lattice(dtype=np.float64) -> Scene:
    """6x6x6 lattice on the ground plane, 648 DOF, 36 contacts, mu = 0.5."""
    return lattice_scene(6, 6, 6, seed=SEED_BASE + 1, mu=0.5, dtype=dtype)


def fem_block(dtype=np.float32, cells=(64, 64, 16)) -> Scene:
    """64x64x16-cell Kuhn-split tetrahedral block, 215,475 DOF, 4,225 contacts."""
    return fem_block_scene(*cells, seed=SEED_BASE + 2, dtype=dtype)


def terrain_lattice(dtype=np.float32, dims=(128, 128, 32)) -> Scene:
    """128x128x32 lattice draped on a sinusoid+noise heightfield, 1,572,864 DOF,
    16,384 contacts with mu ~ U[0.2, 0.8]."""
    return lattice_scene(*dims, seed=SEED_BASE + 3, terrain=True, v_down=0.2,
                         mu_range=(0.2, 0.8), dtype=dtype)


def random_problem(rng, n_nodes, n_contacts, *, density=0.3, d_contacts=0,
                   mu_range=(0.1, 1.0), phi_scale=0.2, dtype=np.float64,
                   couple=1.0) -> Scene:
    """Small random SPD block problem with random contact frames (test input).

    ``A = M + couple * G G^T`` with a random sparse block pattern for ``G``; the
    first ``n_contacts`` distinct nodes carry S-contacts, the next
    ``2 * d_contacts`` nodes pair up into D-contacts.
    """
    n = 3 * n_nodes
    mask = rng.random((n_nodes, n_nodes)) < density
    mask = mask | mask.T
    np.fill_diagonal(mask, True)
    Gm = rng.standard_normal((n, n)) * np.kron(mask, np.ones((3, 3)))
    A = np.diag(rng.uniform(1.0, 2.0, n)) + couple * (Gm @ Gm.T) / n
    pattern = (np.abs(A.reshape(n_nodes, 3, n_nodes, 3)).sum(axis=(1, 3)) > 0)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n_nodes):
        js = np.nonzero(pattern[i])[0]
        row_ptr[i + 1] = row_ptr[i] + len(js)
        cols.extend(js)
        vals.extend(A[3 * i:3 * i + 3, 3 * j:3 * j + 3] for j in js)
    perm = rng.permutation(n_nodes)
    ci = perm[:n_contacts]
    dj = perm[n_contacts:n_contacts + 2 * d_contacts].reshape(-1, 2)
    node_i = np.concatenate([ci, dj[:, 0]]).astype(np.int32)
    node_j = np.concatenate([np.full(n_contacts, -1), dj[:, 1]]).astype(np.int32)
    m = len(node_i)
    v0 = rng.standard_normal(n)
    b = A @ rng.standard_normal(n)
    return Scene(
        n_nodes=n_nodes, row_ptr=row_ptr, col_idx=np.array(cols, dtype=np.int32),
        vals=np.array(vals).reshape(-1, 3, 3).astype(dtype), b=b.astype(dtype),
        node_i=node_i, node_j=node_j, R=random_rotations(rng, m).astype(dtype),
        mu=rng.uniform(*mu_range, size=m).astype(dtype),
        phi=(phi_scale * rng.standard_normal(m)).astype(dtype), v0=v0.astype(dtype),
        meta=dict(kind="random"))


def lattice_batch(n_scenes, *, seed, side_range=(4, 12), mass=1e-3, c=0.1, h=1e-3,
                  k_scale_range=(0.5, 2.0), mu_range=(0.2, 0.8), v_down=0.1, v_sigma=1e-3,
                  spacing=0.01, dtype=np.float32, dims=None) -> Scene:
    """``n_scenes`` independent rest-linearized cubic lattices on the ground plane,
    concatenated into one batched problem (vectorised; same physics as
    :func:`batched_lattices`).

    A rest lattice has ``A = M + (h c + h^2 k) L`` with ``L = sum d d^T`` over
    its springs, so every scene of side s reuses one ``L_s`` scaled by its own
    stiffness.  Per scene: side ``U{side_range}``, ``k = 1e3 * U[k_scale_range]``,
    gravity tilted by U[0, 30] degrees, friction ``mu ~ U[mu_range]`` per contact;
    bottom layer on ``z = 0`` (phi = 0).  ``meta`` carries per-scene arrays
    (side, k, coef = h c + h^2 k, gravity) for dynamics harnesses.  ``dims``
    fixes every scene to ``nx x ny x nz`` nodes instead of random cubes.
    """
    rng = np.random.default_rng(seed)
    if dims is None:
        sides = rng.integers(side_range[0], side_range[1] + 1, size=n_scenes)
        shape = {int(s): (int(s),) * 3 for s in np.unique(sides)}
    else:
        sides = np.zeros(n_scenes, dtype=np.int64)      # one shape, key 0
        shape = {0: tuple(int(d) for d in dims)}
    kk = 1e3 * rng.uniform(*k_scale_range, size=n_scenes)
    grav = np.array([tilted_gravity(rng) for _ in range(n_scenes)])
    coef = h * c + h * h * kk
    tmpl = {}
    for s in np.unique(sides):
        s = int(s)
        nx, ny, nz = shape[s]
        nn = nx * ny * nz
        ix, iy, iz = _grid_index(nx, ny, nz)
        x = np.stack([ix, iy, iz], axis=1) * spacing
        rp, col, L, _ = lattice_system(nx, ny, nz, x, x, np.zeros((nn, 3)), mass=0.0, k=1.0,
                                       c=0.0, h=1.0, gravity=(0, 0, 0), dtype=np.float64)
        diag = np.nonzero(col == np.repeat(np.arange(nn), np.diff(rp)))[0]
        tmpl[s] = (rp, col, L.astype(np.float64), diag, x)
    nodes_of = {s: int(np.prod(shape[s])) for s in shape}
    base_of = {s: shape[s][0] * shape[s][1] for s in shape}
    N_q = np.array([nodes_of[int(s)] for s in sides], dtype=np.int64)
    node_off = np.zeros(n_scenes + 1, dtype=np.int64)
    node_off[1:] = np.cumsum(N_q)
    nnzb_q = np.array([tmpl[int(s)][1].shape[0] for s in sides])
    blk_off = np.zeros(n_scenes + 1, dtype=np.int64)
    blk_off[1:] = np.cumsum(nnzb_q)
    N, nnzb = int(node_off[-1]), int(blk_off[-1])
    row_ptr = np.empty(N + 1, dtype=np.int64)
    col = np.empty(nnzb, dtype=np.int32)
    vals = np.empty((nnzb, 3, 3), dtype=dtype)
    x0 = np.empty((N, 3))
    eye = np.eye(3)
    for s in np.unique(sides):
        s = int(s)
        rp, cl, L, diag, xs = tmpl[s]
        qs = np.nonzero(sides == s)[0]
        nn = nodes_of[s]
        for q in qs:
            n0, b0 = node_off[q], blk_off[q]
            row_ptr[n0:n0 + nn] = rp[:-1] + b0
            col[b0:b0 + cl.shape[0]] = cl + n0
            x0[n0:n0 + nn] = xs
        # values of the whole group at once: coef_q * L + M on the diagonal blocks
        blk = coef[qs][:, None, None, None] * L[None]
        blk[:, diag] += mass * eye
        for r, q in enumerate(qs):
            b0 = blk_off[q]
            vals[b0:b0 + L.shape[0]] = blk[r].astype(dtype)
    row_ptr[N] = nnzb
    v = np.zeros((N, 3))
    v[:, 2] = -v_down
    v += rng.normal(0.0, v_sigma, size=(N, 3))
    scene_of = np.repeat(np.arange(n_scenes), N_q)
    g_node = grav[scene_of]
    b = (mass * v + h * mass * g_node).ravel()
    bottom = np.concatenate([node_off[q] + np.arange(base_of[int(sides[q])])
                             for q in range(n_scenes)])
    n_c = bottom.shape[0]
    R = contact_frames(np.tile([0.0, 0.0, 1.0], (n_c, 1)))
    return Scene(
        n_nodes=N, row_ptr=row_ptr.astype(np.int32), col_idx=col, vals=vals,
        b=b.astype(dtype), node_i=bottom.astype(np.int32),
        node_j=np.full(n_c, -1, dtype=np.int32), R=R.astype(dtype),
        mu=rng.uniform(*mu_range, size=n_c).astype(dtype), phi=np.zeros(n_c, dtype=dtype),
        v0=v.ravel().astype(dtype), h=h, x0=x0.ravel(), mass=np.full(3 * N, mass),
        scene_ptr=node_off.astype(np.int32),
        meta=dict(kind="lattice_batch", sides=sides, nodes=N_q, k=kk, coef=coef, gravity=grav,
                  node_mass=mass, seed=seed, dims=dims))


# ----------------------------------------------------------------------------
# virtual nodes (Sec. III.A, eq. vforce / eq. vnode) and rigid bodies
# ----------------------------------------------------------------------------

def skew(r) -> np.ndarray:
    """Matrix of ``x -> r x x``."""
    return np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])


def add_virtual_nodes(scene: Scene, jv_blocks, n_virtual: int, k_v: float, contacts,
                      v_warm=None) -> Scene:
    """Augment ``A_o v = b_o`` with ``n_virtual`` virtual nodes coupled by the
    viscous force ``f_v = -k_v (J_v v - v_v)`` (eq. vforce):
    ``A = [[A_o + k_v J_v^T J_v, -k_v J_v^T], [-k_v J_v, k_v I]]``,
    ``b = [b_o; 0]`` (eq. vnode).

    ``jv_blocks``: list of ``(p, i, B)`` -- virtual node p takes ``B v_i`` from
    original node i (``J_v`` block row p).  ``contacts``: ``(node_i, node_j, R,
    mu, phi)`` whose node indices may refer to virtual nodes as
    ``scene.n_nodes + p``.  The warm start of a virtual node is ``J_v v``
    (Sec. V.A).  Dense assembly: small systems only.
    """
    No, Nv = scene.n_nodes, n_virtual
    N = No + Nv
    A = np.zeros((3 * N, 3 * N))
    A[:3 * No, :3 * No] = scene.dense_A()
    Jv = np.zeros((3 * Nv, 3 * No))
    for p, i, B in jv_blocks:
        Jv[3 * p:3 * p + 3, 3 * i:3 * i + 3] += B
    A[:3 * No, :3 * No] += k_v * Jv.T @ Jv
    A[:3 * No, 3 * No:] = -k_v * Jv.T
    A[3 * No:, :3 * No] = -k_v * Jv
    A[3 * No:, 3 * No:] = k_v * np.eye(3 * Nv)
    blocks = np.abs(A.reshape(N, 3, N, 3)).sum(axis=(1, 3)) > 0
    row_ptr = np.zeros(N + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(N):
        js = np.nonzero(blocks[i])[0]
        row_ptr[i + 1] = row_ptr[i] + len(js)
        cols.extend(js)
        vals.extend(A[3 * i:3 * i + 3, 3 * j:3 * j + 3] for j in js)
    node_i, node_j, R, mu, phi = contacts
    v_o = np.asarray(scene.v0 if v_warm is None else v_warm, dtype=np.float64)
    v0 = np.concatenate([v_o, Jv @ v_o])
    dt = scene.vals.dtype
    return Scene(
        n_nodes=N, row_ptr=row_ptr, col_idx=np.array(cols, dtype=np.int32),
        vals=np.array(vals).reshape(-1, 3, 3).astype(dt),
        b=np.concatenate([np.asarray(scene.b, float), np.zeros(3 * Nv)]).astype(dt),
        node_i=np.asarray(node_i, dtype=np.int32), node_j=np.asarray(node_j, dtype=np.int32),
        R=np.asarray(R, dtype=dt), mu=np.asarray(mu, dtype=dt), phi=np.asarray(phi, dtype=dt),
        v0=v0.astype(dt), h=scene.h,
        meta=dict(scene.meta, kind="virtual", k_v=k_v, n_original=No, Jv=Jv))


def rigid_boxes(boxes, h=1e-3, gravity=(0.0, 0.0, -GRAVITY), dtype=np.float64):
    """Rigid boxes as two nodes each (linear and angular velocity, 6 DOF), no
    coupling: ``A = diag(m I, I_body)``, ``b = M v + h (m g + F, tau)``
    (backward Euler without gyroscopic terms).  ``boxes``: dicts with ``m``,
    ``size`` (3), ``v`` (6) and optional ``force`` (3, at the centre of mass)."""
    N = 2 * len(boxes)
    vals, b, v0 = [], [], []
    g = np.asarray(gravity, float)
    for bx in boxes:
        m = bx["m"]
        sx, sy, sz = bx["size"]
        Ib = m / 12.0 * np.diag([sy * sy + sz * sz, sx * sx + sz * sz, sx * sx + sy * sy])
        vals += [m * np.eye(3), Ib]
        v = np.asarray(bx["v"], float)
        F = np.asarray(bx.get("force", (0, 0, 0)), float)
        b += [m * v[:3] + h * (m * g + F), Ib @ v[3:]]
        v0 += [v[:3], v[3:]]
    return Scene(
        n_nodes=N, row_ptr=np.arange(N + 1, dtype=np.int32), col_idx=np.arange(N, dtype=np.int32),
        vals=np.array(vals).astype(dtype), b=np.concatenate(b).astype(dtype),
        node_i=np.zeros(0, np.int32), node_j=np.zeros(0, np.int32), R=np.zeros((0, 3, 3), dtype),
        mu=np.zeros(0, dtype), phi=np.zeros(0, dtype), v0=np.concatenate(v0).astype(dtype), h=h,
        meta=dict(kind="rigid", boxes=boxes))


def point_jacobian(body: int, r) -> list:
    """``J_v`` blocks of a point at offset ``r`` from body ``body``'s centre:
    ``v_p = v - [r]x omega``."""
    return [(None, 2 * body, np.eye(3)), (None, 2 * body + 1, -skew(r))]
