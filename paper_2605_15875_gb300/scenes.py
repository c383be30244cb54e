"""Seeded synthetic scene generators.

This module is shared by the FP64 oracle tests and by the CUDA path: it only
builds geometry (meshes, body placements, velocities) from a seed and packs it
into flat arrays.  It holds none of the method's arithmetic: no mass
properties, energies, distances, candidate tests or solver steps.

The scenes stand in for the paper's artist meshes (Sec. 6, Table 1), which are
not available: unit-cube stacks, noisy icospheres (radial factor U[0.9, 1.1]
per vertex), a static open box, and piles over a ground plane.  Gravity is
(0, -9.8, 0) (y up) and density 1000 unless a recipe states otherwise.

Conventions shared with the C ABI:
  * q = (p0, p1, p2, A00, A01, A02, A10, A11, A12, A20, A21, A22): the affine
    map x = A xbar + p with A row-major (Sec. 3, Eq. 1 DoFs).
  * body kind 0 = dynamic, 1 = static, 2 = kinematic.
  * ground planes are axis-aligned: distance = sign * x[axis] - offset.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

KIND_DYNAMIC = 0
KIND_STATIC = 1
KIND_KINEMATIC = 2

IDENTITY_Q = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float64)


@dataclasses.dataclass
class Mesh:
    xbar: np.ndarray  # [V, 3] float64
    tris: np.ndarray  # [T, 3] int32, mesh-local vertex indices


@dataclasses.dataclass
class SceneArrays:
    """Flat arrays in exactly the layout the C ABI and the oracle consume."""

    mesh_n_verts: np.ndarray
    mesh_n_tris: np.ndarray
    mesh_xbar: np.ndarray  # [sum V, 3]
    mesh_tris: np.ndarray  # [sum T, 3]
    body_mesh: np.ndarray
    body_density: np.ndarray
    body_kappa: np.ndarray
    body_kind: np.ndarray
    body_q0: np.ndarray  # [B, 12]
    body_v0: np.ndarray  # [B, 12]
    plane_axis: np.ndarray
    plane_sign: np.ndarray
    plane_offset: np.ndarray
    gravity: np.ndarray  # [3]
    name: str = ""
    body_omega: Optional[np.ndarray] = None  # [B, 3] angular velocity of kinematic bodies

    @property
    def n_bodies(self) -> int:
        return int(self.body_mesh.shape[0])

    @property
    def n_dynamic(self) -> int:
        return int(np.sum(self.body_kind == KIND_DYNAMIC))

    def body_vertex_counts(self) -> np.ndarray:
        return self.mesh_n_verts[self.body_mesh]

    def body_tri_counts(self) -> np.ndarray:
        return self.mesh_n_tris[self.body_mesh]

    def total_tris(self) -> int:
        return int(np.sum(self.body_tri_counts()))

    def mesh(self, m: int) -> Mesh:
        vo = int(np.sum(self.mesh_n_verts[:m]))
        to = int(np.sum(self.mesh_n_tris[:m]))
        return Mesh(self.mesh_xbar[vo:vo + self.mesh_n_verts[m]],
                    self.mesh_tris[to:to + self.mesh_n_tris[m]])

    def world_vertices(self, q: Optional[np.ndarray] = None) -> np.ndarray:
        """Vertex positions x = A xbar + p for every body, mesh frame (no
        centre-of-mass shift), concatenated in body order.  Used only to place
        bodies in the generators and to make test inputs."""
        q = self.body_q0 if q is None else q
        out = []
        for b in range(self.n_bodies):
            m = self.mesh(int(self.body_mesh[b]))
            A = q[b, 3:].reshape(3, 3)
            out.append(m.xbar @ A.T + q[b, :3])
        return np.concatenate(out, axis=0)


def _pack(meshes: Sequence[Mesh], body_mesh, density, kappa, kind, q0, v0,
          planes=(), gravity=(0.0, -9.8, 0.0), name="", omega=None) -> SceneArrays:
    body_mesh = np.asarray(body_mesh, dtype=np.int32)
    B = body_mesh.shape[0]
    q0 = np.asarray(q0, dtype=np.float64).reshape(B, 12)
    v0 = np.zeros((B, 12)) if v0 is None else np.asarray(v0, np.float64).reshape(B, 12)
    planes = list(planes)
    return SceneArrays(
        mesh_n_verts=np.array([m.xbar.shape[0] for m in meshes], dtype=np.int32),
        mesh_n_tris=np.array([m.tris.shape[0] for m in meshes], dtype=np.int32),
        mesh_xbar=np.ascontiguousarray(np.concatenate([m.xbar for m in meshes]), dtype=np.float64),
        mesh_tris=np.ascontiguousarray(np.concatenate([m.tris for m in meshes]), dtype=np.int32),
        body_mesh=body_mesh,
        body_density=np.broadcast_to(np.asarray(density, np.float64), (B,)).copy(),
        body_kappa=np.broadcast_to(np.asarray(kappa, np.float64), (B,)).copy(),
        body_kind=np.broadcast_to(np.asarray(kind, np.int32), (B,)).copy(),
        body_q0=np.ascontiguousarray(q0),
        body_v0=np.ascontiguousarray(v0),
        plane_axis=np.array([p[0] for p in planes], dtype=np.int32),
        plane_sign=np.array([p[1] for p in planes], dtype=np.float64),
        plane_offset=np.array([p[2] for p in planes], dtype=np.float64),
        gravity=np.asarray(gravity, dtype=np.float64),
        name=name,
        body_omega=np.ascontiguousarray(np.zeros((B, 3)) if omega is None
                                        else np.asarray(omega, np.float64).reshape(B, 3)),
    )


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _orient_outward(verts: np.ndarray, tris: np.ndarray, centre) -> np.ndarray:
    tris = tris.copy()
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0 - centre) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def cube_mesh(size: float = 1.0) -> Mesh:
    """Axis-aligned cube centred at the origin: 8 vertices, 12 triangles."""
    h = 0.5 * size
    v = np.array([[x, y, z] for x in (-h, h) for y in (-h, h) for z in (-h, h)], dtype=np.float64)
    # index = 4*ix + 2*iy + iz
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    t = []
    for a, b, c, d in quads:
        t.append((a, b, c))
        t.append((a, c, d))
    tris = _orient_outward(v, np.array(t, dtype=np.int32), np.zeros(3))
    return Mesh(v, tris.astype(np.int32))


def box_mesh(ex: float, ey: float, ez: float) -> Mesh:
    """Closed axis-aligned box centred at the origin with extents ex, ey, ez."""
    c = cube_mesh(1.0)
    return Mesh(c.xbar * np.array([ex, ey, ez]), c.tris.copy())


def icosphere(level: int) -> Mesh:
    """Unit icosphere: 12/42/162/642 vertices for levels 0..3."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0),
         (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi),
         (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    T = _orient_outward(V, np.array(faces, dtype=np.int32), np.zeros(3))
    return Mesh(V, T.astype(np.int32))


def noisy_icosphere(rng: np.random.Generator, level: int, radius: float,
                    lo: float = 0.9, hi: float = 1.1) -> Mesh:
    """Icosphere of the given radius with a per-vertex radial factor U[lo, hi]."""
    m = icosphere(level)
    f = rng.uniform(lo, hi, size=(m.xbar.shape[0], 1))
    return Mesh(m.xbar * radius * f, m.tris.copy())


def open_box_mesh(ex: float, ey: float, ez: float) -> Mesh:
    """Static open box (floor + 4 walls, no lid): 8 vertices, 10 triangles.
    Floor at y = 0, inner extent ex x ey x ez centred on the y axis."""
    hx, hz = 0.5 * ex, 0.5 * ez
    v = np.array([[-hx, 0, -hz], [hx, 0, -hz], [hx, 0, hz], [-hx, 0, hz],
                  [-hx, ey, -hz], [hx, ey, -hz], [hx, ey, hz], [-hx, ey, hz]], dtype=np.float64)
    quads = [(0, 1, 2, 3), (0, 4, 5, 1), (1, 5, 6, 2), (2, 6, 7, 3), (3, 7, 4, 0)]
    t = []
    for a, b, c, d in quads:
        t += [(a, b, c), (a, c, d)]
    return Mesh(v, np.array(t, dtype=np.int32))


# --------------------------------------------------------------------------
# scene recipes
# --------------------------------------------------------------------------

def _q_at(p) -> np.ndarray:
    q = IDENTITY_Q.copy()
    q[:3] = p
    return q


def cube_stack(seed: int = 0, nx: int = 2, ny: int = 2, nz: int = 2, spacing: float = 1.01,
               bottom_gap: float = 0.01, jitter: float = 1e-3, density: float = 1000.0,
               kappa: float = 1e8, ground: bool = True) -> SceneArrays:
    """Unit cubes (8 v / 12 t) in an nx x ny x nz stack, centres `spacing`
    apart, bottom layer `bottom_gap` above the plane y = 0, each position
    jittered by U[-jitter, jitter]^3.  The 2x2x2 default is the small
    single-partition stacking workload."""
    rng = np.random.default_rng(seed)
    mesh = cube_mesh(1.0)
    q0 = []
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                c = np.array([(ix - (nx - 1) / 2) * spacing,
                              0.5 + bottom_gap + iy * spacing,
                              (iz - (nz - 1) / 2) * spacing])
                q0.append(_q_at(c + rng.uniform(-jitter, jitter, 3)))
    B = len(q0)
    planes = [(1, 1.0, 0.0)] if ground else []
    return _pack([mesh], [0] * B, density, kappa, KIND_DYNAMIC, q0, None, planes,
                 name=f"cube_stack_{nx}x{ny}x{nz}")


def colliding_pair(size: float = 0.2) -> SceneArrays:
    """Two cubes of edge `size` and densities 1000 and 3000 flying at each
    other without gravity or planes (velocities (2, 0, 0) and (-1, 0.3, 0)),
    the second offset by (0.05, 0.02) across the line of approach so that the
    impact is off-centre: only contact forces act, and they are internal."""
    q0 = [_q_at([-0.75 * size, 0.0, 0.0]), _q_at([0.75 * size, 0.25 * size, 0.1 * size])]
    v0 = np.zeros((2, 12))
    v0[0, :3] = [2.0, 0.0, 0.0]
    v0[1, :3] = [-1.0, 0.3, 0.0]
    return _pack([cube_mesh(size)], [0, 0], [1000.0, 3000.0], 1e8, KIND_DYNAMIC, q0, v0, [],
                 gravity=(0.0, 0.0, 0.0), name="colliding_pair")


def static_only(gap: float = 5e-4) -> SceneArrays:
    """Degenerate scene without unknowns: two static unit cubes side by side,
    `gap` apart (inside the usual activation distance), 0.1 above the ground
    plane y = 0.  Pairs of static bodies are never candidates, so a step has
    nothing to solve."""
    q0 = [_q_at([-0.5 - 0.5 * gap, 0.6, 0.0]), _q_at([0.5 + 0.5 * gap, 0.6, 0.0])]
    return _pack([cube_mesh(1.0)], [0, 0], 1000.0, 1e8, KIND_STATIC, q0, None, [(1, 1.0, 0.0)],
                 name="static_only")


def sphere_grid_in_box(seed: int = 0, n: int = 8, level: int = 2, radius: float = 0.1,
                       spacing: float = 0.25, lowest: float = 0.3, box=(2.4, 3.0, 2.4),
                       density: float = 1000.0, kappa: float = 1e8, ny: Optional[int] = None,
                       nz: Optional[int] = None) -> SceneArrays:
    """n x ny x nz noisy icospheres (distinct mesh per body) on a grid with the
    given spacing, lowest centre `lowest` above the floor of a static open box.
    The 8x8x8, level-2, r = 0.1 default is the 512-body slab-partition
    workload."""
    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    meshes, q0 = [], []
    for ix in range(n):
        for iy in range(ny):
            for iz in range(nz):
                meshes.append(noisy_icosphere(rng, level, radius))
                q0.append(_q_at([(ix - (n - 1) / 2) * spacing, lowest + iy * spacing,
                                 (iz - (nz - 1) / 2) * spacing]))
    B = len(q0)
    meshes.append(open_box_mesh(*box))
    body_mesh = list(range(B)) + [B]
    q0.append(IDENTITY_Q.copy())
    kind = [KIND_DYNAMIC] * B + [KIND_STATIC]
    return _pack(meshes, body_mesh, density, kappa, kind, q0, None, [],
                 name=f"sphere_grid_{n}x{ny}x{nz}_L{level}")


def mesh_volume(m: Mesh) -> float:
    """Enclosed volume of a closed, outward-oriented triangle mesh (sum of
    signed tetrahedra against the origin)."""
    a, b, c = (m.xbar[m.tris[:, k]] for k in range(3))
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


# (mass, orthogonality stiffness) of the three groups of the heterogeneity
# experiment (Sec. 6.2, Table 2), and of its uniform baseline
HETERO_GROUPS = ((1.0, 1e8), (100.0, 1e10), (1e4, 1e12))
UNIFORM_GROUP = (100.0, 1e10)


def heterogeneous_pile(seed: int = 0, nx: int = 5, ny: int = 8, nz: int = 5, hetero: bool = True,
                       level: int = 1, radius: float = 0.1, spacing: float = 0.25, lowest: float = 0.15,
                       box=(2.4, 3.0, 2.4)) -> SceneArrays:
    """Material-heterogeneity workload (Sec. 6.2, Table 2): nx*ny*nz noisy
    icospheres (200 by default) on a grid in a static open box, split into
    three groups by a seeded shuffle, group g having body mass m_g and
    orthogonality stiffness kappa_g = E_g from HETERO_GROUPS; with
    hetero=False every body takes UNIFORM_GROUP.  Each body's density is
    m_g / (its own mesh volume), so its mass is m_g exactly."""
    rng = np.random.default_rng(seed)
    B = nx * ny * nz
    meshes, q0 = [], []
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                meshes.append(noisy_icosphere(rng, level, radius))
                q0.append(_q_at([(ix - (nx - 1) / 2) * spacing, lowest + iy * spacing,
                                 (iz - (nz - 1) / 2) * spacing]))
    group = np.empty(B, dtype=np.int32)
    group[rng.permutation(B)] = np.arange(B) % 3
    mk = np.array([HETERO_GROUPS[g] if hetero else UNIFORM_GROUP for g in group])
    density = mk[:, 0] / np.array([mesh_volume(m) for m in meshes])
    meshes.append(open_box_mesh(*box))
    q0.append(IDENTITY_Q.copy())
    kind = [KIND_DYNAMIC] * B + [KIND_STATIC]
    sa = _pack(meshes, list(range(B)) + [B], np.append(density, 1000.0), np.append(mk[:, 1], 1e8),
               kind, q0, None, [], name=f"hetero_pile_{B}" if hetero else f"uniform_pile_{B}")
    sa.body_group = group
    return sa


def random_pile(seed: int, n_bodies: int, levels=(1, 2, 3), radius: float = 0.05,
                density_range=(1e2, 1e4), kappa: float = 1e8, cell: float = 1.2) -> SceneArrays:
    """Loose random pile of noisy icospheres over a ground plane: bodies on a
    jittered lattice of cells `cell * 2r` wide, one density per scene drawn
    log-uniform from `density_range`, mesh level uniform over `levels`."""
    rng = np.random.default_rng(seed)
    side = max(1, int(math.ceil(n_bodies ** (1.0 / 3.0))))
    pitch = cell * 2.0 * radius * 1.1 * 1.05
    rho = float(math.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1]))))
    meshes, q0 = [], []
    for k in range(n_bodies):
        ix, iy, iz = k % side, (k // side) % side, k // (side * side)
        lvl = int(levels[rng.integers(0, len(levels))])
        meshes.append(noisy_icosphere(rng, lvl, radius))
        c = np.array([(ix - (side - 1) / 2) * pitch, radius * 1.2 + 0.01 + iy * pitch,
                      (iz - (side - 1) / 2) * pitch])
        c += rng.uniform(-0.05, 0.05, 3) * radius
        q0.append(_q_at(c))
    return _pack(meshes, list(range(n_bodies)), rho, kappa, KIND_DYNAMIC, q0, None,
                 [(1, 1.0, 0.0)], name=f"pile_{n_bodies}")


def two_body_free_flight(seed: int = 0, gap: float = 0.5) -> SceneArrays:
    """Two unit cubes far apart with initial velocities and no ground: the
    free-flight workload (no contact)."""
    rng = np.random.default_rng(seed)
    mesh = cube_mesh(1.0)
    q0 = [_q_at([-0.5 - gap, 2.0, 0.0]), _q_at([0.5 + gap, 2.0, 0.0])]
    v0 = np.zeros((2, 12))
    v0[:, :3] = rng.uniform(-1.0, 1.0, (2, 3))
    return _pack([mesh], [0, 0], 1000.0, 1e8, KIND_DYNAMIC, q0, v0, [], name="free_flight")


def log_uniform_sizes(rng: np.random.Generator, n: int, lo: int, hi: int) -> np.ndarray:
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(np.int64)


def batched_subdomains(seed: int = 0, n_scenes: int = 64, lo: int = 16, hi: int = 2048,
                       levels=(1, 2, 3)) -> List[SceneArrays]:
    """Independent subdomains with body counts log-uniform in [lo, hi], each a
    random-density pile over a ground plane (the uneven-batch workload)."""
    rng = np.random.default_rng(seed)
    sizes = log_uniform_sizes(rng, n_scenes, lo, hi)
    return [random_pile(int(seed * 1000 + i), int(s), levels=levels) for i, s in enumerate(sizes)]


def serving_requests(seed: int = 0, n_scenes: int = 256, lo: int = 8, hi: int = 4096):
    """Serving workload: independent scenes (half cube stacks, half sphere
    piles) with log-uniform sizes, and the number of steps each request
    advances, U{1..10}.  Returns a list of (SceneArrays, n_steps)."""
    rng = np.random.default_rng(seed)
    sizes = log_uniform_sizes(rng, n_scenes, lo, hi)
    out = []
    for i, s in enumerate(sizes):
        steps = int(rng.integers(1, 11))
        if i % 2 == 0:
            k = max(1, int(round(float(s) ** (1.0 / 3.0))))
            sc = cube_stack(seed=int(seed * 1000 + i), nx=k, ny=max(1, int(s) // (k * k)), nz=k)
        else:
            sc = random_pile(int(seed * 1000 + i), int(s), levels=(1, 2))
        out.append((sc, steps))
    return out


def kinematic_sweeper(seed: int = 0, n_cubes: int = 3, omega: float = 2.0, size: float = 0.1,
                      gap: float = 0.002, density: float = 1000.0, kappa: float = 1e8) -> SceneArrays:
    """A kinematic bar (1.0 x 0.1 x 0.1, centre 0.11 above the ground plane
    y = 0) spinning about the vertical axis through its centre at `omega`
    rad/s (which turns its +x end toward -z), and `n_cubes` dynamic cubes
    resting `gap` above the plane in its sweep (radius 0.35, 0.5 + 0.5 i rad
    ahead of the bar), positions jittered U[+-1e-3]: frictionless
    kinematic-dynamic contact."""
    rng = np.random.default_rng(seed)
    meshes = [box_mesh(1.0, 0.1, 0.1), cube_mesh(size)]
    body_mesh, kind, q0, om = [0], [KIND_KINEMATIC], [_q_at([0.0, 0.11, 0.0])], [[0.0, omega, 0.0]]
    for i in range(n_cubes):
        r, a = 0.35, 0.5 + 0.5 * i
        c = np.array([r * math.cos(a), 0.5 * size + gap, -r * math.sin(a)])
        c += rng.uniform(-1e-3, 1e-3, 3) * np.array([1.0, 0.0, 1.0])
        body_mesh.append(1)
        kind.append(KIND_DYNAMIC)
        q0.append(_q_at(c))
        om.append([0.0, 0.0, 0.0])
    return _pack(meshes, body_mesh, density, kappa, np.array(kind, dtype=np.int32), q0, None,
                 [(1, 1.0, 0.0)], name="kinematic_sweeper", omega=np.array(om))


def perforated_disk_mesh(radius: float = 1.4, thickness: float = 0.05, cell: float = 0.07,
                         hole_radius: float = 0.09, rings: int = 3) -> Mesh:
    """Closed perforated turntable: the square cells of side `cell` whose
    centres lie inside the disk and outside every hole, extruded to
    `thickness` (centred on y = 0), as one watertight outward mesh (caps of
    every kept cell, walls wherever a kept cell meets a dropped one).  Holes:
    1 + 6 + 12 + ... centres of a hexagonal pattern with `rings` rings (37 for
    3 rings) spaced to fill the disk.  Volume = kept cells x cell^2 x thickness."""
    n = int(math.ceil(radius / cell))
    pitch = (radius - hole_radius) / (rings + 0.5)
    holes = [(0.0, 0.0)]
    for r in range(1, rings + 1):
        for k in range(6):
            a0, a1 = math.pi / 3 * k, math.pi / 3 * (k + 1)
            p0 = np.array([math.cos(a0), math.sin(a0)]) * r * pitch
            p1 = np.array([math.cos(a1), math.sin(a1)]) * r * pitch
            for j in range(r):
                holes.append(tuple(p0 + (p1 - p0) * j / r))
    holes = np.array(holes)

    def kept(i, j):
        if not (-n <= i < n and -n <= j < n):
            return False
        cx, cz = (i + 0.5) * cell, (j + 0.5) * cell
        if cx * cx + cz * cz > radius * radius:
            return False
        return bool(np.min((holes[:, 0] - cx) ** 2 + (holes[:, 1] - cz) ** 2) > hole_radius ** 2)

    keep = {(i, j) for i in range(-n, n) for j in range(-n, n) if kept(i, j)}
    vid, verts, tris = {}, [], []
    h = 0.5 * thickness

    def v(i, j, top):
        key = (i, j, top)
        if key not in vid:
            vid[key] = len(verts)
            verts.append((i * cell, h if top else -h, j * cell))
        return vid[key]

    def quad(a, b, c, d, normal):
        for t in ((a, b, c), (a, c, d)):
            p = [np.array(verts[x]) for x in t]
            if np.dot(np.cross(p[1] - p[0], p[2] - p[0]), normal) < 0:
                t = (t[0], t[2], t[1])
            tris.append(t)

    for (i, j) in sorted(keep):
        quad(v(i, j, 1), v(i + 1, j, 1), v(i + 1, j + 1, 1), v(i, j + 1, 1), (0, 1, 0))
        quad(v(i, j, 0), v(i + 1, j, 0), v(i + 1, j + 1, 0), v(i, j + 1, 0), (0, -1, 0))
        if (i - 1, j) not in keep:
            quad(v(i, j, 0), v(i, j + 1, 0), v(i, j + 1, 1), v(i, j, 1), (-1, 0, 0))
        if (i + 1, j) not in keep:
            quad(v(i + 1, j, 0), v(i + 1, j + 1, 0), v(i + 1, j + 1, 1), v(i + 1, j, 1), (1, 0, 0))
        if (i, j - 1) not in keep:
            quad(v(i, j, 0), v(i + 1, j, 0), v(i + 1, j, 1), v(i, j, 1), (0, 0, -1))
        if (i, j + 1) not in keep:
            quad(v(i, j + 1, 0), v(i + 1, j + 1, 0), v(i + 1, j + 1, 1), v(i, j + 1, 1), (0, 0, 1))
    m = Mesh(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32))
    m.n_cells = len(keep)  # kept cells, for the volume closed form
    return m


def funnel_mesh(top_radius: float = 1.5, neck_radius: float = 0.35, top_y: float = 3.4, neck_y: float = 2.2,
                segments: int = 48) -> Mesh:
    """Static open funnel: the lateral surface of a truncated cone from the
    neck ring (neck_y, neck_radius) to the top ring (top_y, top_radius)."""
    verts, tris = [], []
    for k in range(segments):
        a = 2.0 * math.pi * k / segments
        verts.append((neck_radius * math.cos(a), neck_y, neck_radius * math.sin(a)))
        verts.append((top_radius * math.cos(a), top_y, top_radius * math.sin(a)))
    for k in range(segments):
        a0, a1, b0, b1 = 2 * k, 2 * ((k + 1) % segments), 2 * k + 1, 2 * ((k + 1) % segments) + 1
        tris.append((a0, a1, b1))
        tris.append((a0, b1, b0))
    return Mesh(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32))


def funnel_scene(seed: int = 0, n_bodies: int = 5000, level: int = 3, radius: float = 0.05,
                 omega: float = 1.0, density: float = 1000.0, kappa: float = 1e8,
                 dense: bool = False) -> SceneArrays:
    """Funnel-and-turntables workload: `n_bodies` noisy icospheres (radial
    factor U[0.9, 1.1]) on a jittered lattice inside radius 1.25 above a
    static open funnel (top radius 1.5 at y = 3.4, neck radius 0.35 at
    y = 2.2, 48 segments), falling into a static open chamber 3 x 2 x 3 with
    two kinematic perforated turntables (radius 1.4, 37 holes) at y = 0.6 and
    y = 1.3 turning at +omega and -omega about the vertical axis.

    dense=True starts the bodies packed instead: a lattice of pitch
    2.2 r + 2 mm (jitter +-0.5 mm) filling the funnel from its neck upward,
    each body at least 0.08 from the cone along the radius (about 2 mm of
    clearance normal to the wall), then the cylinder of radius 1.25 above
    the funnel: bodies reach the funnel wall and one another within a few
    steps, the dense contact state the free drop reaches only after it has
    fallen into the funnel."""
    if dense:
        return _funnel_dense(seed, n_bodies, level, radius, omega, density, kappa)
    rng = np.random.default_rng(seed)
    meshes = [open_box_mesh(3.0, 2.0, 3.0), funnel_mesh(), perforated_disk_mesh()]
    body_mesh = [0, 1, 2, 2]
    kind = [KIND_STATIC, KIND_STATIC, KIND_KINEMATIC, KIND_KINEMATIC]
    q0 = [_q_at([0.0, 0.0, 0.0]), _q_at([0.0, 0.0, 0.0]), _q_at([0.0, 0.6, 0.0]), _q_at([0.0, 1.3, 0.0])]
    om = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, omega, 0.0], [0.0, -omega, 0.0]]
    pitch = 2.0 * radius * 1.1 * 1.15
    per_layer = [(ix, iz) for ix in range(-12, 13) for iz in range(-12, 13)
                 if (ix * pitch) ** 2 + (iz * pitch) ** 2 <= 1.25 ** 2]
    for k in range(n_bodies):
        ix, iz = per_layer[k % len(per_layer)]
        layer = k // len(per_layer)
        c = np.array([ix * pitch, 3.5 + radius * 1.2 + layer * pitch, iz * pitch])
        c += rng.uniform(-0.05, 0.05, 3) * radius
        meshes.append(noisy_icosphere(rng, level, radius))
        body_mesh.append(len(meshes) - 1)
        kind.append(KIND_DYNAMIC)
        q0.append(_q_at(c))
        om.append([0.0, 0.0, 0.0])
    return _pack(meshes, body_mesh, density, kappa, np.array(kind, dtype=np.int32), q0, None, [],
                 name=f"funnel_{n_bodies}", omega=np.array(om))


def _funnel_dense(seed, n_bodies, level, radius, omega, density, kappa) -> SceneArrays:
    rng = np.random.default_rng(seed)
    meshes = [open_box_mesh(3.0, 2.0, 3.0), funnel_mesh(), perforated_disk_mesh()]
    body_mesh = [0, 1, 2, 2]
    kind = [KIND_STATIC, KIND_STATIC, KIND_KINEMATIC, KIND_KINEMATIC]
    q0 = [_q_at([0.0, 0.0, 0.0]), _q_at([0.0, 0.0, 0.0]), _q_at([0.0, 0.6, 0.0]), _q_at([0.0, 1.3, 0.0])]
    om = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, omega, 0.0], [0.0, -omega, 0.0]]
    pitch = 2.2 * radius + 0.002
    neck_r, neck_y, top_r, top_y = 0.35, 2.2, 1.5, 3.4

    def limit(y):
        if y <= top_y:
            return neck_r + (y - neck_y) * (top_r - neck_r) / (top_y - neck_y) - 0.08
        return 1.25
    n, layer = 0, 0
    while n < n_bodies:
        y = neck_y + 1.2 * radius + layer * pitch
        lim = limit(y)
        m = int(lim / pitch) + 1
        for ix in range(-m, m + 1):
            for iz in range(-m, m + 1):
                x, z = ix * pitch, iz * pitch
                if n >= n_bodies or x * x + z * z > lim * lim:
                    continue
                c = np.array([x, y, z]) + rng.uniform(-5e-4, 5e-4, 3)
                meshes.append(noisy_icosphere(rng, level, radius))
                body_mesh.append(len(meshes) - 1)
                kind.append(KIND_DYNAMIC)
                q0.append(_q_at(c))
                om.append([0.0, 0.0, 0.0])
                n += 1
        layer += 1
    return _pack(meshes, body_mesh, density, kappa, np.array(kind, dtype=np.int32), q0, None, [],
                 name=f"funnel_dense_{n_bodies}", omega=np.array(om))
