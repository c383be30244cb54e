"""The seeded input generators against the recipe they state: mesh counts
and watertight outward orientation, noise ranges, layouts, sizes and body
counts of the workloads, and non-overlapping starts.  CPU only; no method
arithmetic is involved."""
import math
from collections import Counter

import numpy as np
import pytest

from paper_2605_15875_gb300 import scenes


def _edges(tris):
    d = Counter()
    for a, b, c in tris:
        for u, v in ((a, b), (b, c), (c, a)):
            d[(int(u), int(v))] += 1
    return d


def _closed_and_outward(m):
    """Every directed edge once and its reverse once (a closed, consistently
    oriented 2-manifold) and a positive enclosed volume."""
    d = _edges(m.tris)
    assert all(n == 1 for n in d.values())
    assert all(d[(v, u)] == 1 for (u, v) in d)
    x = m.xbar[m.tris]
    vol = np.einsum("ij,ij->i", x[:, 0], np.cross(x[:, 1], x[:, 2])).sum() / 6.0
    assert vol > 0
    return vol, len(d) // 2


@pytest.mark.parametrize("level,V,T", [(1, 42, 80), (2, 162, 320), (3, 642, 1280)])
def test_icosphere_counts_and_topology(level, V, T):
    m = scenes.icosphere(level)
    assert m.xbar.shape == (V, 3) and m.tris.shape == (T, 3)
    vol, E = _closed_and_outward(m)
    assert E == 3 * T // 2 and V - E + T == 2  # sphere: Euler characteristic 2
    assert np.allclose(np.linalg.norm(m.xbar, axis=1), 1.0, atol=1e-15)
    assert vol < 4.0 / 3.0 * math.pi


def test_noisy_icosphere_radial_factor():
    rng = np.random.default_rng(5)
    m = scenes.noisy_icosphere(rng, 2, 0.1)
    r = np.linalg.norm(m.xbar, axis=1) / 0.1
    assert r.min() >= 0.9 and r.max() <= 1.1 and r.std() > 0.04  # U[0.9, 1.1] per vertex
    _closed_and_outward(m)


def test_cube_and_boxes():
    _closed_and_outward(scenes.cube_mesh(1.0))
    b = scenes.open_box_mesh(2.4, 3.0, 2.4)
    assert b.xbar.shape == (8, 3) and b.tris.shape == (10, 3)
    assert b.xbar[:, 1].min() == 0.0  # floor at y = 0


def test_benchmark_workload_layout():
    """512 level-2 noisy icospheres (distinct meshes), 8 x 8 x 8 at spacing
    0.25, lowest centre 0.3 above the floor of the static open box."""
    sa = scenes.sphere_grid_in_box(seed=0)
    assert sa.n_bodies == 513 and sa.n_dynamic == 512
    assert sa.total_tris() == 512 * 320 + 10
    dyn = sa.body_kind == scenes.KIND_DYNAMIC
    assert len(set(int(m) for m in sa.body_mesh[dyn])) == 512
    p = sa.body_q0[dyn, :3]
    for k in range(3):
        u = np.unique(np.round(p[:, k], 12))
        assert len(u) == 8 and np.allclose(np.diff(u), 0.25)
    assert abs(p[:, 1].min() - 0.3) < 1e-12
    assert np.all(sa.body_v0 == 0) and sa.gravity.tolist() == [0.0, -9.8, 0.0]
    # spheres of radius <= 0.11 at spacing 0.25 cannot touch
    assert 0.25 > 2 * 0.1 * 1.1


def test_cube_stack_recipe():
    sa = scenes.cube_stack()
    p = sa.body_q0[:, :3]
    assert sa.n_bodies == 8 and len(sa.plane_offset) == 1
    ideal = np.array([[(ix - 0.5) * 1.01, 0.51 + iy * 1.01, (iz - 0.5) * 1.01]
                      for ix in range(2) for iy in range(2) for iz in range(2)])
    assert np.abs(p - ideal).max() <= 1e-3 and np.abs(p - ideal).max() > 0  # jitter U[-1e-3, 1e-3]^3


def test_serving_and_batched_workloads():
    reqs = scenes.serving_requests(seed=0, n_scenes=12, lo=8, hi=64)
    for i, (sa, k) in enumerate(reqs):
        assert 1 <= k <= 10
        assert (sa.name.startswith("cube_stack")) == (i % 2 == 0)
        assert 1 <= sa.n_dynamic <= 64
    subs = scenes.batched_subdomains(seed=0, n_scenes=6, lo=16, hi=64, levels=(1, 2))
    for sa in subs:
        assert 16 <= sa.n_dynamic <= 64
        rho = np.unique(sa.body_density)
        assert len(rho) == 1 and 1e2 <= rho[0] <= 1e4  # one density per subdomain
        per_body = sa.mesh_n_tris[sa.body_mesh]
        assert set(per_body.tolist()) <= {80, 320}


def test_random_pile_starts_apart():
    sa = scenes.random_pile(3, 27, levels=(1, 2))
    c = sa.body_q0[:, :3]
    r = max(np.linalg.norm(sa.mesh(int(m)).xbar, axis=1).max() for m in sa.body_mesh)
    d = np.linalg.norm(c[:, None] - c[None], axis=2) + np.eye(len(c)) * 1e9
    assert d.min() > 2 * r
    assert (c[:, 1] - r).min() > 0  # above the ground plane y = 0


def test_funnel_crop_layout():
    """The funnel workload's statics, kinematic turntables and sphere lattice
    (a crop of 30 bodies; the full 5000-body scene has 6.41 M triangles)."""
    sa = scenes.funnel_scene(n_bodies=30, level=1)
    kinds = sa.body_kind.tolist()
    assert kinds[:4] == [scenes.KIND_STATIC, scenes.KIND_STATIC, scenes.KIND_KINEMATIC, scenes.KIND_KINEMATIC]
    assert sa.n_dynamic == 30
    assert sa.body_omega[2].tolist() == [0.0, 1.0, 0.0] and sa.body_omega[3].tolist() == [0.0, -1.0, 0.0]
    assert [sa.body_q0[b, 1] for b in (2, 3)] == [0.6, 1.3]
    disk = sa.mesh(int(sa.body_mesh[2]))
    _closed_and_outward(disk)
    # square cells of side 0.07 whose centres lie inside radius 1.4
    assert 1.4 < np.linalg.norm(disk.xbar[:, [0, 2]], axis=1).max() <= 1.4 + 0.07 / math.sqrt(2)
    c = sa.body_q0[4:, :3]
    assert np.linalg.norm(c[:, [0, 2]], axis=1).max() <= 1.25 + 0.05 * 0.05 * 2
    assert c[:, 1].min() > 3.4  # above the funnel's rim
    full_tris = 5000 * 1280 + sum(int(sa.mesh_n_tris[int(sa.body_mesh[b])]) for b in range(4))
    assert full_tris == pytest.approx(6.41e6, rel=2e-3)
