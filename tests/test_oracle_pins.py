"""Pins of the FP64 CPU oracle against things other than itself: closed forms,
finite differences, brute-force sampling and enumeration, numpy's eigh,
textbook special cases and invariants.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_15875_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def fd_grad(f, x, h=1e-7):
    g = np.zeros_like(x)
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


# --------------------------------------------------------------------------- O1

def test_unit_cube_mass_closed_form():
    m = scenes.cube_mesh(1.0)
    mass, com, S, V = O.mass_properties(m.xbar, m.tris, 1000.0)
    assert abs(V - 1.0) < 1e-14 and abs(mass - 1000.0) < 1e-11
    assert np.abs(com).max() < 1e-15
    assert np.allclose(S, np.eye(3) * 1000.0 / 12.0, rtol=0, atol=1e-11)


def test_mass_translation_and_scaling():
    m = scenes.cube_mesh(2.0)
    shift = np.array([0.3, -1.2, 5.0])
    mass, com, S, V = O.mass_properties(m.xbar + shift, m.tris, 7.0)
    assert abs(V - 8.0) < 1e-12
    assert np.allclose(com, shift, atol=1e-13)
    # second moment about the centre: rho * a^5 / 12 for an a-cube
    assert np.allclose(S, np.eye(3) * 7.0 * 32.0 / 12.0, atol=1e-11)


def test_icosphere_volume_converges_to_sphere():
    errs = []
    for lvl in range(4):
        m = scenes.icosphere(lvl)
        _, com, S, V = O.mass_properties(m.xbar * 0.1, m.tris, 1000.0)
        errs.append(abs(V - 4.0 / 3.0 * math.pi * 1e-3) / (4.0 / 3.0 * math.pi * 1e-3))
        assert np.abs(com).max() < 1e-15
        # solid sphere: S = (2/5) m r^2 / 2 * I per axis ... int x^2 dm = m r^2 / 5
        if lvl == 3:
            assert np.allclose(S, np.eye(3) * 1000.0 * V * 0.01 / 5.0, rtol=0.02)
    assert all(errs[i + 1] < errs[i] for i in range(3)) and errs[-1] < 0.01


def test_mass_spectral_bound_holds_for_workloads():
    """lambda_max(M) <= m (Sec. 4.3) requires lambda_max(S) <= m: true for sub-metre bodies."""
    for sa in (scenes.cube_stack(), scenes.sphere_grid_in_box(n=2)):
        sc = O.Scene(sa)
        for b in range(sa.n_bodies):
            if sa.body_kind[b] != 0:
                continue
            m, _, S, _ = sc.body_props(b)
            assert np.linalg.eigvalsh(S).max() <= m


# --------------------------------------------------------------------------- O2

def test_free_fall_closed_form():
    sa = scenes.two_body_free_flight(seed=3)
    sc = O.Scene(sa)
    q0, v0 = sc.state()
    p = O.default_params()
    g, h = sa.gravity, 1e-2
    for n in range(1, 11):
        st = sc.step(p)
        q, v = sc.state()
        pred = q0[:, :3] + n * h * v0[:, :3] + h * h * g * n * (n + 1) / 2
        assert np.abs(q[:, :3] - pred).max() < 1e-12
        assert np.abs(q[:, 3:] - q0[:, 3:]).max() == 0.0
        assert st["status"] == 0 and st["admm_iters"] == 1


@pytest.mark.parametrize("slabs", [1, 2])
def test_collision_conserves_linear_momentum(slabs):
    """Without gravity or planes only contact forces act, and they are
    internal: the barrier of Eq. 1 depends on relative positions, the
    orthogonality term on A alone, so the implicit-Euler step conserves
    sum_b m_b dp_b/dt up to the Newton tolerance.  An off-centre impact of two
    unequal cubes changes both velocities (and spins the bodies) while the
    total momentum stays put; a contact force applied to one side only, or
    mapped through a wrong J^T on the translation part, fails."""
    sa = scenes.colliding_pair()
    sc = O.Scene(sa)
    m = np.array([sc.body_props(b)[0] for b in range(2)])
    q0, v0 = sc.state()
    P0 = (m[:, None] * v0[:, :3]).sum(0)
    p = O.default_params(n_slabs=slabs, axis=0, kappa_barrier=1e3)
    active = 0
    for _ in range(12):
        st = sc.step(p)
        assert st["status"] == 0 and st["min_distance"] > 0
        active = max(active, st["n_active_peak"])
        q, v = sc.state()
        P = (m[:, None] * v[:, :3]).sum(0)
        assert np.abs(P - P0).max() <= 1e-12 * np.abs(P0).max()
    assert active > 0
    assert np.abs(v[:, :3] - v0[:, :3]).min() > 0.05 or np.abs(v[0, :3] - v0[0, :3]).max() > 1.0
    assert np.abs(q[:, 3:] - q0[:, 3:]).max() > 1e-4  # the off-centre hit rotates the bodies


def test_frictionless_plane_keeps_tangential_velocity():
    """Eq. 1 has no friction term and a ground-plane contact acts along the
    plane's normal only: a cube landing on y = 0 while sliding at (0.5, 0.3)
    in x and z keeps those velocities to rounding while its vertical
    velocity goes to zero (a plane gradient leaking into another axis, or any
    tangential drag, fails)."""
    sa = scenes.cube_stack(nx=1, ny=1, nz=1, jitter=0.0)
    v = np.zeros((1, 12))
    v[0, 0], v[0, 2] = 0.5, 0.3
    sa.body_v0 = np.ascontiguousarray(v)
    sc = O.Scene(sa)
    p = O.default_params()
    active = 0
    for _ in range(25):
        st = sc.step(p)
        active = max(active, st["n_active_peak"])
        _, vv = sc.state()
        assert abs(vv[0, 0] - 0.5) < 1e-12 and abs(vv[0, 2] - 0.3) < 1e-12
    assert active > 0 and abs(vv[0, 1]) < 1e-9


def _moved(sa, R, t):
    """The scene rigidly moved by x -> R x + t (R a signed axis permutation,
    so axis-aligned planes stay axis-aligned): q = (R p + t, R A), velocities
    rotated, plane offsets shifted."""
    import copy
    sb = copy.deepcopy(sa)
    q, v = sb.body_q0.copy(), sb.body_v0.copy()
    for b in range(sb.n_bodies):
        q[b, :3] = R @ q[b, :3] + t
        q[b, 3:] = (R @ q[b, 3:].reshape(3, 3)).ravel()
        v[b, :3] = R @ v[b, :3]
        v[b, 3:] = (R @ v[b, 3:].reshape(3, 3)).ravel()
    sb.body_q0, sb.body_v0 = np.ascontiguousarray(q), np.ascontiguousarray(v)
    sb.plane_offset = np.array([sb.plane_offset[i] + sb.plane_sign[i] * t[sb.plane_axis[i]]
                                for i in range(len(sb.plane_offset))])
    return sb


@pytest.mark.parametrize("which", ["spheres_in_box", "cubes_on_plane"])
def test_step_is_frame_indifferent(which):
    """Eq. 1 has no preferred frame apart from gravity: moving the scene by a
    rotation about the gravity axis (x -> z, z -> -x) and a translation gives
    the moved trajectory, with the same Newton counts, through contact with a
    static mesh and with a ground plane.  Index or axis mistakes (a swapped
    component, a plane handled on the wrong axis) fail it."""
    if which == "spheres_in_box":
        sa = scenes.sphere_grid_in_box(n=2, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)
    else:
        sa = scenes.cube_stack(nx=2, ny=2, nz=1)
    R = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    t = np.array([0.375, 0.5, -1.25])
    a, b = O.Scene(sa), O.Scene(_moved(sa, R, t))
    dyn = sa.body_kind == scenes.KIND_DYNAMIC
    p = O.default_params()
    contact = 0
    for _ in range(20):
        sa_, sb_ = a.step(p), b.step(p)
        assert sa_["newton_iters"] == sb_["newton_iters"]
        contact = max(contact, sa_["n_active_peak"])
        qa, qb = a.state()[0][dyn], b.state()[0][dyn]
        pred = np.concatenate([qa[:, :3] @ R.T + t, np.einsum("ij,bjk->bik", R, qa[:, 3:].reshape(-1, 3, 3))
                               .reshape(-1, 9)], axis=1)
        assert np.abs(qb - pred).max() <= 1e-8
    assert contact > 0


def test_static_only_scene_has_nothing_to_solve():
    """Degenerate case: no dynamic or kinematic body, so Eq. 1 has no
    unknowns; static pairs are excluded even within dhat, the state stays bit
    for bit, and a four-slab partition changes nothing."""
    sa = scenes.static_only()
    for slabs in (1, 4):
        sc = O.Scene(sa)
        q0, v0 = sc.state()
        p = O.default_params(n_slabs=slabs, axis=0)
        for _ in range(3):
            st = sc.step(p)
            assert st["status"] == 0 and st["newton_iters"] == 0 and st["n_slots"] == 0
            assert st["n_candidates_peak"] == 0 and st["n_active_peak"] == 0
        q, v = sc.state()
        assert np.array_equal(q, q0) and np.array_equal(v, v0)


# --------------------------------------------------------------------------- O3

def test_orthogonality_fd_and_rotation_invariance():
    for _ in range(5):
        q = np.r_[RNG.normal(size=3), np.eye(3).ravel() + 0.2 * RNG.normal(size=9)]
        E, g, H = O.orth(q, 1e3, 0.37)
        gfd = fd_grad(lambda y: O.orth(y, 1e3, 0.37)[0], q, 1e-6)
        Hfd = np.stack([fd_grad(lambda y: O.orth(y, 1e3, 0.37)[1][i], q, 1e-6) for i in range(12)])
        assert np.abs(g - gfd).max() <= 1e-7 * np.abs(g).max()
        assert np.abs(H - Hfd).max() <= 1e-7 * np.abs(H).max()
        assert np.allclose(H, H.T, atol=0)
    for _ in range(5):
        R, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
        q = np.r_[RNG.normal(size=3), R.ravel()]
        E, g, _ = O.orth(q, 1e8, 1.0)
        assert E < 1e-20 and np.abs(g).max() < 1e-6  # kappa 1e8 times rounding of R R^T - I


def test_barrier_limits_and_fd():
    dhat = 1e-3
    for d in np.linspace(1e-5, 0.999e-3, 17):
        b, b1, b2 = O.barrier(d, dhat)
        h = 1e-9
        assert abs(b1 - (O.barrier(d + h, dhat)[0] - O.barrier(d - h, dhat)[0]) / (2 * h)) < 1e-6 * max(1, abs(b1))
        assert abs(b2 - (O.barrier(d + h, dhat)[1] - O.barrier(d - h, dhat)[1]) / (2 * h)) < 1e-5 * max(1, abs(b2))
        assert b > 0 and b1 < 0 and b2 > 0
    assert np.all(O.barrier(dhat, dhat) == 0) and np.all(O.barrier(2 * dhat, dhat) == 0)
    # C1 at dhat: value and slope tend to zero from below
    assert O.barrier(dhat * (1 - 1e-6), dhat)[0] < 1e-20


def _sampled_distance(is_ee, X, n=401):
    """Dense sampling of the parameter domain: an upper bound of the exact distance."""
    X = X.reshape(4, 3)
    u = np.linspace(0, 1, n)
    if not is_ee:
        U, V = np.meshgrid(u, u)
        keep = U + V <= 1
        U, V = U[keep], V[keep]
        pts = X[1] + U[:, None] * (X[2] - X[1]) + V[:, None] * (X[3] - X[1])
        return np.sqrt(((pts - X[0]) ** 2).sum(1)).min()
    S, T = np.meshgrid(u, u)
    a = X[0] + S.ravel()[:, None] * (X[1] - X[0])
    b = X[2] + T.ravel()[:, None] * (X[3] - X[2])
    return np.sqrt(((a - b) ** 2).sum(1)).min()


@pytest.mark.parametrize("is_ee", [0, 1])
def test_distance_against_dense_sampling(is_ee):
    types = set()
    for _ in range(300):
        X = RNG.normal(size=12)
        d2, t, _ = O.dist_type(is_ee, X)
        ds = _sampled_distance(is_ee, X)
        d = math.sqrt(d2)
        assert d <= ds + 1e-12
        assert ds - d <= 5e-3 * (1 + np.abs(X).max())
        types.add(t)
    assert len(types) >= (6 if is_ee else 5)


@pytest.mark.parametrize("is_ee", [0, 1])
def test_pair_energy_fd_every_type(is_ee):
    dhat, seen = 1.0, {}
    for _ in range(20000):
        X = RNG.normal(size=12) * 0.5
        d2, t, _ = O.dist_type(is_ee, X)
        if not (0.05 < math.sqrt(d2) < 0.9) or t in seen:
            continue
        seen[t] = X
        if len(seen) == (9 if is_ee else 7):
            break
    assert len(seen) == (9 if is_ee else 7)
    for t, X in seen.items():
        for eps in ((1e9, 1e-9) if is_ee else (0.0,)):  # mollifier active / inactive
            d, E, g, H, ty = O.pair(is_ee, X, dhat, 3.0, eps)
            assert ty == t
            gfd = fd_grad(lambda y: O.pair(is_ee, y, dhat, 3.0, eps)[1], X)
            Hfd = np.stack([fd_grad(lambda y: O.pair(is_ee, y, dhat, 3.0, eps)[2][i], X) for i in range(12)])
            assert np.abs(g - gfd).max() <= 1e-6 * max(1e-9, np.abs(g).max()), (t, eps)
            assert np.abs(H - Hfd).max() <= 1e-6 * max(1e-9, np.abs(H).max()), (t, eps)


def test_mollifier_fd_and_limits():
    for _ in range(10):
        X = RNG.normal(size=12)
        ea, eb = X[3:6] - X[0:3], X[9:12] - X[6:9]
        c = np.sum(np.cross(ea, eb) ** 2)
        eps = 2.0 * c
        m, g, H = O.mollifier(X, eps)
        assert abs(m - (0.5 * (2 - 0.5))) < 1e-12  # c/eps = 1/2
        gfd = fd_grad(lambda y: O.mollifier(y, eps)[0], X)
        Hfd = np.stack([fd_grad(lambda y: O.mollifier(y, eps)[1][i], X) for i in range(12)])
        assert np.abs(g - gfd).max() <= 1e-6 * np.abs(g).max()
        assert np.abs(H - Hfd).max() <= 1e-6 * np.abs(H).max()
        assert O.mollifier(X, 0.5 * c)[0] == 1.0
    X = np.r_[0, 0, 0, 1, 0, 0, 0, 1, 0, 1, 1, 0.0]  # parallel edges
    assert O.mollifier(X, 1e-3)[0] == 0.0


def test_psd_projection():
    for _ in range(200):
        n = int(RNG.choice([9, 12]))
        A = RNG.normal(size=(n, n))
        A = (A + A.T) * 10 ** RNG.uniform(-3, 8)
        P = O.psd_project(A)
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T
        assert np.abs(P - ref).max() <= 1e-12 * np.abs(A).max()
        assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.abs(A).max()
        B = A @ A.T
        assert np.array_equal(O.psd_project(B), B)  # PSD input unchanged


# --------------------------------------------------------------------------- O5

@pytest.mark.parametrize("is_ee", [0, 1])
def test_ccd_never_beyond_sampled_contact(is_ee):
    hits = 0
    for _ in range(150):
        X = RNG.normal(size=12)
        dX = RNG.normal(size=12) * 3.0
        toi = O.ccd(is_ee, X, dX)
        d0 = math.sqrt(O.dist_type(is_ee, X)[0])
        ts = np.linspace(0.0, 1.0, 4001)
        ds = np.array([math.sqrt(O.dist_type(is_ee, X + t * dX)[0]) for t in ts])
        # the path up to the returned time stays clear: d >= (1-c) * s * d0
        assert ds[ts <= toi].min() >= 0.01 * d0 * (1 - 1e-9)
        close = np.nonzero(ds < 0.005 * d0)[0]
        if len(close):
            hits += 1
            assert toi <= ts[close[0]]
        if toi < 1.0:
            assert math.sqrt(O.dist_type(is_ee, X + toi * dX)[0]) >= 0.1 * d0 * (1 - 1e-9)
    assert hits > 5


def test_ccd_closed_forms():
    # point falling head-on onto a triangle's interior at unit speed:
    # the first advance (1 - s) d0 / l_p is accepted, the next overshoots s d0.
    X = np.r_[0.2, 0.5, 0.2, 0, 0, 0, 1, 0, 0, 0, 0, 1.0]
    dX = np.r_[0, -1.0, 0, np.zeros(9)]
    assert abs(O.ccd(0, X, dX) - 0.9 * 0.5) < 1e-15
    # separating motion and common translation certify the whole path
    assert O.ccd(0, X, -dX) == 1.0
    assert O.ccd(0, X, np.tile([0.3, -7.0, 1.0], 4)) == 1.0
    # vertex-plane: d0 + t dd reaches s d0 at t = (1 - s) d0 / -dd
    assert abs(O.ccd_plane(0.5, -1.0, 0.1) - 0.45) < 1e-16
    assert O.ccd_plane(0.5, 0.2, 0.1) == 1.0 and O.ccd_plane(0.5, -0.1, 0.1) == 1.0


# --------------------------------------------------------------------------- O4

def _brute_candidates(sa, x0, x1, dhat, edges):
    """O(n^2) scan over every primitive pair of the scene (no prefilters)."""
    half = 0.5 * dhat
    nv = sa.body_vertex_counts()
    voff = np.r_[0, np.cumsum(nv)]
    nt = sa.body_tri_counts()
    tris = []
    for b in range(sa.n_bodies):
        m = sa.mesh(int(sa.body_mesh[b]))
        tris.append(m.tris + voff[b])
    tris = np.concatenate(tris)
    tri_body = np.repeat(np.arange(sa.n_bodies), nt)
    vert_body = np.repeat(np.arange(sa.n_bodies), nv)
    edge_body = vert_body[edges[:, 0]]
    dyn = sa.body_kind == 0

    def boxes(ix):
        pts = x0[ix] if x1 is None else np.concatenate([x0[ix], x1[ix]], axis=1)
        return pts.min(axis=1) - half, pts.max(axis=1) + half

    vlo, vhi = boxes(np.arange(x0.shape[0])[:, None])
    tlo, thi = boxes(tris)
    elo, ehi = boxes(edges)
    out = set()
    ov = lambda alo, ahi, blo, bhi: np.all((alo[:, None] <= bhi[None]) & (blo[None] <= ahi[:, None]), axis=2)
    M = ov(vlo, vhi, tlo, thi)
    for i, j in zip(*np.nonzero(M)):
        a, b = vert_body[i], tri_body[j]
        if a != b and (dyn[a] or dyn[b]):
            out.add((0, int(i), int(j)))
    M = ov(elo, ehi, elo, ehi)
    for i, j in zip(*np.nonzero(M)):
        a, b = edge_body[i], edge_body[j]
        if i < j and a != b and (dyn[a] or dyn[b]):
            out.add((1, int(i), int(j)))
    return out


def test_candidates_match_brute_force():
    sa = scenes.sphere_grid_in_box(n=2, ny=2, nz=1, level=1, spacing=0.2005, lowest=0.1004)
    sc = O.Scene(sa)
    x = sc.vertices()
    edges = sc.edges()
    dhat = 2e-3
    got = {tuple(int(v) for v in r) for r in sc.candidates(x, None, dhat)}
    ref = _brute_candidates(sa, x, None, dhat, edges)
    assert got == ref and len(ref) > 50
    x1 = x + RNG.normal(size=x.shape) * 0.01
    got = {tuple(int(v) for v in r) for r in sc.candidates(x, x1, dhat)}
    ref = _brute_candidates(sa, x, x1, dhat, edges)
    assert got == ref and len(ref) > 100


# --------------------------------------------------------------------------- O6

def _recentred_xbar(sc, q):
    qi = q.copy()
    qi[:, :3] = 0
    qi[:, 3:] = np.eye(3).ravel()
    return sc.vertices(qi)


def test_objective_gradient_fd_and_assembly_rebuilt_in_numpy():
    """Energy/gradient by finite differences; Hessian re-assembled here from the
    pair Hessians with an independent J^T H J scatter."""
    sa = scenes.cube_stack(nx=1, ny=2, nz=1, bottom_gap=4e-4, spacing=1.0005, jitter=1e-4)
    sc = O.Scene(sa)
    q, _ = sc.state()
    h, dhat, kB = 1e-2, 1e-3, 1e5
    p = O.default_params(kappa_barrier=kB)
    qt = q.copy()
    qt[:, :3] += sa.gravity * h * h
    E, g, H = sc.objective(p, q, qt)
    gfd = fd_grad(lambda y: sc.objective(p, y.reshape(q.shape), qt, False)[0], q.ravel(), 1e-9)
    assert np.abs(g - gfd).max() <= 1e-5 * np.abs(g).max()
    # independent assembly
    x = sc.vertices(q)
    xb = _recentred_xbar(sc, q)
    nv = sa.body_vertex_counts()
    vb = np.repeat(np.arange(sa.n_bodies), nv)
    voff = np.r_[0, np.cumsum(nv)]
    tris = np.concatenate([sa.mesh(int(sa.body_mesh[b])).tris + voff[b] for b in range(sa.n_bodies)])
    edges = sc.edges()
    erest2 = ((xb[edges[:, 0]] - xb[edges[:, 1]]) ** 2).sum(1)
    n = 12 * sa.n_bodies
    Href = np.zeros((n, n))

    def J(v):
        Jv = np.zeros((3, 12))
        Jv[:, :3] = np.eye(3)
        for k in range(3):
            Jv[k, 3 + 3 * k:6 + 3 * k] = xb[v]
        return Jv

    npairs = 0
    for t, i, j in sc.candidates(x, None, dhat):
        vs = [i, *tris[j]] if t == 0 else [*edges[i], *edges[j]]
        eps = 0.0 if t == 0 else 1e-3 * erest2[i] * erest2[j]
        d, e, gp, Hp, _ = O.pair(t, x[vs].ravel(), dhat, kB, eps)
        if d >= dhat:
            continue
        npairs += 1
        Hp = O.psd_project(Hp) * h * h
        Jall = np.zeros((12, n))
        for k, v in enumerate(vs):
            Jall[3 * k:3 * k + 3, 12 * vb[v]:12 * vb[v] + 12] = J(v)
        Href += Jall.T @ Hp @ Jall
    for v in range(x.shape[0]):
        d = x[v, 1]
        if d < dhat:
            npairs += 1
            b2 = O.barrier(d, dhat)[2]
            Jv = J(v)
            Href[12 * vb[v]:12 * vb[v] + 12, 12 * vb[v]:12 * vb[v] + 12] += h * h * kB * b2 * np.outer(Jv[1], Jv[1])
    for b in range(sa.n_bodies):
        m, _, S, V = sc.body_props(b)
        M = np.zeros((12, 12))
        M[:3, :3] = m * np.eye(3)
        for k in range(3):
            M[3 + 3 * k:6 + 3 * k, 3 + 3 * k:6 + 3 * k] = S
        _, _, Ho = O.orth(q[b], sa.body_kappa[b], V)
        Ho[3:, 3:] = O.psd_project(Ho[3:, 3:])
        Href[12 * b:12 * b + 12, 12 * b:12 * b + 12] += M + h * h * Ho
    assert npairs > 10
    assert np.abs(H - Href).max() <= 1e-10 * np.abs(Href).max()
    assert np.linalg.eigvalsh(H).min() > 0


@pytest.mark.parametrize("solver,dims,steps", [("dense", (2, 2, 2), 14), ("pcg", (6, 5, 6), 8)])
def test_step_ends_at_a_newton_stationary_point_of_the_objective(solver, dims, steps):
    """The state a single-partition step returns is where projected Newton
    on Eq. 1 stops: a Newton step computed outside the solver -- numpy's
    dense solve with the objective's own gradient and projected Hessian at
    the returned state and the step's q~ -- is below epsilon_N h l, while at
    the step's start state it is not (free fall and stacking contact).  The
    180-cube stack (2160 unknowns) takes the oracle's block-Jacobi PCG branch
    (above 2000 unknowns), the 8-cube stack its dense Cholesky."""
    sa = scenes.cube_stack(nx=dims[0], ny=dims[1], nz=dims[2])
    assert (12 * sa.n_dynamic > 2000) == (solver == "pcg")
    sc = O.Scene(sa)
    p = O.default_params(kappa_barrier=1e5)
    dyn = sa.body_kind == scenes.KIND_DYNAMIC
    contact = 0
    for _ in range(steps):
        q0, v0 = sc.state()
        st = sc.step(p)
        assert st["status"] == 0
        contact = max(contact, st["n_active_peak"])
        q1, _ = sc.state()
        qt = q0 + p.h * v0
        qt[:, :3] += p.h * p.h * sa.gravity
        tol = p.newton_tol * p.h * st["l"]
        _, g1, H1 = sc.objective(p, q1[dyn], qt[dyn])
        _, g0, H0 = sc.objective(p, q0[dyn], qt[dyn])
        assert np.abs(np.linalg.solve(H1, g1)).max() < tol
        assert np.abs(np.linalg.solve(H0, g0)).max() > 100 * tol
    assert contact > 0


def test_cube_resting_on_plane_balances_weight():
    """Vertex-plane equilibrium: at rest, -kB * sum_c b'(d_c) = m |g|."""
    sa = scenes.cube_stack(nx=1, ny=1, nz=1, bottom_gap=2e-4, jitter=0.0)
    sc = O.Scene(sa)
    p = O.default_params(newton_tol=1e-11)  # equilibrium to solver precision
    for _ in range(150):
        st = sc.step(p)
    q, v = sc.state()
    assert np.abs(v).max() < 1e-7
    x = sc.vertices(q)
    kB = st["kappa_barrier"]
    m = sc.body_props(0)[0]
    force = -kB * sum(O.barrier(d, p.dhat)[1] for d in x[:, 1] if d < p.dhat)
    assert abs(force - m * 9.8) < 1e-6 * m * 9.8  # residual motion v < 1e-7 m/s


def test_stack_invariants_100_steps():
    sc = O.Scene(scenes.cube_stack())
    p = O.default_params()
    for _ in range(100):
        st = sc.step(p)
        assert st["min_distance"] > 0 and st["status"] == 0
    q, _ = sc.state()
    for b in range(q.shape[0]):
        A = q[b, 3:].reshape(3, 3)
        assert np.linalg.norm(A @ A.T - np.eye(3)) < 1e-3


# --------------------------------------------------------------------------- O7

def test_partition_masks_rule():
    sa = scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, spacing=0.3)
    sc = O.Scene(sa)
    planes = [-0.25, 0.0, 0.3]
    p = O.default_params(n_slabs=4, axis=0, planes=planes)
    mask, w = sc.partition(p)
    x = sc.vertices()
    nv = sa.body_vertex_counts()
    off = np.r_[0, np.cumsum(nv)]
    lo = np.array([x[off[b]:off[b + 1], 0].min() for b in range(sa.n_bodies)])
    hi = np.array([x[off[b]:off[b + 1], 0].max() for b in range(sa.n_bodies)])
    dyn = sa.body_kind == 0
    diag = [np.linalg.norm(x[off[b]:off[b + 1]].max(0) - x[off[b]:off[b + 1]].min(0)) for b in np.nonzero(dyn)[0]]
    assert abs(w - min(diag)) < 1e-12  # at rest: w = w_min
    edges = [-np.inf] + planes + [np.inf]
    for b in range(sa.n_bodies):
        want = 0
        if dyn[b]:
            for i in range(4):
                rlo = edges[i] - w / 2 if i > 0 else -np.inf
                rhi = edges[i + 1] + w / 2 if i < 3 else np.inf
                if lo[b] <= rhi and hi[b] >= rlo:
                    want |= 1 << i
        assert int(mask[b]) == want


def test_admm_single_partition_is_monolithic():
    sa = scenes.cube_stack(nx=2, ny=2, nz=1)
    a, b = O.Scene(sa), O.Scene(sa)
    for _ in range(8):
        a.step(O.default_params())
        b.step(O.default_params(n_slabs=1, axis=0))
    assert np.array_equal(a.state()[0], b.state()[0])


def test_admm_free_flight_converges_to_prediction():
    sa = scenes.two_body_free_flight(gap=0.05)
    sc = O.Scene(sa)
    q0, v0 = sc.state()
    p = O.default_params(n_slabs=2, axis=0, planes=[0.0])
    st = sc.step(p)
    q, _ = sc.state()
    assert st["n_shared"] == 2 and st["status"] == 0
    # two local solves: the first moves to q~, the second certifies no change
    assert st["admm_iters"] == 2 and st["r_inf"] < 1e-14 and st["s_inf"] < 1e-14
    pred = q0[:, :3] + 1e-2 * v0[:, :3] + 1e-4 * sa.gravity
    assert np.abs(q[:, :3] - pred).max() < 1e-12


@pytest.mark.parametrize("slabs", [2, 3])
@pytest.mark.parametrize("static_base", [False, True])
def test_local_objectives_sum_to_global_at_consensus(slabs, static_base):
    """Eq. 3's weights split Eq. 1 exactly: at a consensus point (every
    replica at the body's q, so the augmented term is zero) the partitions'
    objectives sum to the single-partition objective, and so do their
    gradients and projected Hessians.  A touching row of six cubes (gaps 5e-4 < dhat, resting 5e-4
    above the plane) puts contacts between a shared and an internal body,
    between two shared bodies and on the plane; with `static_base` a second
    row rests on it and the first row is static, so contacts pair dynamic
    and static bodies in both orders (static vertex on a dynamic face and the
    reverse).  A wrong kappa_b or kappa_c (e.g. counting partitions holding
    either body instead of both) fails."""
    sa = scenes.cube_stack(nx=6, ny=2 if static_base else 1, nz=1, spacing=1.0005, bottom_gap=5e-4, jitter=0.0)
    if static_base:
        sa.body_kind = np.where(sa.body_q0[:, 1] < 1.0, scenes.KIND_STATIC, scenes.KIND_DYNAMIC).astype(np.int32)
    sc = O.Scene(sa)
    p = O.default_params(n_slabs=slabs, axis=0, kappa_barrier=1e5)
    m, _ = sc.partition(p)
    assert any(bin(int(x)).count("1") >= 2 for x in m) and any(bin(int(x)).count("1") == 1 for x in m)
    q, _ = sc.state()
    qd = q[sa.body_kind == scenes.KIND_DYNAMIC]
    qt = qd + 1e-3 * np.random.default_rng(0).normal(size=qd.shape)
    Ep, gs, Hs = sc.local_objectives(p, qd, qt, want_hess=True)
    E, g, H = sc.objective(p, qd, qt)
    assert len(Ep) == slabs and np.all(Ep > 0)
    # the barrier terms are active: the objective differs from inertia + orthogonality alone
    E_free, _, _ = sc.objective(O.default_params(kappa_barrier=1e-30), qd, qt, want_hess=False)
    assert E - E_free > 1e-3 * E
    assert abs(Ep.sum() - E) <= 1e-12 * abs(E)
    assert np.abs(gs - g.reshape(gs.shape)).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(Hs - H).max() <= 1e-12 * np.abs(H).max()


def test_local_objectives_sum_to_global_with_static_mesh_contacts():
    """The same split on the 16-sphere pile settled in its static box over
    two slabs: contacts between spheres and with the box, where a pair with
    a static body is weighted by the partitions holding the dynamic one."""
    sa = scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)
    sc = O.Scene(sa)
    p = O.default_params(n_slabs=2, axis=0)
    for _ in range(16):
        st = sc.step(p)
    assert st["n_shared"] > 0 and st["n_active_peak"] > 0
    pk = O.default_params(n_slabs=2, axis=0, kappa_barrier=st["kappa_barrier"])
    q, _ = sc.state()
    qd = q[sa.body_kind == scenes.KIND_DYNAMIC]
    qt = qd + 1e-4 * np.random.default_rng(0).normal(size=qd.shape)
    Ep, gs, Hs = sc.local_objectives(pk, qd, qt, want_hess=True)
    E, g, H = sc.objective(pk, qd, qt)
    E_free, _, _ = sc.objective(O.default_params(kappa_barrier=1e-30), qd, qt, want_hess=False)
    assert E - E_free > 0.5 * E  # the barrier terms dominate
    assert abs(Ep.sum() - E) <= 1e-12 * abs(E)
    assert np.abs(gs - g.reshape(gs.shape)).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(Hs - H).max() <= 1e-12 * np.abs(H).max()


def test_admm_rounds_grow_with_the_partition_count():
    """Paper behaviour (Sec. 6, Multi-worker Scaling), not parity: more
    partitions mean more shared bodies to agree on, so the 16-sphere pile
    landing in its box needs more ADMM rounds in total on 4 slabs than on 2,
    and a single partition needs exactly one round per step."""
    sa = scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)
    rounds = {}
    for n in (1, 2, 4):
        sc = O.Scene(sa)
        rounds[n] = sum(sc.step(O.default_params(n_slabs=n, axis=0))["admm_iters"] for _ in range(16))
    assert rounds[1] == 16 and rounds[1] < rounds[2] < rounds[4]


def test_admm_tracks_monolithic_per_step():
    """The converged consensus state lies within O(theta h l) of the
    single-partition solution from the same start (the q* comparison)."""
    sa = scenes.cube_stack(nx=4, ny=2, nz=1)
    mono, adm = O.Scene(sa), O.Scene(sa)
    pm = O.default_params()
    pa = O.default_params(n_slabs=2, axis=0)
    for _ in range(15):
        q, v = mono.state()
        adm.set_state(q, v)
        s1 = mono.step(pm)
        s2 = adm.step(pa)
        tol = pa.theta * pa.h * s2["l"]
        assert s2["status"] == 0 and s2["n_shared"] > 0
        assert np.abs(mono.state()[0] - adm.state()[0]).max() < 2 * tol
        assert s2["min_distance"] > 0


@pytest.mark.parametrize("which", ["spheres_in_box", "touching_cubes"])
def test_admm_reaches_the_single_partition_solution_as_theta_shrinks(which):
    """The paper's q* comparison on contact steps: from the single-partition
    trajectory's state, ADMM with a tighter theta (Eq. 8) ends closer to the
    single-partition step, and at theta = 1e-6 within 1e-6 of it (the floor
    set by the local Newton tolerances).  The 16-sphere pile lands on its box
    over two slabs; two rows of touching cubes (gaps 5e-4 < dhat) over three
    slabs settle after their first, strongly repulsive step.  At the default
    theta = 1e-3 the stopping test may end far sooner: Eq. 10's dual
    residual, the unscaled change of z, can fall below theta h l while z is
    still crawling toward the solution.  The chosen steps are ones where both
    solvers settle in the same local minimum: the IPC energy is not convex,
    and at some contact steps (step 15 of this pile) the consensus and the
    single-partition solves end in different minima, with no theta closing
    the gap."""
    if which == "spheres_in_box":
        sa = scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)
        slabs, steps = 2, (5, 9)
    else:
        sa = scenes.cube_stack(nx=6, ny=2, nz=1, spacing=1.0005, bottom_gap=5e-4, jitter=0.0)
        slabs, steps = 3, (1, 3)
    mono = O.Scene(sa)
    pm = O.default_params()
    states = []
    for _ in range(max(steps) + 1):
        states.append(mono.state())
        mono.step(pm)
    ref, adm = O.Scene(sa), O.Scene(sa)
    for k in steps:
        q, v = states[k]
        ref.set_state(q, v)
        assert ref.step(pm)["n_active_peak"] > 0
        q_ref = ref.state()[0]
        err = {}
        for theta in (1e-3, 1e-4, 1e-6):
            adm.set_state(q, v)
            st = adm.step(O.default_params(n_slabs=slabs, axis=0, theta=theta, max_admm=400))
            assert st["status"] == 0 and st["n_shared"] > 0
            err[theta] = np.abs(adm.state()[0] - q_ref).max()
        assert err[1e-6] < 1e-6 and err[1e-4] < 1e-4
        assert err[1e-6] < err[1e-3]


def test_paper_constants_are_the_defaults():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    p = O.default_params()
    for k in ("beta", "tau", "mu", "sigma_min", "sigma_max", "alpha_w"):
        assert getattr(p, k) == gold[k]["value"], k


def _rot_y(t):
    return np.array([[math.cos(t), 0.0, math.sin(t)], [0.0, 1.0, 0.0], [-math.sin(t), 0.0, math.cos(t)]])


def _lone_bar(omega=2.0, v=(0.0, 0.0, 0.0)):
    import dataclasses
    sa = scenes.kinematic_sweeper(n_cubes=1, omega=omega)
    keep = slice(0, 1)
    v0 = np.zeros((1, 12))
    v0[0, :3] = v
    return dataclasses.replace(sa, body_mesh=sa.body_mesh[keep].copy(), body_density=sa.body_density[keep].copy(),
                               body_kappa=sa.body_kappa[keep].copy(), body_kind=sa.body_kind[keep].copy(),
                               body_q0=sa.body_q0[keep].copy(), body_v0=v0, body_omega=sa.body_omega[keep].copy())


def test_kinematic_body_follows_its_prescription():
    """Without contact the minimiser of a kinematic body's step is its
    prescribed pose (a rotation: zero orthogonality energy and gradient), so
    after n steps A = R_y(n omega h) A0 and p = p0 + n h v, with no gravity."""
    sa = _lone_bar(omega=2.0, v=(0.3, 0.0, -0.1))
    o = O.Scene(sa)
    p = O.default_params(newton_tol=1e-13)
    q0, _ = o.state()
    n = 15
    for _ in range(n):
        o.step(p)
    q, v = o.state()
    A = q[0, 3:].reshape(3, 3)
    assert np.abs(A - _rot_y(2.0 * p.h * n) @ q0[0, 3:].reshape(3, 3)).max() < 1e-12
    assert np.abs(q[0, :3] - (q0[0, :3] + n * p.h * np.array([0.3, 0.0, -0.1]))).max() < 1e-12


def test_kinematic_sweeper_pushes_without_penetration():
    sa = scenes.kinematic_sweeper()
    o = O.Scene(sa)
    p = O.default_params()
    q0, _ = o.state()
    n = 40
    for _ in range(n):
        st = o.step(p)
        assert st["min_distance"] > 0.0
    q, _ = o.state()
    A = q[0, 3:].reshape(3, 3)
    # the bar keeps its prescription to within contact-induced deviations
    assert np.abs(A - _rot_y(2.0 * p.h * n) @ q0[0, 3:].reshape(3, 3)).max() < 1e-6
    # and it pushed the first cube
    assert np.linalg.norm(q[1, :3] - q0[1, :3]) > 0.05


def test_perforated_turntable_mesh_closed_form_volume():
    """The perforated turntable is a watertight outward mesh whose volume is
    kept cells x cell^2 x thickness (divergence theorem in the oracle's mass
    properties), and the oracle weights its inertia as a kinematic body."""
    m = scenes.perforated_disk_mesh()
    sa = scenes.funnel_scene(n_bodies=1, level=1)
    o = O.Scene(sa)
    mass, com, S, V = o.body_props(2)
    assert abs(V - m.n_cells * 0.07 ** 2 * 0.05) < 1e-12
    assert abs(mass - 1000.0 * V * 1e6) < 1e-6 * mass
    assert np.abs(com).max() < 1e-12  # symmetric hole pattern


def test_funnel_crop_turntables_and_free_fall():
    """A crop of the funnel workload: the two turntables turn by +-omega h per
    step and the spheres, not yet in contact, fall as the closed form says."""
    sa = scenes.funnel_scene(n_bodies=8, level=1)
    o = O.Scene(sa)
    p = O.default_params()
    q0, _ = o.state()
    n = 4
    for _ in range(n):
        o.step(p)
    q, _ = o.state()
    for b, sgn in ((2, 1.0), (3, -1.0)):
        R = _rot_y(sgn * 1.0 * p.h * n)
        assert np.abs(q[b, 3:].reshape(3, 3) - R @ q0[b, 3:].reshape(3, 3)).max() < 1e-6
    g = -9.8 * p.h ** 2 * n * (n + 1) / 2
    assert np.abs(q[4:, 1] - q0[4:, 1] - g).max() < 1e-12


def test_kinematic_sweeper_two_slabs_invariants():
    """The sweeping bar straddles the slab plane (replicated on both slabs):
    consensus keeps it on its prescription and every step stays apart."""
    sa = scenes.kinematic_sweeper()
    o = O.Scene(sa)
    p = O.default_params(n_slabs=2, axis=0, planes=[0.0])
    q0, _ = o.state()
    n = 30
    shared = 0
    for _ in range(n):
        st = o.step(p)
        assert st["min_distance"] > 0.0 and st["status"] >= 0
        shared = max(shared, st["n_shared"])
    q, _ = o.state()
    assert shared >= 1
    assert np.abs(q[0, 3:].reshape(3, 3) - _rot_y(2.0 * p.h * n) @ q0[0, 3:].reshape(3, 3)).max() < 1e-6


def test_blocked_merge_retaken_as_two_half_steps():
    """With one ADMM round allowed, some steps of a contact-rich two-slab pile
    end with a blocked merge (fallback); with dt_split_max = 1 those steps are
    taken as two steps of h/2 instead, each penetration-free, and the result
    equals stepping twice with h/2 from the same state."""
    sa = scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)
    base = dict(max_admm=1, n_slabs=2, axis=0)
    o0, o1 = O.Scene(sa), O.Scene(sa)
    split_steps = []
    for k in range(24):
        q, v = o1.state()
        s0 = o0.step(O.default_params(**base))
        s1 = o1.step(O.default_params(dt_split_max=1, **base))
        if s0["status"] == 3:
            assert s1["status"] == 4 and s1["min_distance"] > 0.0
            split_steps.append(k)
            # the same step by hand: two steps of h/2 from the same state
            o2 = O.Scene(sa)
            o2.set_state(q, v)
            half = O.default_params(**base)
            half.h = 0.5 * half.h
            o2.step(half)
            o2.step(half)
            assert np.array_equal(o2.state()[0], o1.state()[0])
        o0.set_state(*o1.state())
    assert split_steps, "no blocked merge in the window"


def test_heterogeneous_pile_groups_and_masses():
    """Material-heterogeneity workload (Sec. 6.2, Table 2): 200 bodies in three
    groups (67/67/66 by a seeded shuffle); each body's mass from the oracle's
    volume integral equals its group mass m_g, its orthogonality stiffness is
    the group's E_g; the uniform baseline gives every body (100, 1e10).  The
    oracle's mass is pinned to closed-form volumes elsewhere, so this checks
    that the generator hands each body the density m_g / V_b."""
    sa = scenes.heterogeneous_pile()
    assert sa.n_dynamic == 200 and np.bincount(sa.body_group).tolist() == [67, 67, 66]
    o = O.Scene(sa)
    for b in range(sa.n_dynamic):
        m_g, e_g = scenes.HETERO_GROUPS[sa.body_group[b]]
        assert abs(o.body_props(b)[0] / m_g - 1.0) < 1e-12
        assert sa.body_kappa[b] == e_g
    su = scenes.heterogeneous_pile(hetero=False)
    ou = O.Scene(su)
    assert np.array_equal(su.body_q0, sa.body_q0)
    for b in range(0, su.n_dynamic, 17):
        assert abs(ou.body_props(b)[0] / 100.0 - 1.0) < 1e-12 and su.body_kappa[b] == 1e10


def test_heterogeneous_crop_steps_penetration_free():
    """A 3 x 2 x 3 crop of the heterogeneous pile (masses 1 to 1e4 side by
    side, stiffness 1e8 to 1e12) settles onto the box floor on two slabs:
    every step ends penetration-free with a status >= 0, and the stiff heavy
    bodies stay rigid (||A A^T - I|| small)."""
    sa = scenes.heterogeneous_pile(nx=3, ny=2, nz=3)
    o = O.Scene(sa)
    p = O.default_params(n_slabs=2, axis=0, planes=[0.0])
    contact = False
    for _ in range(16):
        st = o.step(p)
        assert st["status"] >= 0 and st["min_distance"] > 0.0
        contact |= st["min_distance"] < p.dhat
    assert contact
    q = o.state()[0]
    for b in range(sa.n_dynamic):
        A = q[b, 3:].reshape(3, 3)
        assert np.abs(A @ A.T - np.eye(3)).max() < 1e-3


def test_dt_split_depth_is_bounded():
    """A negative or over-deep split request is rejected before any work
    (at most 2^16 sub-steps per step)."""
    sa = scenes.cube_stack(nx=1, ny=1, nz=1)
    o = O.Scene(sa)
    q0 = o.state()[0].copy()
    for bad in (-1, 17):
        with pytest.raises(RuntimeError, match="failed: -1 "):
            o.step(O.default_params(dt_split_max=bad))
    assert np.array_equal(o.state()[0], q0)
    assert o.step(O.default_params(dt_split_max=16))["status"] >= 0


def test_newton_cap_status_boundary():
    """A step whose local solve meets eps_N at its n-th Newton solve is OK with
    max_newton = n and reports NEWTON_MAXITER with max_newton = n - 1 (the
    state is still advanced by the n - 1 iterations taken)."""
    sa = scenes.cube_stack()
    o = O.Scene(sa)
    for _ in range(40):  # the first step with contact Newton work
        q0, v0 = o.state()
        st = o.step(O.default_params())
        n = st["newton_iters"]
        if n > 2:
            break
    assert st["status"] == O.OK and n > 2
    for cap, status in ((n, O.OK), (n - 1, O.NEWTON_MAXITER)):
        o.set_state(q0, v0)
        s2 = o.step(O.default_params(max_newton=cap))
        assert (s2["status"], s2["newton_iters"]) == (status, cap)
