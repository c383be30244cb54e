"""CUDA path vs the FP64 oracle, through the C ABI, on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
from paper_2605_15875_gb300 import abd, scenes

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9   # relative in q per step (FP64 path)
MIXED_TOL = 1e-4  # relative in q over 100 steps (FP32 assembly and PCG)


def rel(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_15875_gb300 import build
    build.build()
    abd.load()


def test_body_constants_match_oracle():
    sa = scenes.sphere_grid_in_box(n=2, level=2)
    g, o = abd.Scene(sa), O.Scene(sa)
    for b in range(sa.n_bodies):
        mg, cg, Sg, Vg = g.body_props(b)
        mo, co, So, Vo = o.body_props(b)
        assert abs(mg - mo) <= 1e-12 * max(1, mo) and abs(Vg - Vo) <= 1e-12 * max(1, Vo)
        assert np.abs(cg - co).max() < 1e-15 and np.abs(Sg - So).max() <= 1e-12 * max(1e-30, np.abs(So).max())
    assert np.array_equal(g.state()[0], g.state()[0])
    assert rel(g.state()[0], o.state()[0]) < 1e-15


def _cand_set(arr):
    return {tuple(int(v) for v in r) for r in arr}


@pytest.mark.parametrize("swept", [False, True])
def test_candidates_bit_exact(swept):
    sa = scenes.sphere_grid_in_box(n=3, ny=2, nz=2, level=2, spacing=0.2004, lowest=0.1003)
    g, o = abd.Scene(sa), O.Scene(sa)
    x = o.vertices()
    rng = np.random.default_rng(7)
    x1 = x + rng.normal(size=x.shape) * 0.004 if swept else None
    for dhat in (1e-3, 4e-3):
        got = g.candidates(x, x1, dhat)
        ref = o.candidates(x, x1, dhat)
        assert len(ref) > 100
        assert _cand_set(got) == _cand_set(ref)
        assert len(got) == len(ref)  # no duplicates


def _run_pair(sa, steps, params_g, params_o, tol, partition=None, traj_tol=1e-7):
    """Per-step parity: before every step the CUDA scene takes the oracle's
    state, so each comparison measures the error of one step (the FP64
    contract).  A second CUDA scene runs free and its drift over the whole
    trajectory is bounded by `traj_tol`.  Discrete decisions (ADMM rounds,
    Newton iterations) must agree."""
    g, free, o = abd.Scene(sa), abd.Scene(sa), O.Scene(sa)
    if partition:
        g.partition(**partition)
        free.partition(**partition)
    worst = 0.0
    for k in range(steps):
        qo, vo = o.state()
        g.set_state(qo, vo)
        sg = g.step(params_g)
        free.step(params_g)
        so = o.step(params_o)
        qg, _ = g.state()
        qo, _ = o.state()
        e = rel(qg, qo)
        worst = max(worst, e)
        assert e <= tol, (k, e, sg, so)
        assert sg["status"] >= 0
        assert sg["min_distance"] > 0.0, (k, sg)  # no penetration in the final state, across partitions
        assert (sg["admm_iters"], sg["newton_iters"]) == (so["admm_iters"], so["newton_iters"]), (k, sg, so)
    drift = rel(free.state()[0], o.state()[0])
    print(f"per-step worst {worst:.3e}, trajectory drift {drift:.3e}")
    assert drift <= traj_tol
    return worst, g, o


def test_free_fall_closed_form_gpu():
    sa = scenes.two_body_free_flight(seed=3)
    g = abd.Scene(sa)
    q0, v0 = g.state()
    for n in range(1, 11):
        st = g.step(abd.default_params())
        q, _ = g.state()
        pred = q0[:, :3] + n * 1e-2 * v0[:, :3] + 1e-4 * sa.gravity * n * (n + 1) / 2
        assert np.abs(q[:, :3] - pred).max() < 1e-12
        assert np.abs(q[:, 3:] - q0[:, 3:]).max() == 0.0


def test_cube_stack_fp64_parity_100_steps():
    sa = scenes.cube_stack()
    worst, g, o = _run_pair(sa, 100, abd.default_params(), O.default_params(), FP64_TOL)
    print("worst rel err", worst)


def test_cube_row_admm_fp64_parity():
    sa = scenes.cube_stack(nx=4, ny=2, nz=1)
    worst, g, o = _run_pair(sa, 25, abd.default_params(), O.default_params(n_slabs=2, axis=0), FP64_TOL,
                            partition=dict(n_slabs=2, axis=0))
    print("worst rel err", worst)


def test_cube_stack_mixed_100_steps():
    sa = scenes.cube_stack()
    g, o = abd.Scene(sa), O.Scene(sa)
    pg = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-4)
    for k in range(100):
        st = g.step(pg)
        o.step(O.default_params())
        assert st["status"] >= 0
    e = rel(g.state()[0], o.state()[0])
    print("mixed rel err after 100 steps", e)
    assert e <= MIXED_TOL


def _sphere_admm_scene():
    return scenes.sphere_grid_in_box(n=4, ny=2, nz=2, level=1, lowest=0.12, spacing=0.25)


def test_sphere_pile_admm_fp64_parity():
    """Contact-rich consensus ADMM (2 slabs, shared spheres landing on the box
    floor): FP64 path within 1e-9 of the oracle every step."""
    sa = _sphere_admm_scene()
    worst, g, o = _run_pair(sa, 16, abd.default_params(), O.default_params(n_slabs=2, axis=0), FP64_TOL,
                            partition=dict(n_slabs=2, axis=0))
    print("worst rel err", worst)


def test_sphere_pile_admm_mixed():
    sa = _sphere_admm_scene()
    g, o = abd.Scene(sa), O.Scene(sa)
    g.partition(n_slabs=2, axis=0)
    pg = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5)
    for k in range(16):
        st = g.step(pg)
        o.step(O.default_params(n_slabs=2, axis=0))
        assert st["status"] >= 0
    e = rel(g.state()[0], o.state()[0])
    print("mixed rel err after 16 steps", e)
    assert e <= MIXED_TOL


def test_sphere_pile_admm_mixed_100_steps():
    """The mixed path on a multi-partition contact pile over 100 steps (16
    spheres on two slabs landing in their box and settling): every step from
    the oracle's state within 1e-4 of the oracle's step, and a free-running
    mixed trajectory with positive minimum distance after every step.  The
    free run's drift from the oracle's own trajectory is printed: on a pile the
    two FP64-vs-FP32 trajectories part like any two nearby trajectories of a
    contact-rich system, so the per-step comparison is the bound."""
    sa = _sphere_admm_scene()
    g, free, o = abd.Scene(sa), abd.Scene(sa), O.Scene(sa)
    for sc in (g, free):
        sc.partition(n_slabs=2, axis=0)
    pg = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5)
    po = O.default_params(n_slabs=2, axis=0)
    worst, drift, contact = 0.0, [], 0
    for k in range(100):
        qo, vo = o.state()
        g.set_state(qo, vo)
        sg = g.step(pg)
        sf = free.step(pg)
        so = o.step(po)
        e = rel(g.state()[0], o.state()[0])
        worst = max(worst, e)
        assert e <= MIXED_TOL, (k, e)
        assert sg["status"] >= 0 and sf["status"] >= 0
        assert sf["min_distance"] > 0.0 and sg["min_distance"] > 0.0, (k, sf, sg)
        contact += so["n_active_peak"] > 0
        drift.append(rel(free.state()[0], o.state()[0]))
    print(f"per-step worst {worst:.3e}; free-run drift after 10/50/100 steps "
          f"{drift[9]:.3e}/{drift[49]:.3e}/{drift[99]:.3e}; contact steps {contact}")
    assert contact >= 50


def test_kinematic_sweeper_fp64_parity():
    """A kinematic bar (prescribed rotation) sweeping into cubes: FP64 path
    within 1e-9 of the oracle every step, equal Newton counts, no penetration."""
    sa = scenes.kinematic_sweeper()
    worst, g, o = _run_pair(sa, 30, abd.default_params(), O.default_params(), FP64_TOL)
    print("worst rel err", worst)


def test_kinematic_sweeper_two_slabs_mixed():
    """The sweeping bar straddles the slab plane (a shared kinematic body):
    mixed path within 1e-4 of the oracle after 30 steps."""
    sa = scenes.kinematic_sweeper()
    g, o = abd.Scene(sa), O.Scene(sa)
    g.partition(n_slabs=2, axis=0, planes=[0.0])
    pg = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5)
    for k in range(30):
        st = g.step(pg)
        o.step(O.default_params(n_slabs=2, axis=0, planes=[0.0]))
        assert st["status"] >= 0 and st["min_distance"] > 0.0
    e = rel(g.state()[0], o.state()[0])
    print("mixed rel err after 30 steps", e)
    assert e <= MIXED_TOL


def test_load_balanced_planes_fp64_parity():
    """PD load balancing on two slabs starting from an uneven plane: every step
    the CUDA scene moves the plane toward balance; handing the oracle the same
    plane each step keeps FP64 per-step parity."""
    sa = scenes.cube_stack(nx=4, ny=2, nz=1)
    g, o = abd.Scene(sa), O.Scene(sa)
    g.partition(n_slabs=2, axis=0, planes=[-1.0], pd_kp=0.1, pd_kd=0.02, pd_smooth=0.5)
    planes = []
    for k in range(12):
        pl = g.partition_planes()
        planes.append(float(pl[0]))
        qo, vo = o.state()
        g.set_state(qo, vo)
        sg = g.step(abd.default_params())
        so = o.step(O.default_params(n_slabs=2, axis=0, planes=[float(pl[0])]))
        e = rel(g.state()[0], o.state()[0])
        assert e <= FP64_TOL, (k, e)
        assert (sg["admm_iters"], sg["newton_iters"]) == (so["admm_iters"], so["newton_iters"])
    print("planes", planes)
    # slab 0 starts with one column of cubes, slab 1 with three: the plane moves up
    assert planes[-1] > planes[0] + 0.05


def test_funnel_crop_fp64_parity():
    """A crop of the funnel workload (static funnel and chamber, two kinematic
    perforated turntables, a few spheres), two slabs: FP64 per-step parity."""
    sa = scenes.funnel_scene(n_bodies=8, level=1)
    worst, g, o = _run_pair(sa, 4, abd.default_params(), O.default_params(n_slabs=2, axis=0, planes=[0.0]),
                            FP64_TOL, partition=dict(n_slabs=2, axis=0, planes=[0.0]))
    print("worst rel err", worst)


def test_blocked_merges_split_fp64_parity():
    """One ADMM round allowed on a contact-rich two-slab pile with adaptive time
    stepping: blocked merges are retaken as two half steps, on the GPU as in the
    oracle (same statuses and ADMM rounds each step; q at the local solves' own
    resolution)."""
    sa = _sphere_admm_scene()
    g, o = abd.Scene(sa), O.Scene(sa)
    g.partition(n_slabs=2, axis=0)
    # With one ADMM round nothing refines a local solve: q is where each
    # partition's Newton stopped (Eq. 8's epsilon_N: ||dq||_inf < epsilon_N h l).
    # In this contact configuration the FP64 gradient's rounding, through the
    # barrier-stiff Hessian, leaves q determined only to ~7e-10 (the oracle's
    # own Newton stalls there: every trial raises E until alpha = 2^-32), and
    # the two sides may stop one Newton step apart; such a step is below
    # epsilon_N h l, and a split step compounds two half steps, so q is bounded
    # by 2 epsilon_N h l (l >= the box diagonal, 4.53).  The 1e-9 per-step bound
    # holds for the converged ADMM tests above.
    pg = abd.default_params(max_admm=1, dt_split_max=1)
    po = O.default_params(max_admm=1, dt_split_max=1, n_slabs=2, axis=0)
    tol_q = 2.0 * pg.newton_tol * pg.h * float(np.linalg.norm([2.4, 3.0, 2.4]))
    splits, worst, dn = 0, 0.0, 0
    for k in range(26):
        qo, vo = o.state()
        g.set_state(qo, vo)
        sg = g.step(pg)
        so = o.step(po)
        assert (sg["status"], sg["admm_iters"]) == (so["status"], so["admm_iters"]), (k, sg, so)
        dn = max(dn, abs(sg["newton_iters"] - so["newton_iters"]))
        e = rel(g.state()[0], o.state()[0])
        worst = max(worst, e)
        assert e <= tol_q, (k, e, tol_q)
        splits += sg["status"] == abd.DT_SPLIT
    print("worst rel err", worst, "bound", tol_q, "split steps", splits, "max newton count gap", dn)
    assert dn <= 2
    assert splits >= 1
