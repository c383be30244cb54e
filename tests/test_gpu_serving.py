"""Serving runtime on the GPU: a request's result is the same alone and in a
mix of concurrent requests (within the parity tolerance of its precision),
admission under a tiny HBM budget still completes every request, and
partition membership agrees with the body masks."""
import numpy as np
import pytest

from paper_2605_15875_gb300 import abd, scenes

pytestmark = pytest.mark.gpu


def _mix():
    return [scenes.cube_stack(seed=1, nx=2, ny=2, nz=1),
            scenes.random_pile(7, 12, levels=(1,)),
            scenes.cube_stack(seed=2, nx=1, ny=3, nz=1),
            scenes.random_pile(9, 20, levels=(1, 2))]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def _run(server, sas, steps, params, together):
    tickets = []
    if together:
        tickets = [server.submit(sa, steps, params) for sa in sas]
        infos = [server.wait(t) for t in tickets]
    else:
        infos = []
        for sa in sas:
            t = server.submit(sa, steps, params)
            infos.append(server.wait(t))
            tickets.append(t)
    return [server.result(t)[0] for t in tickets], infos


@pytest.mark.parametrize("precision,tol", [(abd.FP64, 1e-9), (abd.MIXED, 1e-4)])
def test_result_same_alone_and_in_mix(precision, tol):
    sas = _mix()
    p = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5,
                           kappa_barrier=1e5)
    alone_srv = abd.Server(n_streams=1)
    alone, ia = _run(alone_srv, sas, 6, p, together=False)
    alone_srv.close()
    mix_srv = abd.Server(n_streams=4)
    mixed, im = _run(mix_srv, sas, 6, p, together=True)
    mix_srv.close()
    for qa, qm, a, m in zip(alone, mixed, ia, im):
        assert a["status"] >= 0 and m["status"] >= 0
        assert a["steps_done"] == 6 and m["steps_done"] == 6
        assert _rel(qm, qa) <= tol


def test_alone_equals_direct_scene():
    """A served request equals stepping the scene directly through abd_step."""
    sa = scenes.random_pile(7, 12, levels=(1,))
    p = abd.default_params(precision=abd.FP64, kappa_barrier=1e5)
    srv = abd.Server(n_streams=2)
    t = srv.submit(sa, 5, p)
    srv.wait(t)
    qs, _ = srv.result(t)
    srv.close()
    sc = abd.Scene(sa)
    for _ in range(5):
        sc.step(p)
    qd, _ = sc.state()
    assert _rel(qs, qd) <= 1e-9


def test_tiny_budget_admits_one_at_a_time_and_completes():
    sas = _mix()
    srv = abd.Server(n_streams=3, hbm_budget_bytes=1)
    ts = [srv.submit(sa, 2) for sa in sas]
    infos = [srv.wait(t) for t in ts]
    lat = [srv.latencies(t) for t in ts]
    srv.close()
    assert all(i["state"] == abd.REQ_DONE and i["status"] >= 0 and i["steps_done"] == 2 for i in infos)
    assert all(len(x) == 2 for x in lat)
    # later requests waited for memory held by earlier ones
    assert max(i["queue_ms"] for i in infos) > 0.0


def test_partition_get_matches_masks():
    sa = scenes.sphere_grid_in_box(seed=0, n=4, ny=2, nz=2)
    sc = abd.Scene(sa)
    sc.partition(n_slabs=2, axis=0, planes=[0.0])
    st = sc.step(abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5))
    dyn = np.where(sa.body_kind == scenes.KIND_DYNAMIC)[0]
    seen = np.zeros(sa.n_bodies, dtype=np.int64)
    for part in range(st["n_partitions"]):
        bodies, shared = sc.partition_get(part)
        seen[bodies] += 1
        assert set(shared.tolist()) <= set(bodies.tolist())
    assert np.all(seen[dyn] >= 1)
    n_shared = sum(len(sc.partition_get(p)[1]) for p in range(st["n_partitions"]))
    assert n_shared == int(np.sum(seen[seen > 1]))


@pytest.mark.parametrize("budget", [0, 1])
def test_resident_scene_continues_across_requests(budget):
    """Keyed requests advance a resident scene: three requests of 2 + 3 + 1
    steps per key end where 6 steps of the scene stepped directly end (FP64
    1e-9), for several keys whose requests interleave.  With a 1-byte budget
    every admission evicts the idle resident scenes (state kept on the host,
    scene rebuilt at its next request), which changes nothing in the result."""
    sas = _mix()
    p = abd.default_params(precision=abd.FP64, kappa_barrier=1e5)
    direct = []
    for sa in sas:
        sc = abd.Scene(sa)
        for _ in range(6):
            sc.step(p)
        direct.append(sc.state()[0])
        sc.close()
    srv = abd.Server(n_streams=3, hbm_budget_bytes=budget)
    last = {}
    for chunk, n in enumerate((2, 3, 1)):
        for key, sa in enumerate(sas, start=1):
            last[key] = srv.submit(sa if chunk == 0 else None, n, p, key=key)
    for key in last:
        info = srv.wait(last[key])
        assert info["status"] >= 0 and info["steps_done"] == 1
    for key, ref in zip(last, direct):
        q, _ = srv.result(last[key])
        assert _rel(q, ref) <= 1e-9, key
        srv.release(key)
    with pytest.raises(abd.AbdError):
        srv.submit(None, 1, p, key=99)  # a key's first request must describe its scene
    srv.close()
