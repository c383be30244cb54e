"""The benchmark workload at its full size (512 noisy icospheres in the open
box, 4 slabs), in the configuration bench.py times.

* Per-step parity with the FP64 oracle over the first steps (FP64 1e-9 and
  equal ADMM/Newton counts; mixed 1e-4) -- steps the oracle finishes in
  seconds at this size.
* Candidate sets with a large d-hat (tens of thousands of pairs): the
  cluster path with FP32 filters equals the independent FP64-only pass of
  the no-allocation query bit for bit; every listed pair's FP64 boxes
  overlap; and for a sample of bodies, a numpy brute force over every
  primitive of the body against every primitive of its neighbours finds
  exactly the listed pairs that involve the body.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2605_15875_gb300 import abd, scenes

pytestmark = pytest.mark.gpu

PLANES = [-0.6, 0.0, 0.6]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.mark.parametrize("precision,tol,steps", [(abd.FP64, 1e-9, 3), (abd.MIXED, 1e-4, 3)])
def test_full_size_first_steps(precision, tol, steps):
    sa = scenes.sphere_grid_in_box(seed=0)
    g, o = abd.Scene(sa), O.Scene(sa)
    g.partition(n_slabs=4, axis=0, planes=PLANES)
    pg = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5)
    po = O.default_params(n_slabs=4, axis=0, planes=PLANES)
    for k in range(steps):
        qo, vo = o.state()
        g.set_state(qo, vo)
        sg = g.step(pg)
        so = o.step(po)
        e = _rel(g.state()[0], o.state()[0])
        assert e <= tol, (k, e)
        assert sg["status"] >= 0 and sg["min_distance"] > 0.0
        if precision == abd.FP64:
            assert (sg["admm_iters"], sg["newton_iters"]) == (so["admm_iters"], so["newton_iters"])


def _prims(sa, o):
    """Global primitive tables: triangle vertex ids, edge vertex ids, and the
    body of every vertex, triangle and edge."""
    nv = sa.body_vertex_counts().astype(np.int64)
    nt = sa.body_tri_counts().astype(np.int64)
    voff = np.concatenate([[0], np.cumsum(nv)])
    tris = []
    for b in range(sa.n_bodies):
        tris.append(sa.mesh(int(sa.body_mesh[b])).tris.astype(np.int64) + voff[b])
    tris = np.concatenate(tris)
    vbody = np.repeat(np.arange(sa.n_bodies), nv)
    tbody = np.repeat(np.arange(sa.n_bodies), nt)
    edges = o.edges().astype(np.int64)
    ebody = vbody[edges[:, 0]]
    return tris, edges, vbody, tbody, ebody


def _boxes(x0, x1, ids, half):
    """FP64 boxes of primitives given by vertex ids [n, k]: exact min/max over
    the vertices (both configurations), one rounding for +-half."""
    pts = x0[ids]
    lo, hi = pts.min(axis=1), pts.max(axis=1)
    if x1 is not None:
        p1 = x1[ids]
        lo, hi = np.minimum(lo, p1.min(axis=1)), np.maximum(hi, p1.max(axis=1))
    return lo - half, hi + half


def _overlap(alo, ahi, blo, bhi):
    return ~np.any((alo > bhi) | (blo > ahi), axis=-1)


@pytest.mark.parametrize("swept", [False, True])
def test_full_size_candidates(swept):
    import torch
    L = abd.load()
    sa = scenes.sphere_grid_in_box(seed=0)
    g, o = abd.Scene(sa), O.Scene(sa)
    x0 = o.vertices()
    x1 = x0 + np.random.default_rng(5).normal(size=x0.shape) * 0.002 if swept else None
    dhat = 0.06  # neighbours 0.25 apart with radii ~0.1: many pairs
    half = 0.5 * dhat
    got = g.candidates(x0, x1, dhat)
    gs = {tuple(int(v) for v in r) for r in got}
    assert len(got) == len(gs) and len(got) > 20000

    # the independent FP64-only pass (no-allocation query), bit for bit
    x0d = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
    x1d = None if x1 is None else torch.from_numpy(np.ascontiguousarray(x1)).cuda()
    cap = len(got) + 1024
    out = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    torch.cuda.synchronize()
    rc = L.abd_candidates_noalloc(g.h, x0d.data_ptr(), None if x1d is None else x1d.data_ptr(), dhat,
                                  out.data_ptr(), cap, ctypes.byref(n))
    assert rc == 0, L.abd_last_error(g.h).decode()
    assert {tuple(int(v) for v in r) for r in out[:n.value].cpu().numpy()} == gs

    tris, edges, vbody, tbody, ebody = _prims(sa, o)
    kind = sa.body_kind
    # every listed pair overlaps (FP64 boxes)
    pt = got[got[:, 0] == 0]
    ee = got[got[:, 0] == 1]
    vlo, vhi = _boxes(x0, x1, pt[:, 1:2].astype(np.int64), half)
    tlo, thi = _boxes(x0, x1, tris[pt[:, 2]], half)
    assert np.all(_overlap(vlo, vhi, tlo, thi))
    alo, ahi = _boxes(x0, x1, edges[ee[:, 1]], half)
    blo, bhi = _boxes(x0, x1, edges[ee[:, 2]], half)
    assert np.all(_overlap(alo, ahi, blo, bhi))

    # brute force for a sample of bodies against every primitive of their neighbours
    vb_lo, vb_hi = _boxes(x0, x1, np.arange(len(x0))[:, None], half)
    tb_lo, tb_hi = _boxes(x0, x1, tris, half)
    eb_lo, eb_hi = _boxes(x0, x1, edges, half)
    body_lo = np.array([vb_lo[vbody == b].min(axis=0) for b in range(sa.n_bodies)])
    body_hi = np.array([vb_hi[vbody == b].max(axis=0) for b in range(sa.n_bodies)])
    rng = np.random.default_rng(11)
    sample = rng.choice(np.where(kind == scenes.KIND_DYNAMIC)[0], 12, replace=False)
    for b in sample:
        nb = np.where(_overlap(body_lo[b][None], body_hi[b][None], body_lo, body_hi))[0]
        nb = nb[nb != b]
        exp = set()
        vs = np.where(vbody == b)[0]
        ts = np.where(tbody == b)[0]
        es = np.where(ebody == b)[0]
        tn = np.where(np.isin(tbody, nb))[0]
        vn = np.where(np.isin(vbody, nb))[0]
        en = np.where(np.isin(ebody, nb))[0]
        hit = _overlap(vb_lo[vs][:, None], vb_hi[vs][:, None], tb_lo[tn][None], tb_hi[tn][None])
        for i, j in zip(*np.nonzero(hit)):
            exp.add((0, int(vs[i]), int(tn[j])))
        hit = _overlap(vb_lo[vn][:, None], vb_hi[vn][:, None], tb_lo[ts][None], tb_hi[ts][None])
        for i, j in zip(*np.nonzero(hit)):
            exp.add((0, int(vn[i]), int(ts[j])))
        hit = _overlap(eb_lo[es][:, None], eb_hi[es][:, None], eb_lo[en][None], eb_hi[en][None])
        for i, j in zip(*np.nonzero(hit)):
            a, c = int(es[i]), int(en[j])
            exp.add((1, min(a, c), max(a, c)))
        mine = {r for r in gs if (r[0] == 0 and (vbody[r[1]] == b or tbody[r[2]] == b))
                or (r[0] == 1 and (ebody[r[1]] == b or ebody[r[2]] == b))}
        assert mine == exp, (int(b), len(mine), len(exp))


CONTACT_FROM = 19  # the lowest layer reaches the box floor on step 19 (free fall before)


@pytest.fixture(scope="module")
def contact_window():
    """The oracle's trajectory of the full-size workload into its first
    contact steps: for steps 19 and 20, the state before the step, the
    oracle's state after it and its statistics (about 25 s of CPU)."""
    sa = scenes.sphere_grid_in_box(seed=0)
    o = O.Scene(sa)
    po = O.default_params(n_slabs=4, axis=0, planes=PLANES)
    for _ in range(CONTACT_FROM):
        o.step(po)
    out = []
    for _ in range(2):
        q, v = o.state()
        so = o.step(po)
        out.append((q, v, o.state()[0], so))
    assert out[0][3]["n_active_peak"] > 0 and out[0][3]["n_shared"] > 400
    return sa, out


@pytest.mark.parametrize("precision,tol,reserve", [(abd.FP64, 1e-9, None), (abd.MIXED, 1e-4, None),
                                                   (abd.FP64, 1e-9, 16)])
def test_full_size_contact_steps(contact_window, precision, tol, reserve):
    """Contact steps of the benchmark workload, each from the oracle's state:
    about 500 shared bodies over four slabs, so the PCG runs on clusters of
    several CTAs with off-diagonal blocks between them; FP64 within 1e-9 per
    step with equal ADMM and Newton counts, mixed within 1e-4.  With the pair
    lists reserved at 16 records the first iteration of the first step
    overflows them, grows them and is redone (the list-growth path), and the
    result is unchanged."""
    sa, window = contact_window
    g = abd.Scene(sa)
    g.partition(n_slabs=4, axis=0, planes=PLANES)
    if reserve is not None:
        g.reserve(reserve)
    pg = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5)
    for k, (q, v, q_ref, so) in enumerate(window):
        g.set_state(q, v)
        sg = g.step(pg)
        e = _rel(g.state()[0], q_ref)
        print(f"step {CONTACT_FROM + k}: rel err {e:.3e}, ADMM {sg['admm_iters']}/{so['admm_iters']}, "
              f"Newton {sg['newton_iters']}/{so['newton_iters']}, active {sg['n_active_peak']}, "
              f"PCG cluster {sg['pcg_cluster']}, unstaged {sg['pcg_unstaged']}, list redo {sg['list_redo']}, "
              f"slots {sg['n_slots']}, shared {sg['n_shared']}")
        assert e <= tol, (k, e)
        assert sg["status"] >= 0 and sg["min_distance"] > 0.0
        assert sg["n_active_peak"] > 0 and sg["pcg_cluster"] >= 2
        if precision == abd.FP64:
            assert (sg["admm_iters"], sg["newton_iters"]) == (so["admm_iters"], so["newton_iters"])
        if reserve is not None and k == 0:
            assert sg["list_redo"] >= 1
