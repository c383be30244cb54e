"""abd_candidates_noalloc against abd_candidates, through the C ABI.

The no-allocation entry point exists for callers that cannot allocate device
memory (a plugin whose host framework owns the GPU's memory budget, or a
latency-critical loop that cannot absorb an allocation's device-wide
synchronisation).  Here the test allocates the input and output buffers with
torch, as such a caller would hand over buffers it already owns, and checks
that two calls in a row (static set, then swept set with another dhat)
return exactly the candidate sets of the allocating entry point: candidate
work is integer work, compared bit for bit."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ABD_E_PAIR_OVERFLOW = -4  # include/abd.h


def _as_set(a):
    return {tuple(int(v) for v in r) for r in a}


def test_candidates_noalloc_matches_allocating_entry_point():
    import torch
    from paper_2605_15875_gb300 import abd, build, scenes

    build.build()
    L = abd.load()
    torch.cuda.set_device(0)
    sa = scenes.sphere_grid_in_box(n=3, ny=2, nz=2, level=2, spacing=0.2004, lowest=0.1003)
    sc = abd.Scene(sa)
    x0 = np.ascontiguousarray(sa.world_vertices())
    x1 = np.ascontiguousarray(x0 + np.random.default_rng(3).normal(size=x0.shape) * 0.004)
    x0d = torch.from_numpy(x0).cuda()
    x1d = torch.from_numpy(x1).cuda()
    cap = 1 << 18
    out = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for xa, xb, dhat in ((x0d, None, 1e-3), (x0d, x1d, 4e-3)):
        n = ctypes.c_int64(-1)
        rc = L.abd_candidates_noalloc(sc.h, xa.data_ptr(), None if xb is None else xb.data_ptr(), dhat,
                                      out.data_ptr(), cap, ctypes.byref(n))
        assert rc == 0, L.abd_last_error(sc.h).decode()
        assert 100 < n.value <= cap
        got = out[:n.value].cpu().numpy()
        ref = sc.candidates(x0, None if xb is None else x1, dhat)
        assert len(got) == len(ref)
        assert _as_set(got) == _as_set(ref)


def test_candidates_noalloc_truncates_at_cap_and_reports_the_full_count():
    """More candidates than `cap`: the full count comes back in n_out, the
    first `cap` rows are distinct members of the allocating entry point's
    set, and nothing past `cap` is written (a sentinel stays in place)."""
    import torch
    from paper_2605_15875_gb300 import abd, build, scenes

    build.build()
    L = abd.load()
    torch.cuda.set_device(0)
    sa = scenes.sphere_grid_in_box(n=3, ny=2, nz=2, level=2, spacing=0.2004, lowest=0.1003)
    sc = abd.Scene(sa)
    x0 = np.ascontiguousarray(sa.world_vertices())
    ref = _as_set(sc.candidates(x0, None, 1e-3))
    assert len(ref) > 300
    cap = len(ref) // 3
    out = torch.full((cap + 256, 3), -7, dtype=torch.int32, device="cuda")
    x0d = torch.from_numpy(x0).cuda()
    torch.cuda.synchronize()
    for _ in range(2):
        n = ctypes.c_int64(-1)
        rc = L.abd_candidates_noalloc(sc.h, x0d.data_ptr(), None, 1e-3, out.data_ptr(), cap, ctypes.byref(n))
        assert rc == 0, L.abd_last_error(sc.h).decode()
        assert n.value == len(ref)
        got = out.cpu().numpy()
        head = _as_set(got[:cap])
        assert len(head) == cap and head <= ref
        assert (got[cap:] == -7).all()
    assert torch.cuda.current_device() == 0


def test_candidates_noalloc_reports_pair_overflow():
    """3000 cubes whose boxes all overlap give 4.5 million overlapping body
    pairs, beyond the scratch array's (32 MiB - 64 B x 3000) / 8 = 4.17
    million: the call returns ABD_E_PAIR_OVERFLOW with a message, writes
    nothing to the output, and a following call that fits still works."""
    import torch
    from paper_2605_15875_gb300 import abd, build, scenes

    build.build()
    L = abd.load()
    torch.cuda.set_device(0)
    nb = 3000
    q0 = [scenes._q_at(np.array([3.0 * i, 0.0, 0.0])) for i in range(nb)]
    sa = scenes._pack([scenes.cube_mesh(1.0)], [0] * nb, 1000.0, 1e8, scenes.KIND_DYNAMIC, q0, None, [],
                      gravity=(0.0, 0.0, 0.0), name="coincident_cubes")
    sc = abd.Scene(sa)
    xs = np.ascontiguousarray(sa.world_vertices())
    same = np.ascontiguousarray(np.tile(xs[:8], (nb, 1)))  # every cube at the first cube's place
    cap = 1024
    out = torch.full((cap, 3), -7, dtype=torch.int32, device="cuda")
    for x, expect_rc in ((same, ABD_E_PAIR_OVERFLOW), (xs, 0)):
        xd = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        n = ctypes.c_int64(-1)
        rc = L.abd_candidates_noalloc(sc.h, xd.data_ptr(), None, 1e-3, out.data_ptr(), cap, ctypes.byref(n))
        assert rc == expect_rc, (rc, L.abd_last_error(sc.h).decode())
        if rc:
            assert "overlapping body pairs" in L.abd_last_error(sc.h).decode()
            assert n.value == -1
            assert (out.cpu().numpy() == -7).all()
        else:
            assert n.value == 0  # cubes 3 apart: nothing overlaps
    assert torch.cuda.current_device() == 0
