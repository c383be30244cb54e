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
