"""Step statuses through the C ABI against the oracle: the Newton iteration
cap (a local solve that spends max_newton iterations without meeting
Eq. 8's epsilon_N reports NEWTON_MAXITER; one that meets it on its last
allowed iteration is OK), and a scene without unknowns (every body static)
that steps to itself."""
import numpy as np
import pytest

import oracle as O
from paper_2605_15875_gb300 import abd, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_15875_gb300 import build
    build.build()
    abd.load()


def test_newton_cap_status_matches_oracle():
    sa = scenes.cube_stack()
    o = O.Scene(sa)
    for _ in range(40):  # the first step with contact Newton work
        q0, v0 = o.state()
        st = o.step(O.default_params())
        n = st["newton_iters"]
        if n > 2:
            break
    assert n > 2
    g = abd.Scene(sa)
    for cap in (n, n - 1):
        o.set_state(q0, v0)
        g.set_state(q0, v0)
        so = o.step(O.default_params(max_newton=cap))
        sg = g.step(abd.default_params(max_newton=cap))
        assert (sg["status"], sg["newton_iters"]) == (so["status"], so["newton_iters"]), (cap, sg, so)
        qg, qo = g.state()[0], o.state()[0]
        assert np.abs(qg - qo).max() / max(1.0, np.abs(qo).max()) <= 1e-9
    assert sg["status"] == abd.NEWTON_MAXITER
    g.close()


def test_static_only_scene_matches_oracle():
    """Degenerate case: every body static, so a step has no unknowns; both
    sides report OK without Newton work and leave the state bit for bit."""
    sa = scenes.static_only()
    for slabs in (1, 4):
        g, o = abd.Scene(sa), O.Scene(sa)
        g.partition(n_slabs=slabs, axis=0)
        q0, v0 = g.state()
        for _ in range(3):
            sg = g.step(abd.default_params())
            so = o.step(O.default_params(n_slabs=slabs, axis=0))
            for k in ("status", "admm_iters", "newton_iters", "min_distance"):
                assert sg[k] == so[k], (k, sg, so)
        q, v = g.state()
        assert np.array_equal(q, q0) and np.array_equal(v, v0)
        assert np.array_equal(q, o.state()[0])
        g.close()
