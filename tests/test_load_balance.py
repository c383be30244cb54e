"""Control-based load balancing of the slab planes (Sec. 5.2), host law on
CPU through the C ABI (abd_pd_update is a pure host function)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def abd():
    from paper_2605_15875_gb300 import abd as A, build
    build.build()
    A.load()
    return A


def test_pd_law_closed_form(abd):
    rng = np.random.default_rng(3)
    for n in (2, 3, 5):
        tau = rng.uniform(0.1, 10.0, n)
        Tp = rng.uniform(-0.5, 0.5, n - 1)
        kp, kd = 0.07, 0.02
        delta, T = abd.pd_update(tau, Tp, kp, kd)
        eta = tau[:-1] / tau[1:]
        T_ref = (eta - 1.0) / (eta + 1.0)  # the paper's normalisation
        assert np.allclose(T, T_ref, rtol=0, atol=1e-15)
        assert np.allclose(delta, -(kp * T_ref + kd * (T_ref - Tp)), rtol=0, atol=1e-15)


def test_pd_law_direction_and_balance(abd):
    # slab 0 slower: its upper plane moves down (slab 0 shrinks)
    d, T = abd.pd_update([2.0, 1.0], None, 0.1, 0.0)
    assert T[0] > 0 and d[0] < 0
    # slab 1 slower: the plane moves up
    d, T = abd.pd_update([1.0, 3.0], None, 0.1, 0.0)
    assert T[0] < 0 and d[0] > 0
    # balanced, or no work: no move
    for tau in ([4.0, 4.0], [0.0, 0.0]):
        d, T = abd.pd_update(tau, None, 0.1, 0.05)
        assert d[0] == 0.0 and T[0] == 0.0
    # derivative term alone acts on the change of T
    d, T = abd.pd_update([2.0, 1.0], [1.0 / 3.0], 0.0, 0.5)
    assert abs(d[0]) < 1e-16
