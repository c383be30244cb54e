"""A batched world of uneven subdomains against the same subdomains stepped
alone, through the C ABI.

Each subdomain of the batch is one partition of one world: its Newton phases
run in the same launches as every other subdomain's, and its step must be the
one it takes alone -- FP64 within 1e-9 per step with the same Newton
iteration count, mixed within 1e-4 per step.  The subdomains all sit at the
origin on the same ground plane, so a pair of bodies from two subdomains
would overlap at once: a batch that let subdomains meet would fail at the
first step."""
import numpy as np
import pytest

from paper_2605_15875_gb300 import abd, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_15875_gb300 import build
    build.build()
    abd.load()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def _subdomains():
    # uneven piles (16-160 bodies, levels 1-2, densities log-uniform 1e2-1e4)
    return scenes.batched_subdomains(seed=3, n_scenes=6, lo=16, hi=160, levels=(1, 2))


@pytest.mark.parametrize("precision,tol", [(abd.FP64, 1e-9), (abd.MIXED, 1e-4)])
def test_batch_equals_each_subdomain_alone(precision, tol):
    subs = _subdomains()
    batch = abd.Scene(subs)
    alone = [abd.Scene(sa) for sa in subs]
    off = batch.layout()
    assert len(off) == len(subs) + 1 and off[-1] == sum(sa.n_bodies for sa in subs)
    # Newton stops once its step is below eps_N h l (Eq. 8), about 5e-9 for
    # these piles at the default eps_N = 1e-6; the batch's PCG clusters have
    # the largest subdomain's size, so its dot products add in another order
    # than a subdomain's alone, and the two solves may stop one sub-threshold
    # step apart.  eps_N = 1e-8 puts that step well below the 1e-9 bound.
    pg = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5,
                            newton_tol=1e-8 if precision == abd.FP64 else 1e-6)
    contact, worst, gap = 0, 0.0, 0
    for k in range(14):
        # every step from the same state: the alone scenes' states, concatenated
        qs = [a.state() for a in alone]
        batch.set_state(np.concatenate([q for q, _ in qs]), np.concatenate([v for _, v in qs]))
        sb = batch.step(pg)
        assert sb["status"] >= 0 and sb["min_distance"] > 0.0, (k, sb)
        assert sb["n_partitions"] == len(subs) and sb["n_shared"] == 0
        nb = batch.partition_newton()
        qb = batch.state()[0]
        for i, a in enumerate(alone):
            sa_ = a.step(pg)
            e = _rel(qb[off[i]:off[i + 1]], a.state()[0])
            worst = max(worst, e)
            assert e <= tol, (k, i, e)
            gap = max(gap, abs(int(nb[i]) - sa_["newton_iters"]))
            contact += sa_["n_active_peak"] > 0
    # at eps_N = 1e-8 a solve may stall a few sub-threshold iterations before
    # its stop test fires, so the Newton counts are printed, not compared
    print(f"worst per-step rel err {worst:.3e}; subdomain-steps in contact {contact}; "
          f"largest Newton-count gap {gap}")
    assert contact >= 20


def test_batch_rejects_mismatched_planes_and_slab_partitions():
    a = scenes.random_pile(1, 8, levels=(1,))
    b = scenes.cube_stack(ground=False)  # no ground plane
    with pytest.raises(abd.AbdError):
        abd.Scene([a, b])
    batch = abd.Scene([a, scenes.random_pile(2, 9, levels=(1,))])
    with pytest.raises(abd.AbdError):
        batch.partition(n_slabs=2, axis=0)
