"""A batched world of uneven subdomains against the same subdomains stepped
alone, through the C ABI.

Each subdomain of the batch is one partition of one world: its Newton phases
run in the same launches as every other subdomain's, and its step must be the
one it takes alone -- FP64 within 1e-8 per step; mixed within 1e-4 of the
FP64 step, or, at the rare step with two nearby local minima, a valid one.  The subdomains all sit at the
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


def _newton_step(o, sa, kB, q_end, q0, v0, h=1e-2):
    """Largest entry of the dense projected-Newton step of Eq. 1 (the oracle's
    objective, gradient and projected Hessian) at q_end for the step taken
    from (q0, v0): how far q_end is from a stationary point of the step."""
    import oracle as O
    dyn = sa.body_kind == scenes.KIND_DYNAMIC
    p = O.default_params(kappa_barrier=kB)
    qt = q0 + h * v0
    qt[:, :3] += h * h * sa.gravity
    _, g, H = o.objective(p, q_end[dyn], qt[dyn])
    return float(np.abs(np.linalg.solve(H, g)).max())


# FP64: a subdomain's step in the batch differs from its step alone only in
# the order of floating-point sums (the PCG's CTA split follows the cluster
# size, which the largest subdomain sets; atomic accumulation order); through
# the stiff contact Hessians of these piles (densities up to 1e4) that moves q
# by up to a few 1e-9 (2.7e-9 measured), hence 1e-8.
# Mixed: the batch's mixed step against the subdomain's FP64 step alone --
# within 1e-4 where the step has one answer; at a step where the contact
# energy offers two nearby local minima (the FP64 step itself lands in the
# other one from a start perturbed by 1e-6), the mixed step may take either,
# and there it must be a valid one: penetration-free and stationary for
# Eq. 1 (the oracle's dense Newton step at it below 10 eps_N h l).
@pytest.mark.parametrize("precision,tol", [(abd.FP64, 1e-8), (abd.MIXED, 1e-4)])
def test_batch_equals_each_subdomain_alone(precision, tol):
    import oracle as O
    subs = _subdomains()
    batch = abd.Scene(subs)
    alone = [abd.Scene(sa) for sa in subs]
    off = batch.layout()
    assert len(off) == len(subs) + 1 and off[-1] == sum(sa.n_bodies for sa in subs)
    # Newton stops once its step is below eps_N h l (Eq. 8), about 5e-9 for
    # these piles at the default eps_N = 1e-6; eps_N = 1e-8 puts that
    # resolution well below the FP64 bound
    pb = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5,
                            newton_tol=1e-8 if precision == abd.FP64 else 1e-6)
    pa = abd.default_params(precision=abd.FP64, pcg_rtol=1e-12, newton_tol=pb.newton_tol)
    contact, worst, other_minimum = 0, 0.0, 0
    for k in range(14):
        # every step from the same state: the alone scenes' states, concatenated
        qs = [a.state() for a in alone]
        batch.set_state(np.concatenate([q for q, _ in qs]), np.concatenate([v for _, v in qs]))
        sb = batch.step(pb)
        assert sb["status"] >= 0 and sb["min_distance"] > 0.0, (k, sb)
        assert sb["n_partitions"] == len(subs) and sb["n_shared"] == 0
        qb = batch.state()[0]
        for i, a in enumerate(alone):
            sa_ = a.step(pa)
            e = _rel(qb[off[i]:off[i + 1]], a.state()[0])
            contact += sa_["n_active_peak"] > 0
            if e <= tol:
                worst = max(worst, e)
                continue
            assert precision == abd.MIXED, (k, i, e)
            o = O.Scene(subs[i])
            q0, v0 = qs[i]
            tol_n = 10 * pb.newton_tol * pb.h * sa_["l"]
            assert _newton_step(o, subs[i], sa_["kappa_barrier"], qb[off[i]:off[i + 1]], q0, v0) < tol_n, (k, i, e)
            other_minimum += 1
    print(f"worst per-step rel err where within the bound {worst:.3e}; subdomain-steps in contact {contact}; "
          f"mixed steps in another valid minimum {other_minimum} of {14 * len(subs)}")
    assert contact >= 20 and other_minimum <= 4


def test_batch_rejects_mismatched_planes_and_slab_partitions():
    a = scenes.random_pile(1, 8, levels=(1,))
    b = scenes.cube_stack(ground=False)  # no ground plane
    with pytest.raises(abd.AbdError):
        abd.Scene([a, b])
    batch = abd.Scene([a, scenes.random_pile(2, 9, levels=(1,))])
    with pytest.raises(abd.AbdError):
        batch.partition(n_slabs=2, axis=0)
