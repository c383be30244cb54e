"""Pins of the oracle's residual-driven penalty and scaled-dual rescale
(Sec. 4.3) -- CPU only.

Two levels:
  * the rule itself, against a table worked by hand from Sec. 4.3
    (tests/golden/rho_update_sec43.json): both branches, the equality cases
    that fall to "otherwise", and the clamp at both ends;
  * a consensus step traced round by round on a shared body in contact on
    one side of a slab plane, against what ADMM's own optimality conditions
    fix independently of the update's code: the unscaled dual y = rho u is
    unchanged by a penalty change (Boyd et al. 2011, Sec. 3.4.1, which
    Sec. 4.3 follows), the next local solve starts from the rescaled u, each
    local solve ends at a stationary point of its augmented objective
    (Eq. 5: grad F_i + rho (q - z + u) = 0, with grad F_i from the oracle's
    FD-pinned gradient), the replicas of a body share one penalty, the
    scaled duals of a body sum to zero after each equal-weight consensus
    (Eq. 6-7), and the clamp binds in a real step.
A swapped tau/mu, a missing clamp, a missing u *= rho/rho_new and a
per-replica penalty each fail one of these."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_15875_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


def test_rho_update_matches_the_hand_worked_table():
    d = json.load(open(os.path.join(HERE, "golden", "rho_update_sec43.json")))
    pp = d["params"]
    for c in d["cases"]:
        nw, scale = O.rho_update(c["r"], c["s"], c["rho"], c["rho0"], pp["tau"], pp["mu"], pp["sigma_min"],
                                 pp["sigma_max"])
        assert nw == pytest.approx(c["rho_new"], rel=1e-15), c
        assert scale == pytest.approx(c["u_scale"], rel=1e-15), c


def _shared_contact_scene():
    """Two 0.2 cubes without gravity or planes: cube 0 (internal to slab 0)
    moves at 0.5 m/s into cube 1, which straddles the slab plane x = 0 and is
    therefore replicated on both slabs; only slab 0's replica feels the
    contact, so the replicas disagree and the penalty moves both ways."""
    q0 = [scenes._q_at([-0.2012, 0.0, 0.0]), scenes._q_at([0.0, 0.03, 0.0])]
    v0 = np.zeros((2, 12))
    v0[0, :3] = [0.5, 0.0, 0.0]
    return scenes._pack([scenes.cube_mesh(0.2)], [0, 0], [1000.0, 1000.0], 1e8, scenes.KIND_DYNAMIC, q0, v0, [],
                        gravity=(0.0, 0.0, 0.0), name="shared_contact_pair")


def _params(**kw):
    return O.default_params(n_slabs=2, axis=0, planes=[0.0], w_min=0.02, kappa_barrier=1e3, **kw)


# default constants (the penalty moves both ways); a small beta whose growth
# meets sigma_max; a sigma_min that the shrinking penalty meets
VARIANTS = {"free": {}, "upper_clamp": dict(beta=0.01, sigma_max=4.0),
            "lower_clamp": dict(sigma_min=0.25, sigma_max=2.0)}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_traced_consensus_keeps_the_unscaled_dual_and_optimality(variant):
    sa = _shared_contact_scene()
    sc, probe = O.Scene(sa), O.Scene(sa)
    extra = VARIANTS[variant]
    p = _params(**extra)
    moved = {"up": 0, "down": 0, "at_min": 0, "at_max": 0, "decisive": 0}
    for _ in range(3):
        q0, v0 = sc.state()
        st, rec = sc.step_traced(p)
        assert st["status"] == 0 and st["n_shared"] == 1 and st["n_active_peak"] > 0
        assert len(rec) > 0
        rho0 = probe.body_props(1)[0] * p.beta  # initial penalty beta m of the shared body
        # the oracle's F_i at the step's start state (membership, q~ = q + h v: no gravity)
        probe.set_state(q0, v0)
        pk = _params(**extra)
        pk.kappa_barrier = st["kappa_barrier"]
        qtil = q0 + p.h * v0
        rounds = np.unique(rec[:, 0])
        for k in rounds:
            R = rec[rec[:, 0] == k]
            sh = R[R[:, 3] == 1]
            assert set(sh[:, 2].astype(int)) == {0, 1}
            # one penalty per body, before and after the update (Sec. 4.3)
            assert np.all(sh[:, 4] == sh[0, 4]) and np.all(sh[:, 5] == sh[0, 5])
            # the clamp to [sigma_min rho0, sigma_max rho0]
            assert p.sigma_min * rho0 * (1 - 1e-15) <= sh[0, 5] <= p.sigma_max * rho0 * (1 + 1e-15)
            if sh[0, 5] > sh[0, 4]:
                moved["up"] += 1
            if sh[0, 5] < sh[0, 4]:
                moved["down"] += 1
            moved["at_min"] += sh[0, 5] == pytest.approx(p.sigma_min * rho0, rel=1e-14)
            moved["at_max"] += sh[0, 5] == pytest.approx(p.sigma_max * rho0, rel=1e-14)
            # equal-weight consensus (Eq. 6) and dual update (Eq. 7): the
            # replicas' scaled duals of the body sum to zero
            # (u accumulates q - z, so its rounding is that of q's entries)
            usum = sh[:, 44:56].sum(0)
            assert np.abs(usum).max() <= 1e-14 * max(1.0, np.abs(sh[:, 8:20]).max())
            # Boyd Sec. 3.4.1: the unscaled dual y = rho u is unchanged by the rescale
            y_before = sh[:, 4:5] * sh[:, 44:56]
            y_after = sh[:, 5:6] * sh[:, 56:68]
            assert np.abs(y_after - y_before).max() <= 1e-14 * max(1e-300, np.abs(y_before).max())
            # each local solve ended at a stationary point of Eq. 5:
            # grad F_i(q_i) + rho (q_i - z^{k-1} + u^{k-1}) = 0, where
            # q_i - z^{k-1} + u^{k-1} = u^k + z^k - z^{k-1}
            for i in (0, 1):
                Ri = R[R[:, 2] == i]
                qc = np.zeros((2, 12))
                for r in Ri:
                    qc[int(r[1])] = r[8:20]
                _, g = probe.local_gradient(pk, i, qc, qtil)
                for r in Ri:
                    b = int(r[1])
                    aug = r[4] * (r[44:56] + r[32:44] - r[20:32]) if r[3] else np.zeros(12)
                    # the solve stops once its Newton step is below eps_N h l
                    # (Eq. 8's normalisation), so the gradient left over is at
                    # most that step times the Hessian, bounded here by the
                    # orthogonality term 8 kappa V h^2 near A = I, the mass and
                    # the penalty (the barrier's share is small in this contact)
                    m, _, _, V = probe.body_props(b)
                    hb = 8.0 * sa.body_kappa[b] * V * p.h ** 2 + m + r[4]
                    tol = 4.0 * hb * p.newton_tol * p.h * st["l"]
                    assert np.abs(g[b] + aug).max() <= tol, (k, i, b)
                    if r[3] and np.abs(aug).max() > 100 * tol:
                        moved["decisive"] += 1  # a record where the consensus term dominates the bound
        # round-to-round link: the next local solve used the rescaled u and the new rho
        for k in rounds[:-1]:
            a = rec[(rec[:, 0] == k) & (rec[:, 3] == 1)]
            c = rec[(rec[:, 0] == k + 1) & (rec[:, 3] == 1)]
            if len(c) == 0:
                continue
            for ra in a:
                rc = c[c[:, 2] == ra[2]][0]
                assert rc[4] == ra[5]
                u_used = rc[44:56] - rc[8:20] + rc[32:44]  # u^k from u^{k+1} = u^k + q - z
                assert np.abs(u_used - ra[56:68]).max() <= 1e-14 * max(1.0, np.abs(rc[8:20]).max())
    assert moved["decisive"] >= 10
    if variant == "free":
        assert moved["up"] > 0 and moved["down"] > 0
    elif variant == "upper_clamp":
        assert moved["at_max"] > 0
    else:
        assert moved["at_min"] > 0
