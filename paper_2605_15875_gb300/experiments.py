"""Penalty-parameter experiments of the mass-aware consensus (Sec. 4.3, Sec. 6.2):
for a sweep of the initial factor beta (rho_b^0 = beta m_b) and of the body
density, run a contact-rich pile on two slabs with the residual-driven
adaptation and with a fixed penalty, and report the mean ADMM rounds per
step and the mean squared error of q against the single-partition solve.
Per step (default): before every step the two-slab scene takes the
single-partition scene's state, so the error is that of one step from the
same q^t (the paper's q* comparison); with --trajectory both run freely and
the error is taken after the last step (dominated by the pile's chaotic
divergence).

With --hetero it runs the material-heterogeneity comparison instead (Sec. 6.2,
Table 2): the 200-body pile with three (mass, stiffness) groups against its
uniform baseline, on two slabs and on one partition, FP64, reporting the mean
ADMM rounds and Newton iterations per step.

  python -m paper_2605_15875_gb300.experiments [--steps 30] [--start 0] [--quick] [--trajectory]
  python -m paper_2605_15875_gb300.experiments --funnel --steps 8 --betas 0.01,1,100 --densities 10,1000,100000
  python -m paper_2605_15875_gb300.experiments --hetero [--steps 40]

--funnel swaps the 64-sphere box pile for 512 level-2 spheres packed in the
funnel of the funnel-and-turntables workload, split at x = 0.

Prints one JSON object per configuration and a summary line."""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def pile(density: float, funnel: bool = False):
    from . import scenes
    if funnel:
        # 512 level-2 spheres packed in the funnel above the turntables (the
        # paper's penalty study uses a 512-body two-worker scene, Sec. 6.2)
        return scenes.funnel_scene(n_bodies=512, level=2, density=density, dense=True)
    sa = scenes.sphere_grid_in_box(seed=0, n=4, ny=4, nz=4, level=1, lowest=0.12, spacing=0.25,
                                   box=(1.2, 2.0, 1.2), density=density)
    return sa


def run(sa, steps, params, n_slabs):
    from . import abd
    sc = abd.Scene(sa)
    if n_slabs > 1:
        sc.partition(n_slabs=n_slabs, axis=0, planes=[0.0])
    admm, newton, worst = [], [], 0
    for _ in range(steps):
        st = sc.step(params)
        admm.append(st["admm_iters"])
        newton.append(st["newton_iters"])
        worst = max(worst, st["status"])
    q, _ = sc.state()
    sc.close()
    return q, float(np.mean(admm)), float(np.mean(newton)), worst


def ref_trajectory(sa, start, steps, params):
    """Single-partition states: `start` untimed steps into the pile (so the
    measured steps begin in contact), then (q^t, v^t, q^{t+1}) for `steps`
    steps.  Computed once per density and shared by every (beta, rho mode)."""
    from . import abd
    ref = abd.Scene(sa)
    for _ in range(start):
        ref.step(params)
    out = []
    for _ in range(steps):
        q0, v0 = ref.state()
        ref.step(params)
        out.append((q0, v0, ref.state()[0]))
    ref.close()
    return out


def run_per_step(sa, traj, params):
    """Two-slab steps, each from the single-partition state q^t of the same
    step; the error is against that partition's q^{t+1} (the q* comparison)."""
    from . import abd
    sc = abd.Scene(sa)
    sc.partition(n_slabs=2, axis=0, planes=[0.0])
    admm, newton, mse, worst = [], [], [], 0
    for q0, v0, q1 in traj:
        sc.set_state(q0, v0)
        st = sc.step(params)
        mse.append(float(np.mean((sc.state()[0] - q1) ** 2)))
        admm.append(st["admm_iters"])
        newton.append(st["newton_iters"])
        worst = max(worst, st["status"])
    sc.close()
    return float(np.mean(mse)), float(np.mean(admm)), float(np.mean(newton)), worst


def hetero_table(steps):
    """Table 2's four cases: {two slabs, one partition} x {heterogeneous, uniform}."""
    from . import abd, scenes
    rows = []
    for hetero in (True, False):
        sa = scenes.heterogeneous_pile(hetero=hetero)
        for n_slabs in (2, 1):
            _, admm, newton, worst = run(sa, steps, abd.default_params(precision=abd.FP64), n_slabs)
            row = {"case": f"{n_slabs}W, {'hetero.' if hetero else 'uniform'}", "bodies": sa.n_dynamic,
                   "steps": steps, "admm_iters_mean": round(admm, 2) if n_slabs > 1 else None,
                   "newton_iters_mean": round(newton, 2), "worst_status": worst}
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--quick", action="store_true", help="three betas, two densities")
    ap.add_argument("--trajectory", action="store_true", help="free runs, error after the last step")
    ap.add_argument("--hetero", action="store_true", help="material-heterogeneity comparison (Table 2)")
    ap.add_argument("--funnel", action="store_true", help="512 spheres packed in the funnel instead of the box pile")
    ap.add_argument("--betas", default=None, help="comma-separated beta values")
    ap.add_argument("--densities", default=None, help="comma-separated densities (kg/m^3)")
    ap.add_argument("--start", type=int, default=0,
                    help="per-step mode: single-partition steps taken before the measured ones")
    a = ap.parse_args()
    import torch
    from . import abd, build
    build.build()
    abd.load()
    torch.cuda.set_device(0)
    if a.hetero:
        t0 = time.perf_counter()
        hetero_table(a.steps)
        print(json.dumps({"wall_s": round(time.perf_counter() - t0, 1)}))
        return
    betas = [0.1, 1.0, 10.0] if a.quick else [0.01, 0.1, 1.0, 10.0, 100.0]
    densities = [100.0, 10000.0] if a.quick else [10.0, 100.0, 1000.0, 10000.0, 100000.0]
    if a.betas:
        betas = [float(x) for x in a.betas.split(",")]
    if a.densities:
        densities = [float(x) for x in a.densities.split(",")]
    rows = []
    t0 = time.perf_counter()
    for rho_d in densities:
        sa = pile(rho_d, a.funnel)
        base = abd.default_params(precision=abd.FP64)
        qstar = run(sa, a.steps, base, 1)[0] if a.trajectory else None
        traj = None if a.trajectory else ref_trajectory(sa, a.start, a.steps, base)
        for beta in betas:
            for mode in (abd.RHO_ADAPTIVE, abd.RHO_FIXED):
                p = abd.default_params(precision=abd.FP64, beta=beta, rho_mode=mode)
                if a.trajectory:
                    q, admm, newton, worst = run(sa, a.steps, p, 2)
                    mse = float(np.mean((q - qstar) ** 2))
                else:
                    mse, admm, newton, worst = run_per_step(sa, traj, p)
                row = {"density": rho_d, "beta": beta, "rho": "adaptive" if mode == abd.RHO_ADAPTIVE else "fixed",
                       "admm_iters_mean": round(admm, 2), "newton_iters_mean": round(newton, 1),
                       "mse_vs_single_partition": mse, "worst_status": worst}
                rows.append(row)
                print(json.dumps(row), flush=True)
    best = {}
    for r in rows:
        if r["rho"] != "adaptive":
            continue
        k = r["density"]
        if k not in best or r["admm_iters_mean"] < best[k]["admm_iters_mean"]:
            best[k] = r
    print(json.dumps({"summary": {str(k): v["beta"] for k, v in best.items()}, "steps": a.steps, "start": a.start,
                      "wall_s": round(time.perf_counter() - t0, 1)}))


if __name__ == "__main__":
    main()
