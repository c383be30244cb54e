"""Run a workload for `--warmup` steps, then `--steps` steps between
cudaProfilerStart and cudaProfilerStop, so that an external profiler started
with `--profile-from-start off` captures exactly those steps:

  ncu --metrics gpu__time_duration.sum --clock-control none --profile-from-start off \\
      --csv --log-file launches.csv python -m paper_2605_15875_gb300.profile_step --warmup 21

Workloads: c2 (default) the 512-sphere drop on 4 slabs; batch the 64 uneven
subdomains as one batched world (16-2048 bodies each, levels 1-3).
Scenes are created on the legacy default stream, so the Newton iteration is
launched directly (no graph replay; kernels and arithmetic are the same).
Prints one JSON line with the profiled steps' statistics."""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--warmup", type=int, default=21)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="c2", choices=["c2", "batch"])
    a = ap.parse_args()
    import torch
    from . import abd, build, scenes
    build.build()
    abd.load()
    torch.cuda.set_device(0)
    prec = abd.MIXED if a.precision == "mixed" else abd.FP64
    if a.workload == "batch":
        sc = abd.Scene(scenes.batched_subdomains(seed=0, n_scenes=64, lo=16, hi=2048, levels=(1, 2, 3)))
    else:
        sc = abd.Scene(scenes.sphere_grid_in_box(seed=0))
        sc.partition(n_slabs=4, axis=0, planes=[-0.6, 0.0, 0.6])
    p = abd.default_params(precision=prec, pcg_rtol=1e-5 if prec == abd.MIXED else 1e-12)
    for _ in range(a.warmup):
        sc.step(p)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    out = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        st = sc.step(p)
        torch.cuda.synchronize()
        out.append({"ms": round(1e3 * (time.perf_counter() - t0), 3), "admm_iters": st["admm_iters"],
                    "newton_iters": st["newton_iters"], "pcg_iters": st["pcg_iters"],
                    "kernel_launches": st["kernel_launches"], "active_pairs_peak": st["n_active_peak"]})
    torch.cuda.profiler.stop()
    print(json.dumps({"workload": a.workload, "warmup": a.warmup, "precision": a.precision, "steps": out}))


if __name__ == "__main__":
    main()
