#!/usr/bin/env python
"""Benchmark of distributed ABD-IPC on one GB300: body-steps/s of consensus
ADMM over 4 slab partitions of 512 noisy icospheres falling into an open box
(mixed precision: FP32 assembly and PCG, FP64 CCD, energies, residuals and
consensus), beside the plain FP64 path on the same scene, p50/p99 step
latency, the dominant kernel's roofline and the FP64 CPU oracle's throughput.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs independent replicas, one per GPU
(the method's partitions all live on one GPU; nothing is exchanged between
GPUs)."""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "admm4_slabs_512_icosphereL2_open_box"
PLANES = [-0.6, 0.0, 0.6]
# The drop is in free fall until the lowest layer reaches the box floor on
# step 19; the timed window starts there, so every timed step is a contact step.
CONTACT_FROM = 19
METRIC = "ABD-IPC body-steps/s vs plain FP64 GPU at oracle tol; p50/p99 step latency"
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands; a kernel changed since its capture has no entry.
# k_pcg_cluster: mean of the three launches captured on contact step 20 of
# this workload (one FP64 first Newton iteration, 1,362,432 B; two FP32
# iterations, 740,096 B each; writes stay in L2)
TRAFFIC = {"pcg": 947541.3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c4"],
                    help="c2: 512 spheres on 4 slabs (the default line); c4: the 5000-body funnel")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--cmp-steps", type=int, default=6,
                    help="steps of the window the FP64 and fixed-rho comparison legs time (the first ones)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serving", action="store_true", help="skip the served leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven-subdomain leg")
    ap.add_argument("--no-sweep", action="store_true", help="serving: closed batch only, no Poisson sweep")
    ap.add_argument("--batch-steps", type=int, default=4, help="timed steps of the batched leg")
    ap.add_argument("--no-fixed-rho", action="store_true", help="skip the fixed-rho comparison leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="scenes on the legacy default stream (direct launches, no graph replay), e.g. under ncu")
    return ap.parse_args()


def scene_arrays():
    from paper_2605_15875_gb300 import scenes
    return scenes.sphere_grid_in_box(seed=0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def reduce_max_ms(total_ms, world, device):
    """Timed-region length of the slowest rank (every rank gets it)."""
    if world == 1:
        return float(total_ms)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, max_ms):
    """Whole-job throughput: units processed by all ranks over the slowest
    rank's time (each rank runs an independent replica of the workload)."""
    return units_per_rank * world / (max_ms / 1e3)


def run_ours(args, rank, world):
    import torch
    from paper_2605_15875_gb300 import abd, build as B

    B.build()
    abd.load()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    # a stream of its own (not the legacy default stream), so that the
    # library can capture and replay its Newton iteration as a CUDA graph
    stream = torch.cuda.current_stream() if args.no_graph else torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sa = scene_arrays()
    B_ = sa.n_dynamic
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def make(precision, rho_mode=None):
        sc = abd.Scene(sa, stream=int(stream.cuda_stream))
        sc.partition(n_slabs=4, axis=0, planes=PLANES)
        p = abd.default_params(precision=precision, pcg_rtol=1e-12 if precision == abd.FP64 else 1e-5)
        if rho_mode is not None:
            p.rho_mode = rho_mode
        return sc, p

    def settle(sc, p, warmup):
        """Steps 0..18 (free fall) on the same path, then `warmup` contact
        steps from step 19 whose state is restored afterwards: the timed
        window starts at step 19 with the contact path already warm (lists
        grown, Newton-iteration graph captured, PCG cluster size tuned)."""
        for _ in range(CONTACT_FROM):
            sc.step(p)
        q0, v0 = sc.state()
        for _ in range(warmup):
            sc.step(p)
        sc.set_state(q0, v0)

    def timed(sc, p, steps, warmup, profile=False):
        settle(sc, p, warmup)
        if profile:
            sc.profile(True)
        lat, launches, stats = [], 0, []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.start()  # lets an external profiler capture only the timed steps
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = sc.step(p)
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
            launches += st["kernel_launches"]
            stats.append(st)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        if world > 1:
            torch.distributed.barrier()
        return lat, launches, stats

    sc, pm = make(abd.MIXED)
    with Clocks(dev) as clk:
        lat, launches, stats = timed(sc, pm, args.steps, args.warmup, profile=True)
    total_ms = reduce_max_ms(sum(lat), world, "cuda")
    value = job_value(B_ * args.steps, world, total_ms)
    # dominant kernel and its roofline
    names = ["pcg", "pair_moll", "pair_assemble", "slot_assemble", "l2_static", "l2_swept", "ccd", "energy"]
    ks = {n: sc.kernel_stats(n) for n in names}
    dom = max(ks, key=lambda n: ks[n][1])
    n_l, ms_l, by_l = ks[dom]
    peak, peak_kind = measured_peaks()
    achieved = (by_l / (ms_l / 1e3)) / 1e9 if ms_l > 0 else 0.0
    # achieved = algorithmic bytes per launch / average launch time (CUDA
    # events on the scene's stream); for the PCG the bytes are counted per
    # iteration (blocks and seven 12-vectors per slot, each iteration)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": TRAFFIC.get(dom), "peak_source": peak_kind,
            "bytes_per_launch": round(by_l / max(1, n_l), 1),
            "launches": n_l, "avg_launch_us": round(1e3 * ms_l / max(1, n_l), 3),
            "share_of_step": round(ms_l / total_ms, 4) if total_ms else None,
            "kernels_ms": {n: round(v[1], 3) for n, v in ks.items()},
            # every instrumented kernel: compulsory bytes over its live CUDA-event time
            "kernels_gbs": {n: (round(v[2] / (v[1] / 1e3) / 1e9, 2) if v[1] > 0 and v[2] > 0 else None)
                            for n, v in ks.items()}}
    errors = {}  # a comparison leg that fails reports here; the headline stays
    # the comparison legs (plain FP64, fixed rho) time the first `ncmp` steps of
    # the window -- the later contact steps cost the FP64 path many seconds
    # each -- against the mixed path's own time over the same steps
    ncmp = max(1, min(args.steps, args.cmp_steps))
    value_cmp = B_ * ncmp * world / (sum(lat[:ncmp]) / 1e3)
    fp64 = None
    if not args.no_fp64:
        try:
            sc64, p64 = make(abd.FP64)
            lat64, _, _ = timed(sc64, p64, ncmp, args.warmup)
            fp64 = B_ * ncmp * world / (sum(lat64) / 1e3)
            sc64.close()
        except Exception as e:
            errors["fp64"] = f"{type(e).__name__}: {e}"
    # the same window with a fixed penalty rho = beta m (no residual-driven adaptation)
    fixed = None
    if not args.no_fixed_rho:
        try:
            scf, pf = make(abd.MIXED, abd.RHO_FIXED)
            latf, _, statf = timed(scf, pf, ncmp, args.warmup)
            fixed = {"value": round(B_ * ncmp * world / (sum(latf) / 1e3), 3), "unit": "body-steps/s",
                     "steps": ncmp, "mixed_adaptive_same_steps": round(value_cmp, 3),
                     "admm_iters_mean": float(np.mean([x["admm_iters"] for x in statf])),
                     "newton_iters_mean": float(np.mean([x["newton_iters"] for x in statf])),
                     "min_distance_min": float(min(x["min_distance"] for x in statf))}
            scf.close()
        except Exception as e:
            errors["fixed_rho"] = f"{type(e).__name__}: {e}"
    e2e = None
    if not args.no_e2e:
        # the same window through the public C ABI with host buffers: every
        # step copies q, v host -> device (abd_state_set), steps, and copies
        # them back (abd_state_get); L2 flushed between steps as for `value`,
        # outside the per-step timing
        sce, pe = make(abd.MIXED)
        settle(sce, pe, args.warmup)
        qh = torch.empty((sa.n_bodies, 12), dtype=torch.float64).pin_memory()
        vh = torch.empty((sa.n_bodies, 12), dtype=torch.float64).pin_memory()
        q0, v0 = sce.state()
        qh.copy_(torch.from_numpy(q0))
        vh.copy_(torch.from_numpy(v0))
        L = sce.L
        torch.cuda.synchronize()
        dt = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.abd_state_set(sce.h, qh.data_ptr(), vh.data_ptr(), sa.n_bodies)
            sce.step(pe)
            L.abd_state_get(sce.h, qh.data_ptr(), vh.data_ptr(), sa.n_bodies)
            dt += time.perf_counter() - t0
        e2e = {"value": round(B_ * args.steps * world / dt, 3), "unit": "body-steps/s",
               "h2d_bytes_per_step": 2 * 96 * sa.n_bodies, "d2h_bytes_per_step": 2 * 96 * sa.n_bodies,
               "timing": "host clock around abd_state_set + abd_step + abd_state_get per step, L2 flushed "
                         "between steps outside it (the same window and conditions as value)"}
        sce.close()
    serving = batched = None
    if not args.no_serving:
        try:
            serving = serve_legs(abd, sweep=not args.no_sweep)
        except Exception as e:
            errors["serving"] = f"{type(e).__name__}: {e}"
    if not args.no_batched:
        try:
            batched = batched_leg(abd, torch, stream, flush, args.batch_steps, 2)
        except Exception as e:
            errors["batched"] = f"{type(e).__name__}: {e}"
    cpu = cpu_baseline(args.cpu_seconds) if (rank == 0 and world == 1) else None
    lat_sorted = sorted(lat)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "body-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "bodies": B_, "triangles": sa.total_tris(), "partitions": 4,
                   "slab_planes_x": PLANES, "h": pm.h, "dhat": pm.dhat, "precision": "mixed",
                   "rho": "adaptive", "pcg_rtol": pm.pcg_rtol, "newton_tol": pm.newton_tol,
                   "theta": pm.theta, "l2": "flushed between timed steps (256 MB write)",
                   "newton_iteration_graph": not args.no_graph,
                   "window": f"steps {CONTACT_FROM}..{CONTACT_FROM + args.steps - 1} of the drop, all contact "
                             f"steps (the lowest layer lands on the box floor on step {CONTACT_FROM}); before "
                             f"them steps 0..{CONTACT_FROM - 1} (free fall) and {args.warmup} warm-up contact "
                             f"steps from step {CONTACT_FROM}, whose state is then restored, all on the same "
                             "GPU path"},
        "window_totals": {"admm_iters": int(sum(s["admm_iters"] for s in stats)),
                          "newton_iters": int(sum(s["newton_iters"] for s in stats)),
                          "pcg_iters": int(sum(s["pcg_iters"] for s in stats)),
                          "pcg_cluster": int(max(s["pcg_cluster"] for s in stats)),
                          "list_redo": int(sum(s["list_redo"] for s in stats))},
        "p50_ms": round(float(np.percentile(lat_sorted, 50)), 4),
        "p99_ms": round(float(np.percentile(lat_sorted, 99)), 4),
        "fp64_value": None if fp64 is None else round(fp64, 3),
        "fp64_steps": ncmp, "mixed_value_same_steps": round(value_cmp, 3),
        "speedup_vs_fp64": None if fp64 is None else round(value_cmp / fp64, 3),
        "admm_iters_mean": float(np.mean([s["admm_iters"] for s in stats])),
        "newton_iters_mean": float(np.mean([s["newton_iters"] for s in stats])),
        "active_pairs_peak": int(max(s["n_active_peak"] for s in stats)),
        "candidates_peak": int(max(s["n_candidates_peak"] for s in stats)),
        "fixed_rho": fixed,
        "min_distance_min": float(min(x["min_distance"] for x in stats)),
        "serving": serving, "batched": batched,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if errors:
        out["leg_errors"] = errors
    sc.close()
    return out


def _keyed(reqs):
    """Each scene of the serving workload as two keyed requests: the first
    (with the scene) advances half of its steps, the second (key only)
    continues from the resident state for the rest."""
    out = []
    for key, (sa, k) in enumerate(reqs, start=1):
        k1 = max(1, k // 2)
        out.append((key, sa, k1))
        if k - k1 > 0:
            out.append((key, None, k - k1))
    return out


def _body_steps(reqs, infos):
    """Dynamic-body steps done by requests (key, scene or None, steps) or
    (scene, steps): a keyed request without a scene counts its key's scene."""
    nd, total = {}, 0
    for r, i in zip(reqs, infos):
        key, sa = (r[0], r[1]) if len(r) == 3 else (None, r[0])
        if sa is not None:
            nd[key] = sa.n_dynamic
        total += (sa.n_dynamic if sa is not None else nd[key]) * i.get("steps_done", r[-1])
    return total


def _serve(abd, reqs, n_streams, params):
    """Closed batch: every request submitted at once (continuous admission),
    resident scenes released at the end.  reqs: (key, scene or None, steps)."""
    srv = abd.Server(n_streams=n_streams)
    t0 = time.perf_counter()
    ts = [srv.submit(sa, k, params, key=key) for key, sa, k in reqs]
    infos = [srv.wait(t) for t in ts]
    dt = time.perf_counter() - t0
    lat = np.concatenate([srv.latencies(t) for t in ts])
    srv.close()
    bs = _body_steps(reqs, infos)
    return {"value": round(bs / dt, 2), "unit": "body-steps/s", "wall_s": round(dt, 3), "body_steps": int(bs),
            "p50_step_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_step_ms": round(float(np.percentile(lat, 99)), 3),
            "requests": len(reqs), "n_streams": n_streams,
            "worst_status": int(max(i["status"] for i in infos)),
            "queue_ms_p99": round(float(np.percentile([i["queue_ms"] for i in infos], 99)), 3)}


def poisson_arrivals(rate, n, seed):
    """Arrival times (s after the first possible arrival) of n requests of a
    Poisson process with `rate` requests per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def open_loop(server, reqs, params, arrivals, clock=time.perf_counter, sleep=time.sleep):
    """Open-loop serving: request i is submitted at arrival time arrivals[i]
    whether or not earlier requests are done (they keep running on the
    server's workers meanwhile), then every request is waited for.  Response
    time = queue + run of a request (submit to done); step latency = each
    abd_step call of each request.  reqs: (scene, steps) or (key, scene or
    None, steps).  The server is closed on return."""
    lags, ts = [], []
    try:
        t0 = clock()
        for r, ta in zip(reqs, arrivals):
            key, sa, k = r if len(r) == 3 else (None, r[0], r[1])
            d = t0 + ta - clock()
            if d > 0:
                sleep(d)
            lags.append(clock() - (t0 + ta))
            ts.append(server.submit(sa, k, params) if key is None else server.submit(sa, k, params, key=key))
        infos = [server.wait(t) for t in ts]
        span = clock() - t0
        lat = np.concatenate([server.latencies(t) for t in ts])
    finally:
        server.close()
    resp = [i["queue_ms"] + i["run_ms"] for i in infos]
    bs = _body_steps(reqs, infos)
    return {"value": round(bs / span, 2), "unit": "body-steps/s", "span_s": round(span, 4),
            "p50_step_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_step_ms": round(float(np.percentile(lat, 99)), 3),
            "p50_response_ms": round(float(np.percentile(resp, 50)), 3),
            "p99_response_ms": round(float(np.percentile(resp, 99)), 3),
            "queue_ms_p99": round(float(np.percentile([i["queue_ms"] for i in infos], 99)), 3),
            "submit_lag_ms_max": round(1e3 * max(lags), 3),
            "worst_status": int(max(i["status"] for i in infos))}


def poisson_sweep(make_server, reqs, params, capacity_rps, fractions=(0.25, 0.5, 1.0, 2.0), seed=1):
    """The serving workload under Poisson arrivals at rates lambda = f x the
    server's measured closed-batch capacity (requests/s), one open-loop run
    per rate; a run that raises reports its error instead of a number."""
    out = []
    for f in fractions:
        lam = f * capacity_rps
        row = {"fraction_of_capacity": f, "lambda_rps": round(lam, 3)}
        try:
            row.update(open_loop(make_server(), reqs, params, poisson_arrivals(lam, len(reqs), seed)))
        except Exception as e:  # keep the benchmark line; say what failed
            row["error"] = f"{type(e).__name__}: {e}"
        out.append(row)
    return out


def serve_legs(abd, n_scenes=256, lo=8, hi=4096, sweep=True):
    """Served leg, mixed precision: the serving workload (`n_scenes` scenes
    of lo..hi bodies, cube stacks and sphere piles, 1-10 steps each), every
    scene as two keyed requests on a resident scene (the second continues
    from the state the first left on the device); a closed batch (every
    request submitted at once, continuous admission), the plain FP64 path on
    the same requests one at a time, then, with `sweep`, the same requests
    under Poisson arrivals at four rates."""
    from paper_2605_15875_gb300 import scenes
    p = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5)
    p64 = abd.default_params(precision=abd.FP64, pcg_rtol=1e-12)
    reqs = _keyed(scenes.serving_requests(seed=0, n_scenes=n_scenes, lo=lo, hi=hi))
    # each arm is warmed on its first 16 requests (process-wide one-time
    # costs), then timed on the whole request set repeatedly: the median
    # pass is reported with the spread
    _serve(abd, reqs[:16], 4, p)
    runs = [_serve(abd, reqs, 4, p) for _ in range(3)]
    _serve(abd, reqs[:16], 1, p64)
    plain_runs = [_serve(abd, reqs, 1, p64) for _ in range(2)]
    vals = sorted(r["value"] for r in runs)
    serving = sorted(runs, key=lambda r: r["value"])[len(runs) // 2]
    pvals = sorted(r["value"] for r in plain_runs)
    plain = float(np.median(pvals))
    serving["passes"] = {"values": vals, "median": vals[len(vals) // 2]}
    serving["plain_fp64_one_at_a_time"] = round(plain, 2)
    serving["plain_fp64_passes"] = pvals
    serving["speedup_vs_plain_fp64"] = round(serving["value"] / plain, 3)
    serving["speedup_range"] = [round(vals[0] / pvals[-1], 3), round(vals[-1] / pvals[0], 3)]
    serving["sample"] = (f"{n_scenes} scenes of {lo}-{hi} bodies (log-uniform; cube stacks and sphere piles), "
                         "1-10 steps each as two keyed requests on a resident scene")
    if sweep:
        cap_rps = len(reqs) / serving["wall_s"]
        serving["poisson"] = poisson_sweep(lambda: abd.Server(n_streams=4), reqs, p, cap_rps)
        serving["poisson_note"] = ("open loop, 4 streams, the same requests; lambda relative to the closed-batch "
                                   "capacity above (requests/s)")
    return serving


def batched_leg(abd, torch, stream, flush, steps, warmup, n_scenes=64, lo=16, hi=2048, seed=0, pre_steps=12):
    """Uneven subdomains packed into one batched world (one partition per
    subdomain, every Newton phase of every subdomain in the same launches,
    the steady-state iteration replayed as a CUDA graph), mixed precision,
    against the plain FP64 path stepping each subdomain alone, one at a time,
    over the same steps.  The world first takes `pre_steps` untimed steps,
    in which the piles land and come into contact; from that state each side
    warms up on `warmup` steps whose state is then restored, and times
    `steps` steps; L2 is flushed between timed steps (outside the timing)."""
    from paper_2605_15875_gb300 import scenes
    subs = scenes.batched_subdomains(seed=seed, n_scenes=n_scenes, lo=lo, hi=hi, levels=(1, 2, 3))
    nb = sum(sa.n_dynamic for sa in subs)
    pm = abd.default_params(precision=abd.MIXED, pcg_rtol=1e-5)
    p64 = abd.default_params(precision=abd.FP64, pcg_rtol=1e-12)

    def run(sc, p, prof=False, start=None):
        if start is not None:
            sc.set_state(*start)
        q0, v0 = sc.state()
        for _ in range(warmup):
            sc.step(p)
        sc.set_state(q0, v0)
        if prof:
            sc.profile(True)
        lat, sts = [], []
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts.append(sc.step(p))
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
        return lat, sts

    world = abd.Scene(subs, stream=int(stream.cuda_stream))
    for _ in range(pre_steps):  # the piles settle into contact (untimed)
        world.step(pm)
    qw, vw = world.state()
    off = world.layout()
    lat, sts = run(world, pm, prof=True)
    names = ["pcg", "pair_moll", "pair_assemble", "slot_assemble", "l2_static", "l2_swept", "ccd", "energy"]
    ks = {n: world.kernel_stats(n) for n in names}
    world.close()
    t_b = sum(lat) / 1e3
    alone_ms, alone_status = 0.0, 0
    for i, sa in enumerate(subs):
        sc = abd.Scene(sa, stream=int(stream.cuda_stream))
        la, sa_st = run(sc, p64, start=(qw[off[i]:off[i + 1]], vw[off[i]:off[i + 1]]))
        alone_ms += sum(la)
        alone_status = max([alone_status] + [x["status"] for x in sa_st])
        sc.close()
    value = nb * steps / t_b
    plain = nb * steps / (alone_ms / 1e3)
    return {"value": round(value, 2), "unit": "body-steps/s", "subdomains": n_scenes, "bodies": nb,
            "steps": steps, "p50_step_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_step_ms": round(float(np.percentile(lat, 99)), 3),
            "plain_fp64_one_at_a_time": round(plain, 2), "speedup_vs_plain_fp64": round(value / plain, 3),
            "newton_iters_mean": float(np.mean([x["newton_iters"] for x in sts])),
            "active_pairs_peak": int(max(x["n_active_peak"] for x in sts)),
            "worst_status": int(max(x["status"] for x in sts)), "plain_worst_status": int(alone_status),
            "min_distance_min": float(min(x["min_distance"] for x in sts)),
            "kernels_gbs": {n: (round(v[2] / (v[1] / 1e3) / 1e9, 2) if v[1] > 0 and v[2] > 0 else None)
                            for n, v in ks.items()},
            "kernels_ms": {n: round(v[1], 3) for n, v in ks.items()},
            "sample": f"{n_scenes} subdomains of {lo}-{hi} noisy icospheres (log-uniform counts, levels 1-3, "
                      f"densities log-uniform 1e2-1e4, seed {seed}), one batched world; steps {pre_steps}.."
                      f"{pre_steps + steps - 1} timed (the piles in contact) after {warmup} warm-up steps from "
                      f"step {pre_steps} (state restored); the FP64 runs start from the same state"}


def host_cpu():
    """The host the oracle ran on: architecture, logical cores, CPU model where
    the kernel reports one."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:  # Arm kernels list implementer/part codes only; lscpu names the core
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "model": model}


def cpu_baseline(seconds):
    """The FP64 oracle as it stands, on one host core, over the first steps of
    the same workload (stops after `seconds` of CPU work, at least one step)."""
    import oracle as O
    sa = scene_arrays()
    sc = O.Scene(sa)
    p = O.default_params(n_slabs=4, axis=0, planes=PLANES)
    for _ in range(CONTACT_FROM):  # free fall, untimed: the sample is of the timed window's contact steps
        sc.step(p)
    # CPU time of this thread alone: the oracle runs here, while idle numpy
    # worker threads spinning elsewhere in the process would inflate
    # process_time()
    n, t0 = 0, time.thread_time()
    while True:
        sc.step(p)
        n += 1
        if time.thread_time() - t0 > seconds:
            break
    dt = time.thread_time() - t0
    # the 8-cube stack of the plain single-partition workload, all 100 steps
    from paper_2605_15875_gb300 import scenes
    cs = scenes.cube_stack()
    oc, pc = O.Scene(cs), O.default_params()
    t1 = time.thread_time()
    for _ in range(100):
        oc.step(pc)
    dc = time.thread_time() - t1
    return {"value": round(sa.n_dynamic * n / dt, 4), "unit": "body-steps/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"steps {CONTACT_FROM}..{CONTACT_FROM + n - 1} of the same scene (512 bodies, 4 slabs; "
                      f"the first contact steps of the timed window), single thread, {dt:.1f} s CPU",
            "cube_stack_8": {"value": round(cs.n_dynamic * 100 / dc, 2), "unit": "body-steps/s",
                             "sample": f"8 stacked unit cubes on a plane, one partition, 100 steps, {dc:.2f} s CPU"}}


def run_reference(args, rank, world):
    """The FP64 oracle as it stands on one host core, on the same window as
    the GPU arm: steps 0..18 untimed, of which the last `warmup` are the
    warm-up steps, then timed steps from step 19 (contact) until `steps` are
    done or the time budget is spent -- the oracle's contact steps take 10 s
    to minutes each, so the cut is stated in the sample."""
    if rank != 0:
        return None
    import oracle as O
    oracle_build = O.build()  # noqa: F841
    sa = scene_arrays()
    sc = O.Scene(sa)
    p = O.default_params(n_slabs=4, axis=0, planes=PLANES)
    for _ in range(CONTACT_FROM):
        sc.step(p)
    lat, t_start, budget = [], time.perf_counter(), 240.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sc.step(p)
        lat.append(1e3 * (time.perf_counter() - t0))
        if time.perf_counter() - t_start > budget:
            break
    n = len(lat)
    value = sa.n_dynamic * n / (sum(lat) / 1e3)
    sample = (f"steps {CONTACT_FROM}..{CONTACT_FROM + n - 1} of the same scene (contact steps; steps 0..."
              f"{CONTACT_FROM - 1} untimed, the last {args.warmup} being the warm-up) on one host core"
              + ("" if n == args.steps else
                 f"; stopped after {n} of {args.steps} steps at the {budget:.0f} s budget (later steps of the "
                 "window cost more ADMM rounds, so the cut favours the oracle)"))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "body-steps/s",
            "n_gpus": world, "steps": n, "warmup": args.warmup, "ms_per_step": round(sum(lat) / n, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "bodies": sa.n_dynamic, "partitions": 4,
                                            "window_start": CONTACT_FROM},
            "cpu_baseline": {"value": round(value, 4), "unit": "body-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": round(value, 4), "unit": "body-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_c4(args, rank, world):
    """The large funnel workload: 5000 level-3 noisy icospheres (6.4 M
    triangles) starting packed in the funnel above the chamber with its two
    perforated turntables turning at +-1 rad/s; 2 and 8 slab partitions along
    x (equal widths over the bodies' extent, rebuilt every step), mixed
    precision against FP64.  Each run takes `warmup` untimed steps from the
    packed start, then times `steps` steps (CUDA events, L2 flushed between
    steps)."""
    import torch
    from paper_2605_15875_gb300 import abd, build as B, scenes
    B.build()
    abd.load()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    sa = scenes.funnel_scene(dense=True)
    nb = sa.n_dynamic
    names = ["pcg", "pair_moll", "pair_assemble", "slot_assemble", "l2_static", "l2_swept", "ccd", "energy"]
    peak, peak_kind = measured_peaks()
    legs, headline, clk_summary = {}, None, None
    for slabs in (8, 2):
        for prec in (abd.MIXED, abd.FP64):
            key = f"{slabs}slabs_{'mixed' if prec == abd.MIXED else 'fp64'}"
            try:
                sc = abd.Scene(sa, stream=int(stream.cuda_stream))
                sc.partition(n_slabs=slabs, axis=0)
                p = abd.default_params(precision=prec, pcg_rtol=1e-5 if prec == abd.MIXED else 1e-12)
                for _ in range(args.warmup):
                    sc.step(p)
                sc.profile(True)
                lat, sts = [], []
                torch.cuda.synchronize()
                with Clocks(dev) as clk:
                    for _ in range(args.steps):
                        flush.zero_()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        sts.append(sc.step(p))
                        e1.record(stream)
                        e1.synchronize()
                        lat.append(e0.elapsed_time(e1))
                ks = {n: sc.kernel_stats(n) for n in names}
                sc.close()
                leg = {"value": round(nb * len(lat) / (sum(lat) / 1e3), 3), "unit": "body-steps/s",
                       "ms_per_step": round(sum(lat) / len(lat), 2), "steps": len(lat),
                       "admm_iters": [x["admm_iters"] for x in sts], "newton_iters": [x["newton_iters"] for x in sts],
                       "candidates_peak": int(max(x["n_candidates_peak"] for x in sts)),
                       "active_pairs_peak": int(max(x["n_active_peak"] for x in sts)),
                       "min_distance_min": float(min(x["min_distance"] for x in sts)),
                       "worst_status": int(max(x["status"] for x in sts)),
                       "n_slots": int(sts[-1]["n_slots"]), "n_shared": int(sts[-1]["n_shared"]),
                       "pcg_cluster": int(max(x["pcg_cluster"] for x in sts)),
                       "kernels_ms": {n: round(v[1], 3) for n, v in ks.items()},
                       "kernels_gbs": {n: (round(v[2] / (v[1] / 1e3) / 1e9, 2) if v[1] > 0 and v[2] > 0 else None)
                                       for n, v in ks.items()},
                       "clocks": clk.summary()}
                dom = max(ks, key=lambda n: ks[n][1])
                n_l, ms_l, by_l = ks[dom]
                ach = (by_l / (ms_l / 1e3)) / 1e9 if ms_l > 0 else 0.0
                leg["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 2), "peak": peak,
                                   "unit": "GB/s", "frac": round(ach / peak, 4), "peak_source": peak_kind,
                                   "bytes_per_launch": round(by_l / max(1, n_l), 1), "launches": n_l,
                                   "avg_launch_us": round(1e3 * ms_l / max(1, n_l), 3)}
                legs[key] = leg
                if headline is None and prec == abd.MIXED:
                    headline, clk_summary = (key, leg), leg["clocks"]
            except Exception as e:
                legs[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        return None
    key, h = headline if headline else ("none", {"value": None, "ms_per_step": None, "roofline": None})
    for slabs in (8, 2):
        m, f = legs.get(f"{slabs}slabs_mixed", {}), legs.get(f"{slabs}slabs_fp64", {})
        if m.get("value") and f.get("value"):
            m["speedup_vs_fp64"] = round(m["value"] / f["value"], 3)
    return {"metric": METRIC, "value": h["value"], "unit": "body-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "funnel_5000_icosphereL3_dense_start", "bodies": nb,
                       "triangles": sa.total_tris(), "headline_leg": key,
                       "start": "bodies packed in the funnel (lattice pitch 2.2 r + 2 mm), turntables at +-1 rad/s",
                       "window": f"steps {args.warmup}..{args.warmup + args.steps - 1} from the packed start",
                       "l2": "flushed between timed steps (256 MB write)",
                       "paper_scale": "Table 1 'Pokemon': 5.2K bodies, 5.7M triangles, 59.8M candidates and 40.1K "
                                      "contacts at peak, 2 workers (RTX 4090 each), h = 0.0125"},
            "legs": legs, "roofline": h.get("roofline"), "clocks": clk_summary}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "c4":
        out = run_c4(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
