"""Host logic of the benchmark's open-loop serving leg on CPU, against a fake
server: Poisson inter-arrival times, submission no earlier than each arrival
and in arrival order, and the response-time and throughput arithmetic."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Scene:
    def __init__(self, n):
        self.n_dynamic = n


class _FakeServer:
    """Records submit times; every request 'took' queue 2 ms + run 3 ms and
    had step latencies (1, 4) ms."""

    def __init__(self, clock):
        self.clock, self.submits, self.closed = clock, [], False

    def submit(self, sa, k, params):
        self.submits.append((self.clock(), sa.n_dynamic, k))
        return len(self.submits) - 1

    def wait(self, t):
        return {"queue_ms": 2.0, "run_ms": 3.0, "status": 0 if t % 2 else 2}

    def latencies(self, t):
        return np.array([1.0, 4.0])

    def close(self):
        self.closed = True


def test_poisson_arrivals_rate_and_order():
    import bench
    a = bench.poisson_arrivals(50.0, 20000, seed=3)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 50.0) < 0.03 / 50.0
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03
    assert np.array_equal(a, bench.poisson_arrivals(50.0, 20000, seed=3))


def test_open_loop_submits_on_schedule_and_reports():
    import bench
    clock = time.perf_counter
    srv = _FakeServer(clock)
    reqs = [(_Scene(10 + i), 1 + i % 3) for i in range(12)]
    arrivals = bench.poisson_arrivals(100.0, len(reqs), seed=1)
    t_start = clock()
    r = bench.open_loop(srv, reqs, None, arrivals)
    assert srv.closed
    assert [n for _, n, _ in srv.submits] == [10 + i for i in range(12)]
    for (ts, _, _), ta in zip(srv.submits, arrivals):
        assert ts >= t_start + ta - 1e-9  # never before its arrival
    assert r["p50_response_ms"] == 5.0 and r["p99_response_ms"] == 5.0
    assert r["queue_ms_p99"] == 2.0
    assert r["worst_status"] == 2
    assert r["p50_step_ms"] == 2.5
    bs = sum(10 + i for i in range(12) for _ in range(1 + i % 3))
    assert abs(r["value"] - bs / r["span_s"]) <= 1e-2 * r["value"]
    assert r["span_s"] >= arrivals[-1] - 1e-3


def test_sweep_reports_errors_without_raising():
    import bench

    class _Broken(_FakeServer):
        def submit(self, sa, k, params):
            raise RuntimeError("no device")

    rows = bench.poisson_sweep(lambda: _Broken(time.perf_counter), [(_Scene(4), 1)] * 3, None, 1000.0,
                               fractions=(0.5, 2.0))
    assert [r["fraction_of_capacity"] for r in rows] == [0.5, 2.0]
    assert [r["lambda_rps"] for r in rows] == [500.0, 2000.0]
    assert all(r["error"] == "RuntimeError: no device" for r in rows)


def test_clock_summary_reads_reasons_and_median():
    """The nvidia-smi sampler's summary: median SM clock under load, the
    maximum clock, and every throttle reason seen active."""
    import bench
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1900, 2070, 1398.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2000, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2000.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_keyed_requests_split_each_scene_and_count_body_steps():
    """The serving workload as keyed requests: each scene's steps split into
    a first request carrying the scene and a continuation without it (none
    when the scene advances one step), and body-steps counted from each
    request's key scene and its steps done."""
    import bench
    reqs = [(_Scene(10), 5), (_Scene(3), 1), (_Scene(7), 4)]
    keyed = bench._keyed(reqs)
    assert [(k, sa is not None, n) for k, sa, n in keyed] == [
        (1, True, 2), (1, False, 3), (2, True, 1), (3, True, 2), (3, False, 2)]
    infos = [{"steps_done": n} for _, _, n in keyed]
    assert bench._body_steps(keyed, infos) == 10 * 5 + 3 * 1 + 7 * 4
    infos[1]["steps_done"] = 0  # a continuation that did nothing counts nothing
    assert bench._body_steps(keyed, infos) == 10 * 2 + 3 * 1 + 7 * 4
    assert bench._body_steps(reqs, [{"steps_done": n} for _, n in reqs]) == 10 * 5 + 3 + 28
