"""Request server (esp_server_*): every result, alone or in a concurrent mix,
equals a single plan's result for the same system, tolerance and positions.

Requests of several systems and tolerances are submitted all at once (they
overlap on the device, several per plan queue behind each other) and one at a
time (submit, wait); both must match esp_plan + esp_compute within the FP32
bound of the parity tests (only the FP32 atomic summation order differs).
A small memory budget forces plan evictions; a system that cannot fit the
budget fails with ESP_ERR_BUSY.
"""
import numpy as np
import pytest

from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_PARITY = 5e-6


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def alone(esp, s, pos, eps, r_c):
    with esp.Plan(s.L, s.n, eps, r_c=r_c) as p:
        p.set_charges(s.q)
        p.set_positions(pos)
        return p.compute()


def requests_of(systems, n_req, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_req):
        i = int(rng.integers(len(systems)))
        eps = float(rng.choice([1e-3, 1e-4, 1e-5]))
        out.append((i, eps, inputs.perturb(systems[i], 0.01, seed=seed * 1000 + k).pos))
    return out


def check(esp, systems, reqs, results, r_c):
    cache = {}
    for (i, eps, pos), (e, f, u, lat) in zip(reqs, results):
        key = (i, eps, pos.tobytes())
        if key not in cache:
            cache[key] = alone(esp, systems[i], pos, eps, r_c)
        e0, f0, u0 = cache[key]
        assert rel_rms(f, f0) <= FP32_PARITY
        assert rel_rms(u, u0) <= FP32_PARITY
        assert abs(e - e0) <= FP32_PARITY * abs(e0)
        assert lat > 0


def test_mix_and_alone_match_single_plans(esp):
    # tolerances 1e-3, 1e-4 and 1e-5; one system of 2e5 atoms in the mix
    systems = inputs.electrolyte_batch([3000, 5200, 8000, 3600, 12000, 200_000], seed=300)
    reqs = requests_of(systems, 24, seed=301)
    assert {eps for _, eps, _ in reqs} == {1e-3, 1e-4, 1e-5} and any(i == 5 for i, _, _ in reqs)
    with esp.Server(1.0, max_inflight=6) as srv:
        ids = [srv.add_system(s.L, s.q) for s in systems]
        tickets = [srv.submit(ids[i], eps, pos) for i, eps, pos in reqs]       # the mix
        mixed = [srv.wait(t) for t in tickets]
        single = []
        for i, eps, pos in reqs:                                               # one at a time
            single.append(srv.wait(srv.submit(ids[i], eps, pos)))
        st = srv.stats()
    check(esp, systems, reqs, mixed, 1.0)
    check(esp, systems, reqs, single, 1.0)
    for a, b in zip(mixed, single):
        assert rel_rms(a[1], b[1]) <= FP32_PARITY
    assert st["completed"] == 48 and st["failed"] == 0
    assert st["plans_resident"] == st["plans_created"] <= 18
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0


def test_small_budget_evicts_and_still_answers(esp):
    systems = inputs.electrolyte_batch([6000, 7000, 8000, 9000], seed=310)
    reqs = requests_of(systems, 16, seed=311)
    with esp.Plan(systems[-1].L, systems[-1].n, 1e-4, r_c=1.0) as p:
        one = p.info["device_bytes"]
    budget = int(3 * one)       # room for two or three of the eight plans
    with esp.Server(1.0, memory_budget=budget, max_inflight=4) as srv:
        ids = [srv.add_system(s.L, s.q) for s in systems]
        results = [srv.wait(srv.submit(ids[i], eps, pos)) for i, eps, pos in reqs]
        st = srv.stats()
    check(esp, systems, reqs, results, 1.0)
    assert st["evictions"] > 0
    assert st["device_bytes"] <= budget


def test_system_larger_than_budget_is_refused(esp):
    s = inputs.electrolyte(20000, seed=320)
    with esp.Server(1.0, memory_budget=1 << 20) as srv:     # below any plan's need
        sid = srv.add_system(s.L, s.q)
        with pytest.raises(esp.EspError) as exc:
            srv.wait(srv.submit(sid, 1e-4, s.pos))
        assert exc.value.status == 9
        st = srv.stats()
    assert st["failed"] == 1


def test_bad_requests_are_rejected(esp):
    s = inputs.electrolyte(3000, seed=330)
    with esp.Server(1.0) as srv:
        sid = srv.add_system(s.L, s.q)
        with pytest.raises(esp.EspError) as exc:
            srv.submit(sid + 5, 1e-4, s.pos)
        assert exc.value.status == 1
        with pytest.raises(esp.EspError) as exc:
            srv.submit(sid, 0.5, s.pos)
        assert exc.value.status == 1
        bad = s.pos.copy()
        bad[7, 1] = np.nan
        with pytest.raises(esp.EspError) as exc:
            srv.wait(srv.submit(sid, 1e-4, bad))
        assert exc.value.status == 4
        e, f, u, _ = srv.wait(srv.submit(sid, 1e-4, s.pos))                      # still serves
        e0, f0, u0 = alone(esp, s, s.pos, 1e-4, 1.0)
        assert rel_rms(f, f0) <= FP32_PARITY


def test_requests_submitted_while_others_run_overlap_on_the_device(esp):
    """Continuous batching: a second thread submits while the first thread's
    requests are on the device. The server's device intervals (events on each
    request's stream before its first copy and after its last) must overlap,
    and every result must equal the same request run alone."""
    import threading
    systems = inputs.electrolyte_batch([40000, 60000, 30000, 50000], seed=340)
    reqs = requests_of(systems, 16, seed=341)
    with esp.Server(1.0, max_inflight=8) as srv:
        ids = [srv.add_system(s.L, s.q) for s in systems]
        for i, eps, pos in reqs[:4]:                       # plans created before the timed mix
            srv.wait(srv.submit(ids[i], eps, pos))
        esp.esp_server_reset_stats(srv.handle)
        first, second = reqs[:8], reqs[8:]
        tickets_b = []
        started = threading.Event()

        def late_client():
            started.wait()
            for i, eps, pos in second:
                tickets_b.append(srv.submit(ids[i], eps, pos))

        th = threading.Thread(target=late_client)
        th.start()
        tickets_a = []
        for k, (i, eps, pos) in enumerate(first):
            tickets_a.append(srv.submit(ids[i], eps, pos))
            if k == 1:
                started.set()                              # the other client joins mid-stream
        th.join()
        results = [srv.wait(t) for t in tickets_a] + [srv.wait(t) for t in tickets_b]
        st = srv.stats()
    check(esp, systems, first + second, results, 1.0)
    assert st["completed"] == 16 and st["failed"] == 0
    assert st["peak_inflight"] >= 2
    assert st["peak_concurrent"] >= 2, st
    assert st["overlap_ms"] > 0.0


def test_timed_out_request_releases_its_plan(esp):
    """A request that exceeds the server deadline fails with ESP_ERR_TIMEOUT;
    once its device work finishes its plan is free again, so the next request
    for the same system is admitted (and, under the same short deadline,
    times out by itself) instead of waiting forever behind a busy plan."""
    import time
    s = inputs.electrolyte(400_000, seed=350)
    with esp.Server(1.0, timeout_ms=0.05, max_inflight=2) as srv:
        sid = srv.add_system(s.L, s.q)
        for _ in range(2):
            with pytest.raises(esp.EspError) as exc:
                srv.wait(srv.submit(sid, 1e-5, s.pos), timeout_ms=30000.0)
            assert exc.value.status == 8
            assert "server deadline" in str(exc.value)
            for _ in range(2000):                          # the late work drains
                st = srv.stats()
                if st["running"] == 0 and st["pending"] == 0:
                    break
                time.sleep(0.005)
        st = srv.stats()
    assert st["failed"] == 2
    assert st["plans_resident"] == 1
