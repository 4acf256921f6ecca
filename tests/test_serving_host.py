"""The serving loop's admission policy on the host, with fake sessions (no GPU): at most max_active
sessions and never more reserved HBM than the budget, waiting scenes admitted in arrival order as
sessions finish, every request served once, and latency counted from arrival (deferral included)."""
import threading
import time
import types

from paper_2503_13086_gb300.serving import Scene, Server, summarize


class FakeSession:
    """Stands in for a StreamingSession: each request takes `work_s` of host time."""
    lock = threading.Lock()
    active = 0
    peak = 0
    made = []

    def __init__(self, hbm_budget_bytes, work_s=0.03, name=None):
        with FakeSession.lock:
            FakeSession.active += 1
            FakeSession.peak = max(FakeSession.peak, FakeSession.active)
            FakeSession.made.append(name)
        self.work_s = work_s
        self.results = []
        self.stream = types.SimpleNamespace(synchronize=lambda: None)
        self.field = types.SimpleNamespace(stats=lambda: {"n_gaussians": 0},
                                           get_gaussians=lambda with_adam=False: None)

    def arrive(self, cam, target, pts_xyz=None, pts_rgb=None, tracks=None, arrival_time=None):
        time.sleep(self.work_s)
        self.results.append(dict(latency_s=time.perf_counter() - arrival_time, pairs=1000))

    def latency(self):
        lat = sorted(r["latency_s"] for r in self.results)
        return dict(p50=lat[len(lat) // 2], n=len(lat))

    def close(self):
        with FakeSession.lock:
            FakeSession.active -= 1


def reset():
    FakeSession.active = 0
    FakeSession.peak = 0
    FakeSession.made = []


def scenes(n, requests=3, spacing=0.0):
    req = dict(cam=None, target=None)
    return [Scene(f"s{k}", [(k * spacing + 0.001 * r, req) for r in range(requests)], config=dict(name=f"s{k}"))
            for k in range(n)]


def serve(server, sc):
    out = server.run(sc, poll_s=0.0005)
    return out, server.log


def test_at_most_max_active_sessions_and_every_request_served():
    reset()
    srv = Server(hbm_budget_bytes=100, session_budget_bytes=10, max_active=2, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(5))
    assert FakeSession.peak == 2
    assert sorted(out) == [f"s{k}" for k in range(5)]
    assert all(len(r["results"]) == 3 for r in out.values())
    # scenes that found both slots taken were deferred, then admitted in arrival order
    assert [e[2] for e in log if e[1] == "admit"] == [f"s{k}" for k in range(5)]
    assert {e[2] for e in log if e[1] == "defer"} >= {"s2"}


def test_the_hbm_budget_limits_concurrency():
    reset()
    srv = Server(hbm_budget_bytes=25, session_budget_bytes=10, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(4))
    assert FakeSession.peak == 2  # 2 x 10 <= 25 < 3 x 10
    assert len(out) == 4


def test_latency_counts_the_time_a_scene_waited():
    reset()
    srv = Server(hbm_budget_bytes=10, session_budget_bytes=10, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(2, requests=2))
    # s1 arrived with s0 but was admitted only after s0's two requests (~2 x 30 ms)
    first = out["s1"]["results"][0]["latency_s"]
    assert first >= 0.05
    assert out["s0"]["results"][0]["latency_s"] < first
    s = summarize(out, srv.wall_s)
    assert s["per_session"]["s0"]["n"] == 2 and s["pairs_per_s"] > 0


def test_peak_device_memory_is_sampled_from_the_probe():
    reset()
    used = [0]

    def mem_info():
        used[0] += 1
        return (1000 - used[0], 1000)

    srv = Server(hbm_budget_bytes=100, session_budget_bytes=10, max_active=2, session_factory=FakeSession,
                 mem_info=mem_info)
    serve(srv, scenes(2, requests=1))
    assert srv.peak_device_bytes == used[0]
