"""The serving loop's admission policy on the host, with fake sessions (no GPU): at most max_active
sessions, admission against the sessions' measured bytes plus their growth margins, a session that
would outgrow the budget throttled (its next request waits) instead of failing, waiting scenes
admitted in arrival order as sessions finish, every request served once, and latency counted from
arrival (deferral and throttling included)."""
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

    def __init__(self, hbm_budget_bytes, work_s=0.03, name=None, grow=0):
        with FakeSession.lock:
            FakeSession.active += 1
            FakeSession.peak = max(FakeSession.peak, FakeSession.active)
            FakeSession.made.append(name)
        self.work_s = work_s
        self.grow = grow
        self.bytes = 0
        self.results = []
        self.stream = types.SimpleNamespace(synchronize=lambda: None)
        self.field = types.SimpleNamespace(stats=lambda: {"n_gaussians": 0},
                                           get_gaussians=lambda with_adam=False: None,
                                           footprint=lambda: (0, self.bytes))

    def arrive(self, cam, target, pts_xyz=None, pts_rgb=None, tracks=None, arrival_time=None):
        time.sleep(self.work_s)
        self.bytes += self.grow  # the field grows with every arriving image
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


def scenes(n, requests=3, spacing=0.0, grow=0, gap=0.001):
    req = dict(cam=None, target=None)
    return [Scene(f"s{k}", [(k * spacing + gap * r, req) for r in range(requests)], config=dict(name=f"s{k}", grow=grow))
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
    """Before any session has measured its memory, admission counts the estimate: 2 x 10 <= 25 <
    3 x 10, so the third and fourth scenes, arriving with the first two, are deferred."""
    reset()
    srv = Server(hbm_budget_bytes=25, session_budget_bytes=10, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(4))
    assert [e[2] for e in log if e[1] == "admit"][:2] == ["s0", "s1"]
    assert {e[2] for e in log if e[1] == "defer"} >= {"s2"}
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


def test_admission_follows_measured_memory_not_a_fixed_reservation():
    """Sessions whose fields stay small leave room: with an estimate of 10 bytes each and a budget
    of 25, the first two are admitted on the estimate; once each has measured its use (1 byte after
    its first request, margin 2 x 1), the others fit and are admitted while the first two still run."""
    reset()
    srv = Server(hbm_budget_bytes=25, session_budget_bytes=10, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    sc = scenes(4, requests=6, grow=0)
    for s in sc:
        s.config["grow"] = 1
    sc = [Scene(s.sid, s.requests, dict(s.config, work_s=0.02)) for s in sc]
    out, log = serve(srv, sc)
    assert len(out) == 4 and FakeSession.peak == 4
    assert not any(e[1] == "throttle" for e in log)


def test_a_growing_session_is_throttled_instead_of_failing():
    """Two sessions growing by 10 bytes per request under a 45-byte budget: they cannot both keep
    growing, so one waits (a 'throttle' event, time counted in its latency) until the other finishes;
    every request is served and nothing raises."""
    reset()
    srv = Server(hbm_budget_bytes=45, session_budget_bytes=5, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(2, requests=3, grow=10))
    assert all(len(r["results"]) == 3 for r in out.values())
    assert any(e[1] == "throttle" for e in log)
    assert sum(r["throttled_s"] for r in out.values()) > 0
    s = summarize(out, srv.wall_s, log)
    assert set(s["by_admission"]) == {"admitted_on_arrival", "deferred"}


def test_deferred_and_admitted_scenes_are_reported_apart():
    reset()
    srv = Server(hbm_budget_bytes=10, session_budget_bytes=10, max_active=4, session_factory=FakeSession,
                 mem_info=lambda: (0, 0))
    out, log = serve(srv, scenes(2, requests=2))
    s = summarize(out, srv.wall_s, log)
    assert s["by_admission"]["deferred"]["n"] == 2 and s["by_admission"]["admitted_on_arrival"]["n"] == 2
    assert s["per_session"]["s1"]["deferred"] and not s["per_session"]["s0"]["deferred"]
    assert s["by_admission"]["deferred"]["p50"] > s["by_admission"]["admitted_on_arrival"]["p50"]
