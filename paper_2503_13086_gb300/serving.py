"""Serving loop: concurrent scene sessions on one GPU with continuous admission by measured HBM.

Each scene is a stream of requests (one per arriving image, with its arrival time).  A scene is
admitted as a session once its first request has arrived, a session slot is free and the device
memory the active sessions hold -- each session's measured bytes in use (gs_field_stats) plus a
growth margin -- leaves room for a new session's initial estimate; until then its requests wait
(deferred).  Admitted sessions run concurrently, each on its own CUDA stream and host thread (the C
ABI calls release the GIL), so their kernels overlap on the device.  Before each request a session
checks that its own measured bytes plus its margin, with the others' commitments, still fit the
budget; if not it waits (throttled) until a session finishes, instead of failing mid-stream.  When
every active session is throttled, the earliest admitted proceeds.  A session's margin is twice
the largest growth one request has caused so far (the initial estimate before its first request).
When a session has served its last request its memory is released and deferred scenes are admitted
in arrival order.  Latency of a request = completion time - arrival time, with deferral and
throttling included.
"""
from __future__ import annotations

import threading
import time

from . import GSError, _torch
from .streaming import StreamingSession, percentile


class Scene:
    def __init__(self, sid, requests, config=None):
        """requests: list of (arrival_s, dict(cam=..., target=..., pts_xyz=..., pts_rgb=..., tracks=...))."""
        self.sid = sid
        self.requests = sorted(requests, key=lambda r: r[0])
        self.config = dict(config or {})


class Server:
    def __init__(self, hbm_budget_bytes, session_budget_bytes, max_active=4, session_factory=None, mem_info=None,
                 growth_factor=2.0):
        """hbm_budget_bytes: device memory the sessions may hold together.  session_budget_bytes: the
        estimate a new session is admitted against (before it has measured anything).
        session_factory(hbm_budget_bytes=..., **scene.config) makes a scene's session (default: a
        StreamingSession; its field gets the whole budget as its own cap, the server enforcing the
        shared one); its ``field.footprint()`` returns (Gaussians, bytes in use).  mem_info() ->
        (free, total) device bytes, sampled for the peak (default: torch.cuda.mem_get_info).  Both are
        replaceable so that the policy runs without a GPU."""
        self.hbm_budget = int(hbm_budget_bytes)
        self.session_estimate = int(session_budget_bytes)
        self.max_active = int(max_active)
        self.growth_factor = float(growth_factor)
        self.session_factory = session_factory or StreamingSession
        self.mem_info = mem_info
        self.log = []  # (time_s, event, scene id): admit, defer, throttle, finish

    def run(self, scenes, keep_fields=False, poll_s=0.0005):
        """Serve every scene; returns {sid: dict(results, latency, state, stats, deferred_s, throttled_s)}."""
        mem_info = self.mem_info or _torch().cuda.mem_get_info
        t_start = time.perf_counter()
        cond = threading.Condition()
        pending = sorted(scenes, key=lambda s: s.requests[0][0] if s.requests else 0.0)
        active = {}      # sid -> dict(thread, used, margin, order, waiting)
        out, errors = {}, []
        peak_used = [0]
        order = [0]

        def now():
            return time.perf_counter() - t_start

        def committed(exclude=None):
            return sum(a["used"] + a["margin"] for sid, a in active.items() if sid != exclude)

        def wait_for_room(sid):
            """Block until this session's next request fits the budget (or it must go first)."""
            me = active[sid]
            throttled = 0.0
            while True:
                fits = committed(sid) + me["used"] + me["margin"] <= self.hbm_budget
                others = [a for o, a in active.items() if o != sid]
                all_wait = all(a["waiting"] for a in others)
                first = all(me["order"] < a["order"] for a in others)
                if fits or not others or (all_wait and first):
                    me["waiting"] = False
                    return throttled
                if not me["waiting"]:
                    self.log.append((now(), "throttle", sid))
                me["waiting"] = True
                t0 = time.perf_counter()
                cond.wait(timeout=0.05)
                throttled += time.perf_counter() - t0

        def worker(scene, deferred_s):
            sess = None
            throttled = 0.0
            try:
                sess = self.session_factory(hbm_budget_bytes=self.hbm_budget, **scene.config)
                for arrival, req in scene.requests:
                    wait = arrival - now()
                    if wait > 0:
                        time.sleep(wait)
                    with cond:
                        throttled += wait_for_room(scene.sid)
                    sess.arrive(req["cam"], req["target"], req.get("pts_xyz"), req.get("pts_rgb"), req.get("tracks"),
                                arrival_time=t_start + arrival)
                    used = int(sess.field.footprint()[1])
                    with cond:
                        me = active[scene.sid]
                        me["growth"] = max(me["growth"], used - me["used"])
                        me["used"] = used
                        me["margin"] = int(self.growth_factor * me["growth"])
                        cond.notify_all()
                state = sess.field.get_gaussians(with_adam=True) if keep_fields else None
                out[scene.sid] = dict(results=sess.results, latency=sess.latency(), state=state,
                                      stats=sess.field.stats(), deferred_s=deferred_s, throttled_s=throttled)
            except GSError as e:
                errors.append((scene.sid, e))
            finally:
                if sess is not None:
                    sess.stream.synchronize()
                    sess.close()
                with cond:
                    del active[scene.sid]
                    self.log.append((now(), "finish", scene.sid))
                    cond.notify_all()

        while True:
            with cond:
                if not pending and not active:
                    break
                while (pending and len(active) < self.max_active
                       and committed() + self.session_estimate <= self.hbm_budget
                       and (not pending[0].requests or pending[0].requests[0][0] <= now())):
                    sc = pending.pop(0)
                    first_arrival = sc.requests[0][0] if sc.requests else now()
                    order[0] += 1
                    active[sc.sid] = dict(used=0, margin=self.session_estimate, growth=0, order=order[0],
                                          waiting=False)
                    th = threading.Thread(target=worker, args=(sc, max(0.0, now() - first_arrival)), daemon=True)
                    active[sc.sid]["thread"] = th
                    self.log.append((now(), "admit", sc.sid))
                    th.start()
                if pending and pending[0].requests and pending[0].requests[0][0] <= now() and \
                        (len(active) >= self.max_active or committed() + self.session_estimate > self.hbm_budget):
                    if not any(e[1] == "defer" and e[2] == pending[0].sid for e in self.log):
                        self.log.append((now(), "defer", pending[0].sid))
            free, total = mem_info()
            peak_used[0] = max(peak_used[0], total - free)
            time.sleep(poll_s)
        if errors:
            raise errors[0][1]
        self.wall_s = now()
        self.peak_device_bytes = peak_used[0]
        return out


def summarize(out, wall_s, log=None):
    """Per-session p50/p99 latency, the same over the scenes admitted on arrival and over the deferred
    ones (from the server's log), and aggregate Gaussian-pixel pairs/s."""
    lat_all, pairs = [], 0
    per = {}
    deferred = {e[2] for e in (log or []) if e[1] == "defer"}
    groups = {"admitted_on_arrival": [], "deferred": []}
    for sid, r in out.items():
        lat = [x["latency_s"] for x in r["results"]]
        lat_all += lat
        pairs += sum(x["pairs"] for x in r["results"])
        per[sid] = dict(p50=percentile(lat, 50), p99=percentile(lat, 99), n=len(lat),
                        deferred=sid in deferred, deferred_s=r.get("deferred_s", 0.0),
                        throttled_s=r.get("throttled_s", 0.0))
        groups["deferred" if sid in deferred else "admitted_on_arrival"] += lat
    return dict(per_session=per, p50=percentile(lat_all, 50), p99=percentile(lat_all, 99),
                by_admission={k: dict(p50=percentile(v, 50), p99=percentile(v, 99), n=len(v))
                              for k, v in groups.items()},
                pairs_per_s=pairs / wall_s if wall_s > 0 else float("nan"))
