"""Serving loop: concurrent scene sessions on one GPU with continuous admission by HBM budget.

Each scene is a stream of requests (one per arriving image, with its arrival time).  A scene is
admitted as a session once its first request has arrived, a session slot is free and the
session's HBM budget fits in what the server has left; until then its requests wait (deferred).
Admitted sessions run concurrently, each on its own CUDA stream and host thread (the C ABI calls
release the GIL), so their kernels overlap on the device.  When a session has served its last
request its memory is released and deferred scenes are admitted in arrival order.  Latency of a
request = completion time - arrival time, queueing and deferral included.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import GSError, _torch
from .streaming import StreamingSession, percentile


class Scene:
    def __init__(self, sid, requests, config=None):
        """requests: list of (arrival_s, dict(cam=..., target=..., pts_xyz=..., pts_rgb=..., tracks=...))."""
        self.sid = sid
        self.requests = sorted(requests, key=lambda r: r[0])
        self.config = dict(config or {})


class Server:
    def __init__(self, hbm_budget_bytes, session_budget_bytes, max_active=4, session_factory=None, mem_info=None):
        """session_factory(hbm_budget_bytes=..., **scene.config) makes a scene's session (default: a
        StreamingSession); mem_info() -> (free, total) device bytes, sampled for the peak (default:
        torch.cuda.mem_get_info).  Both are replaceable so that the admission policy runs without a GPU."""
        self.hbm_budget = int(hbm_budget_bytes)
        self.session_budget = int(session_budget_bytes)
        self.max_active = int(max_active)
        self.session_factory = session_factory or StreamingSession
        self.mem_info = mem_info
        self.log = []  # (time_s, event, scene id)

    def run(self, scenes, keep_fields=False, poll_s=0.0005):
        """Serve every scene; returns {sid: dict(results, latency, state)}."""
        mem_info = self.mem_info or _torch().cuda.mem_get_info
        t_start = time.perf_counter()
        lock = threading.Lock()
        pending = sorted(scenes, key=lambda s: s.requests[0][0] if s.requests else 0.0)
        active, done, out, errors = {}, set(), {}, []
        reserved = [0]
        peak_used = [0]

        def now():
            return time.perf_counter() - t_start

        def worker(scene):
            sess = None
            try:
                sess = self.session_factory(hbm_budget_bytes=self.session_budget, **scene.config)
                for arrival, req in scene.requests:
                    wait = arrival - now()
                    if wait > 0:
                        time.sleep(wait)
                    sess.arrive(req["cam"], req["target"], req.get("pts_xyz"), req.get("pts_rgb"), req.get("tracks"),
                                arrival_time=t_start + arrival)
                state = sess.field.get_gaussians(with_adam=True) if keep_fields else None
                out[scene.sid] = dict(results=sess.results, latency=sess.latency(), state=state,
                                      stats=sess.field.stats())
            except GSError as e:
                errors.append((scene.sid, e))
            finally:
                if sess is not None:
                    sess.stream.synchronize()
                    sess.close()
                with lock:
                    reserved[0] -= self.session_budget
                    del active[scene.sid]
                    done.add(scene.sid)
                    self.log.append((now(), "finish", scene.sid))

        while pending or active:
            with lock:
                while (pending and len(active) < self.max_active
                       and reserved[0] + self.session_budget <= self.hbm_budget
                       and (not pending[0].requests or pending[0].requests[0][0] <= now())):
                    sc = pending.pop(0)
                    reserved[0] += self.session_budget
                    th = threading.Thread(target=worker, args=(sc,), daemon=True)
                    active[sc.sid] = th
                    self.log.append((now(), "admit", sc.sid))
                    th.start()
                if pending and pending[0].requests and pending[0].requests[0][0] <= now() and \
                        (len(active) >= self.max_active or reserved[0] + self.session_budget > self.hbm_budget):
                    if not self.log or self.log[-1][1:] != ("defer", pending[0].sid):
                        self.log.append((now(), "defer", pending[0].sid))
            free, total = mem_info()
            peak_used[0] = max(peak_used[0], total - free)
            time.sleep(poll_s)
        if errors:
            raise errors[0][1]
        self.wall_s = now()
        self.peak_device_bytes = peak_used[0]
        return out


def summarize(out, wall_s):
    """Per-session p50/p99 latency and aggregate Gaussian-pixel pairs/s."""
    lat_all, pairs = [], 0
    per = {}
    for sid, r in out.items():
        lat = [x["latency_s"] for x in r["results"]]
        lat_all += lat
        pairs += sum(x["pairs"] for x in r["results"])
        per[sid] = dict(p50=percentile(lat, 50), p99=percentile(lat, 99), n=len(lat))
    return dict(per_session=per, p50=percentile(lat_all, 50), p99=percentile(lat_all, 99),
                pairs_per_s=pairs / wall_s if wall_s > 0 else float("nan"))
