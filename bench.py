"""Benchmark of the On-the-Fly GS hot path on GB300.

Headline (one "step" = one pass of the whole hot path): the scene-scale single view -- 200k
Gaussians in a ring-shaped outdoor-like volume, one 1297 x 840 view, SH degree 3, loss
0.8 L1 + 0.2 D-SSIM: projection, binning, sort, blend forward, loss, blend backward, projection
backward and Adam with the per-image learning rate, through the session API (gs_optimize_step),
replayed from a CUDA graph.  value = Gaussian-pixel pairs per second (P counted by the oracle's
definition: per pixel, list entries evaluated up to its stop) / step device time.  The same line
carries, measured in the same run with the clocks sampled during each:
  integration_latency_s  the streaming session at full length (150 arrivals, the field growing to
                         about 1.5-1.9M Gaussians): p50/p99 new-image integration latency of the
                         plain per-view, graph per-view and batched paths, PSNR against the targets
                         and of the GPU's renders against the oracle's renders of the final field;
  batched_step           500k Gaussians x 9 mixed-size views per step, per-kernel times;
  serving                4 concurrent scenes admitted by HBM budget, p50/p99 per session.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs|reference]
                  [--workload scene|batched|serve|stream] [--segments stream,batched,serve|none]

--impl reference times the oracle (CPU, fp32, one thread) on the same workload.  Under torchrun
each rank runs its own independent session (weak scaling, no data exchange); rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gsinputs as gi  # noqa: E402

METRIC = "new-image integration latency p50/p99 (s); fwd+bwd Gaussian-pixel pairs/s"
N_GAUSS = 200_000
W, H = 1297, 840
WORKLOAD = "scene-scale single view: 200k Gaussians (ring volume), 1297x840, SH3, 0.8 L1 + 0.2 D-SSIM, fwd+bwd+Adam"
KERNELS = ["K1 project", "K2 scan", "K3 emit", "K4 sort", "K5 ranges+order", "K6 blend fwd", "K7 loss", "K8 blend bwd",
           "K9+K10 project bwd + Adam"]


def workload_config(ws=1):
    """The workload as both arms name it (the same dict in the CUDA line and the reference line)."""
    return {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "width": W, "height": H, "sh_degree": 3,
            "loss": "0.8 L1 + 0.2 D-SSIM", "tiling": "16x16 tiles (3DGS), blend batch 256",
            "l2": "flushed before every timed step (256 MiB write, untimed)",
            "state": "every timed step starts from the same snapshot (device copy, untimed)",
            "parallelism": f"{ws} independent session(s), one per GPU"}


def make_workload(seed):
    p = gi.ring_scene(N_GAUSS, seed=seed, stride=N_GAUSS)
    cam = gi.ring_camera(0.3 + 0.7 * seed, W, H, 1000.0)
    tgt = gi.uniform_target(W, H, seed + 1)
    return p, cam, tgt


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per kernel launch: FP32 lane-operations for the blend kernels,
# counted from the formulas they evaluate; bytes for the memory-bound kernels.
def kernel_work(k, st, n, passes):
    P, B, M = st["pairs"], st["blended"], st["instances"]
    if k == 5:   # K6: exponent + cutoff test for every evaluated pair, the blend for blended ones
        return "alu", 8.0 * P + 10.0 * B
    if k == 7:   # K8: 45 lane-ops per blended pair; pairs a pixel did not blend cost nothing
        return "alu", 45.0 * B
    if k == 8:   # K9+K10: read + write p, m, v (3 x 236 B each way) + 48 B per instance + count/offset
        return "hbm", 1416.0 * n + 48.0 * M + 8.0 * n
    if k == 3:   # K4: one read and one write of key + value per pass
        return "hbm", 24.0 * M * passes
    if k == 0:   # K1: geometry of every Gaussian, SH of the visible ones, the records written
        return "hbm", 44.0 * n + st["visible"] * (192.0 + 80.0)
    if k == 6:   # K7: forward reads render + target (6 H W floats) and writes the 9 partial maps;
        # backward reads the partials, render and target and writes dL/dimage (3 H W)
        return "hbm", 4.0 * W * H * (6 + 9 + 9 + 6 + 3)
    if k == 2:
        return "hbm", 12.0 * M + 24.0 * n
    return "hbm", 8.0 * n


# The per-pair instruction counts the scope table states for the two blend kernels (K6 "~16 FP32
# instructions + 1 ex2 per pair" over the evaluated pairs; K8 "~55-65" over the pairs it walks, the
# blended ones), reported beside the finer counts above.
SURVEY_PER_PAIR = {5: ("pairs", 16.0), 7: ("blended", 60.0)}


def device_sm_count(default=152):
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return default


def roofline(kernel_ms, steps, st, n, passes, peaks, peaks_kind, traffic, n_sms=None):
    per = [k / max(1, steps) for k in kernel_ms]
    dom = int(np.argmax(per))
    n_sms = device_sm_count() if n_sms is None else int(n_sms)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12

    def frac_of(k):
        t = per[k] * 1e-3
        bound, work = kernel_work(k, st, n, passes)
        if bound == "alu":
            peak = alu_peak
            unit = "Tops/s"
            src = (f"{n_sms} SMs (cudaDeviceProp.multiProcessorCount) x 128 FP32 lanes x {sm_mhz:.0f} MHz "
                   f"(sm_max_mhz, {peaks_kind}): derived from unit counts and clock")
            ach = work / t / 1e12 if t > 0 else 0.0
        else:
            peak = peaks["hbm_gbs"]
            unit, src = "GB/s", f"HBM copy, {peaks_kind}"
            ach = work / t / 1e9 if t > 0 else 0.0
        return bound, work, ach, peak, unit, src

    bound, work, ach, peak, unit, src = frac_of(dom)
    # every kernel against its own roofline (the same algorithmic-work definitions)
    each = {}
    for k, nm in enumerate(KERNELS):
        b, _, a, pk, _, _ = frac_of(k)
        each[nm] = {"bound": b, "frac": round(a / pk, 4)}
    out = dict(kernel=KERNELS[dom], bound=bound, achieved=ach, peak=peak, unit=unit, frac=ach / peak,
               traffic=traffic.get(KERNELS[dom]), peak_source=src, work_per_launch=work, n_sms=n_sms,
               per_kernel_ms={nm: round(x, 4) for nm, x in zip(KERNELS, per)}, per_kernel_frac=each)
    if dom in SURVEY_PER_PAIR and per[dom] > 0:
        key, ops = SURVEY_PER_PAIR[dom]
        w2 = ops * st[key]
        a2 = w2 / (per[dom] * 1e-3) / 1e12
        out["survey_count"] = {"ops_per_pair": ops, "pairs": key, "work_per_launch": w2, "achieved": a2,
                               "frac": a2 / alu_peak}
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the committed ncu
# summaries of the current kernels (profiles/), taken with the tiling below; None for a kernel
# changed since its capture.
TRAFFIC_TILING = (16, 16, 256)
TRAFFIC = {"K8 blend bwd": 62.5e6, "K6 blend fwd": 21.7e6, "K9+K10 project bwd + Adam": 253.5e6,
           "K4 sort": 5 * 4.1e6, "K7 loss": 94.3e6}


def cpu_baseline_run(steps, warmup, seed=0, rows=None):
    """The oracle (fp32, one thread) doing full steps of the same workload; with rows, each step
    covers a horizontal band of that many rows in the middle of the view (the same camera, its
    principal point moved), so that many steps stay within a bounded CPU time."""
    import oracle
    from oracle import Camera
    p, cam, tgt = make_workload(seed)
    h = H if rows is None else int(min(H, max(16, rows)))
    y0 = (H - h) // 2
    c = Camera(cam["R"], cam["t"], cam["fx"], cam["fy"], cam["cx"], cam["cy"] - y0, cam["width"], h)
    tg = np.ascontiguousarray(tgt[:, y0:y0 + h, :])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lrs = [1.6e-4 * 7.0, 5e-3, 1e-3, 0.05, 2.5e-3, 1.25e-4]
    times, pairs = [], []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        L, g, r = oracle.loss_and_grad(p, [c], [tg], lam=0.2, prec="f32")
        oracle.adam(p, g, m, v, lrs, s + 1, prec="f32")
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
            pairs.append(oracle.pairs(r))
    return float(np.sum(pairs) / np.sum(times)), float(np.mean(times)), int(np.mean(pairs))


REFERENCE_BUDGET_S = 120.0  # the reference arm's CPU time for all its steps, about
ORACLE_STEP_S = 2.5         # one full oracle step of the workload on one GPU-box host core


def reference_rows(steps, warmup):
    """Rows of the view each reference step covers: the whole view while K + W full steps fit the
    budget, else a band small enough that they do."""
    total = (steps + warmup) * ORACLE_STEP_S
    return None if total <= REFERENCE_BUDGET_S else max(16, int(H * REFERENCE_BUDGET_S / total))


_BARRIER = None


def _oracle_worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(seed):
    """One full oracle step (fp32, one thread) in a pool process, started together with the others:
    (start, end, pairs) on the host's monotonic clock."""
    import oracle
    from oracle import Camera
    p, cam, tgt = make_workload(0)
    c = Camera(cam["R"], cam["t"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"])
    m, v = np.zeros_like(p), np.zeros_like(p)
    lrs = [1.6e-4 * 7.0, 5e-3, 1e-3, 0.05, 2.5e-3, 1.25e-4]
    oracle.lib()
    _BARRIER.wait()
    t0 = time.perf_counter()
    L, g, r = oracle.loss_and_grad(p, [c], [tgt], lam=0.2, prec="f32")
    oracle.adam(p, g, m, v, lrs, 1, prec="f32")
    return t0, time.perf_counter(), oracle.pairs(r)


def cpu_baseline_all_cores(procs=None):
    """The same oracle step in one process per host core at once (a spawn pool; every process starts
    its step at a common barrier): pairs of all steps / the span from the first start to the last
    end."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(barrier,)) as pool:
        res = pool.map(_oracle_worker, range(procs), chunksize=1)
    span = max(e for _, e, _ in res) - min(s for s, _, _ in res)
    pairs = sum(pp for _, _, pp in res)
    return pairs / span, procs, span, int(pairs / procs)


def combine_ranks(ms, pairs, ws, device):
    """Whole-job figures over the ranks' independent sessions: the slowest rank's time (max) and
    the pairs of all ranks (sum).  One rank: unchanged."""
    if ws <= 1:
        return ms, pairs
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, pairs], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t)
    return float(tmax[0].item()), float(t[1].item())


def host_cpu():
    """The host the oracle runs on: logical CPUs and the CPU model (lscpu's "Model name", else
    /proc/cpuinfo's "model name", else the machine type)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine()}


def run_reference(args):
    """The oracle (fp32, one host thread) on the same workload: W untimed and K timed full steps
    (about 2.3 s each on the GPU machine's Arm host), printed with the steps it actually ran."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    rows = reference_rows(args.steps, args.warmup)
    val, sec, pairs = cpu_baseline_run(args.steps, args.warmup, rows=rows)
    sample = (f"{args.steps} full oracle steps (after {args.warmup} untimed) of the workload, {pairs} pairs each"
              if rows is None else
              f"{args.steps} oracle steps (after {args.warmup} untimed), each over the middle {rows} of the view's "
              f"{H} rows (all 200k Gaussians projected; {pairs} pairs each) to bound the CPU time")
    line = {"metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ring scene, uniform target; the paper's scenes are not available)",
            "impl": "reference", "config": workload_config(ws),
            "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": sample + ", fp32, one thread", "host": host_cpu()},
            "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# streaming: new-image integration latency, plain per-view eager path vs batched graph path
# ------------------------------------------------------------------------------------------
def stream_inputs(n_images, seed=0, n_gt=1_500_000, Wv=W, Hv=H, pts_range=(5000, 20001)):
    import torch
    import paper_2503_13086_gb300 as gs
    gt = gi.ring_scene(n_gt, seed=seed + 100, stride=n_gt + (-n_gt) % 32)
    cams = gi.random_walk_cameras(n_images, seed=seed + 7, W=Wv, H=Hv, f=1000.0 * Wv / W)
    f = gs.Field(scene_extent=7.0)
    f.set_gaussians(gt, n_gt)
    targets = [f.render(c).clone() for c in cams]
    torch.cuda.synchronize()
    f.close()
    rng = np.random.default_rng(seed)
    pts = [gi.sparse_points(gt, n_gt, c, int(rng.integers(*pts_range)), seed=seed * 1000 + k)
           for k, c in enumerate(cams)]
    return cams, targets, pts


def run_stream(cams, targets, pts, batch, graph, asyn, T_I=200, k_neighbours=8, scaling=0, kernel_times=False,
               thresh=0.0, sparse=0, keep_field=False, weights=None, prune_opacity=None):
    import torch
    from paper_2503_13086_gb300.streaming import StreamingSession
    w = {} if weights is None else dict(lambda_l1=weights[0], lambda_ssim=weights[1], lambda_load=weights[2])
    sess = StreamingSession(T_I=T_I, N_m=k_neighbours + 1, batch_views=batch, use_graph=graph, async_steps=asyn,
                            scene_extent=7.0, seed=3, batch_scaling=scaling, add_dist_thresh=thresh,
                            sparse_adam=sparse, prune_opacity=prune_opacity, **w)
    if kernel_times:
        sess.field.set_timing(True)
    pairs, add_s, int_s = 0, [], []
    t0 = time.perf_counter()
    for c, t, (xyz, rgb, tr) in zip(cams, targets, pts):
        r = sess.arrive(c, t, xyz, rgb, tr)
        pairs += r["pairs"]
        add_s.append(r["add_image_s"])
        int_s.append(r["integrate_s"])
    wall = time.perf_counter() - t0
    lat = sess.latency()
    psnr = sess.psnr(cams, targets)
    n = sess.field.stats()["n_gaussians"]
    final = sess.field.get_gaussians() if keep_field else None
    kt = None
    if kernel_times:
        kms, ksteps = sess.field.kernel_times()
        kt = {nm: round(x / max(1, ksteps), 4) for nm, x in zip(KERNELS, kms)}
    torch.cuda.synchronize()
    sess.close()
    steps = sum(r["steps"] for r in sess.results)
    return dict(p50_s=lat["p50"], p99_s=lat["p99"], psnr_db=psnr, n_gaussians=n, arrivals=len(cams),
                ms_per_step=1e3 * float(np.sum(int_s)) / max(1, steps),
                pruned=int(sum(r.get("pruned", 0) for r in sess.results)),
                pairs_per_s=pairs / wall, batch_views=batch, graph=bool(graph), steps_between_syncs=asyn,
                batch_scaling=scaling, sparse_adam=bool(sparse), add_image_mean_s=float(np.mean(add_s)),
                integrate_mean_s=float(np.mean(int_s)),
                **({"kernel_ms_per_step": kt} if kt else {}), **({"field": final} if keep_field else {}))


def run_gs(args):
    import torch
    import paper_2503_13086_gb300 as gs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gs.load()
    p, cam, tgt = make_workload(rank)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    def make_field(tiling):
        f = gs.Field(stream=stream, scene_extent=7.0, lambda_ssim=0.2, use_graph=1, tiling=tiling)
        f.set_gaussians(p)
        return f, f.add_image(cam, tgt)

    def timed_loop(f, img, steps):
        """steps timed optimisation steps, each from the same snapshot (restored untimed) after an
        untimed L2 flush.  Two clocks, both CUDA events on the session's stream: the library's events
        around the enqueued step (the step's device time; the step's own readback of its ledger and
        loss follows them), and events recorded here around the call (which also cover that readback
        and the host's return from it)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        acc = dict(pairs=0, blended=0, instances=0, launches=0, device_ms=0.0)
        for k in range(steps):
            f.restore()
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            f.optimize_step([img])
            ev[k][1].record(stream)
            st = f.stats()
            acc["pairs"] += st["last_pairs"]
            acc["blended"] += st["last_blended"]
            acc["instances"] += st["last_instances"]
            acc["launches"] += st["last_kernels"]
            acc["device_ms"] += st["last_run_ms"]
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in ev)), acc

    # the autotuned session (the library's default): its choice and step time, reported beside
    # the headline, which uses the 16 x 16 binning the pair count P is defined on
    auto = None
    if not args.no_autotune_report:
        fa, img_a = make_field(None)
        tune = fa.autotune([img_a], reps=5)
        for _ in range(args.warmup):
            fa.optimize_step([img_a])
        fa.snapshot()
        _, auto_acc = timed_loop(fa, img_a, args.steps)
        auto_tiling = fa.stats()["last_tiling"]
        fa.close()
        auto_ms = auto_acc["device_ms"]
        auto = {"tiling": f"{auto_tiling[0]}x{auto_tiling[1]}/{auto_tiling[2]}",
                "ms_per_step": auto_ms / max(1, args.steps), "pairs_per_step": int(auto_acc["pairs"] / max(1, args.steps)),
                "pairs_per_s": auto_acc["pairs"] / (auto_ms * 1e-3),
                "candidates_ms": {f"{c[0]}x{c[1]}/{c[2]}": round(t, 4) for c, t in tune["candidates"]},
                "note": "the same workload with the tiling the autotuner picks; P then counts that binning's list "
                        "entries (smaller tiles evaluate fewer pairs)"}

    field, img = make_field(None if args.tiling == "auto" else tuple(int(x) for x in args.tiling.split("x")))
    for _ in range(args.warmup):
        field.optimize_step([img])
    field.snapshot()

    def sync_all():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sync_all()
    sampler.start()
    call_ms, acc = timed_loop(field, img, args.steps)
    launches = acc.pop("launches")
    ms = acc.pop("device_ms")
    sync_all()
    clocks = sampler.stop()
    # per-kernel times from a second run of the same steps with an event around every kernel (the
    # events sit between the kernels of the replayed graph, so that run is not the timed one)
    field.set_timing(True)
    timed_loop(field, img, args.steps)
    sync_all()
    kms, ksteps = field.kernel_times()
    field.set_timing(False)
    tiling = field.stats()["last_tiling"]
    ms_max, pairs_total = combine_ranks(ms, float(acc["pairs"]), ws, "cuda")
    call_ms_max, _ = combine_ranks(call_ms, 0.0, ws, "cuda")
    value = pairs_total / (ms_max * 1e-3)

    # end to end through the C ABI, as a user calls it: the step's target as decoded (H x W x 3,
    # pinned host memory) -> device (transposed there by gs_set_image's kernel), the step, and the
    # library's readback of the step's ledger and loss; all inside the timed region
    tgt_hwc = torch.from_numpy(np.ascontiguousarray(np.transpose(tgt, (1, 2, 0)))).pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    e2e_pairs, e2e_h2d, e2e_d2h = 0, 0, 0
    sync_all()
    for k in range(args.steps):
        field.restore()
        e2e_ev[k][0].record(stream)
        field.set_image(img, tgt_hwc)
        field.optimize_step([img])
        e2e_ev[k][1].record(stream)
        st = field.stats()
        e2e_pairs += st["last_pairs"]
        e2e_h2d += tgt_hwc.numel() * 4 + st["last_h2d_bytes"]
        e2e_d2h += st["last_d2h_bytes"]
    sync_all()
    e2e_ms = float(sum(a.elapsed_time(b) for a, b in e2e_ev))
    e2e_ms, e2e_pairs = combine_ranks(e2e_ms, float(e2e_pairs), ws, "cuda")
    field.close()

    steps = max(1, args.steps)
    st_mean = {k: v / steps for k, v in acc.items()}
    tiles = (-(-W // tiling[0])) * (-(-H // tiling[1]))
    passes = (32 + int(tiles - 1).bit_length() + 7) // 8
    # visible Gaussians of the view (for K1's algorithmic bytes)
    ras = gs.Raster()
    ras.forward(torch.tensor(p, device="cuda"), N_GAUSS, [cam])
    st_mean["visible"] = int((ras.read(6, np.uint32) > 0).sum())
    ras.close()
    del flush
    torch.cuda.empty_cache()

    segments = {}
    if ws == 1:
        wanted = [x for x in args.segments.split(",") if x] if args.segments != "none" else []
        for name in wanted:
            fn = {"stream": segment_stream, "load": segment_load, "batched": segment_batched,
                  "serve": segment_serve}[name]
            smp = ClockSampler(local)
            smp.start()
            t0 = time.perf_counter()
            try:
                res = fn(args)
            except Exception as exc:  # a failed measurement is reported, the others still run
                res = {"error": f"{type(exc).__name__}: {exc}"}
            res["wall_s"] = time.perf_counter() - t0
            res["clocks"] = smp.stop()
            segments[name] = res
            torch.cuda.empty_cache()

    if rank == 0:
        peaks, kind = measured_peaks()
        rl = roofline(kms, ksteps, st_mean, N_GAUSS, passes, peaks, kind,
                      TRAFFIC if tuple(tiling) == TRAFFIC_TILING else {})
        cfg = workload_config(ws)
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded ring scene, uniform target; the paper's scenes are not available)",
                "config": cfg,
                "counts": {"instances": int(st_mean["instances"]), "pairs_per_step": int(st_mean["pairs"]),
                           "blended_pairs_per_step": int(st_mean["blended"]),
                           "tiling": f"{tiling[0]}x{tiling[1]}/{tiling[2]}", "graph": True},
                "timing": {"ms_per_step_device": ms_max / steps,
                           "ms_per_step_with_readback": call_ms_max / steps,
                           "note": "value: the library's CUDA events around each step's device work; the second "
                                   "figure adds the step's readback of its ledger and loss and the host's return "
                                   "(events recorded by the caller around gs_optimize_step)"},
                "e2e": {"value": e2e_pairs / (e2e_ms * 1e-3), "unit": "pairs/s",
                        "h2d_bytes_per_step": int(e2e_h2d // steps), "d2h_bytes_per_step": int(e2e_d2h // steps)},
                "gpu_launches": int(launches),
                "autotuned": auto,
                "roofline": rl, "clocks": clocks}
        if "stream" in segments and "graph_async_per_view" in segments["stream"]:
            sd = segments["stream"]
            line["integration_latency_s"] = {"p50": sd["graph_async_per_view"]["p50_s"],
                                             "p99": sd["graph_async_per_view"]["p99_s"], "detail": sd}
        for nm in ("load", "batched", "serve"):
            if nm in segments:
                line[{"load": "load_balance", "batched": "batched_step", "serve": "serving"}[nm]] = segments[nm]
        if not args.no_cpu_baseline and ws == 1:
            val, sec, pp = cpu_baseline_run(3, 0)
            line["cpu_baseline"] = {"value": val, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                                    "sample": f"3 full oracle steps of the workload ({pp} pairs each), fp32, one thread",
                                    "host": host_cpu()}
            aval, procs, span, app = cpu_baseline_all_cores()
            line["cpu_baseline_all_cores"] = {
                "value": aval, "unit": "pairs/s", "cores": procs, "kind": "oracle",
                "sample": f"{procs} processes (one per host core), one full oracle step each ({app} pairs), "
                          f"started together; pairs / {span:.2f} s from the first start to the last end",
                "host": host_cpu()}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def _oracle_render_worker(job):
    """Render one view of a saved field with the oracle (fp32); returns (view, image)."""
    import oracle
    from oracle import Camera
    path, n, cam = job
    prm = np.load(path, mmap_mode="r")
    c = Camera(cam["R"], cam["t"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"])
    r = oracle.render(np.ascontiguousarray(prm), [c], prec="f32", n=n)
    return r["outs"][0]["image"]


def oracle_psnr_of_field(params, cams, views):
    """PSNR of the field's GPU renders against the oracle's renders of the same field, per view (a
    spawn pool, one host process per view)."""
    import multiprocessing as mp
    import tempfile
    import torch
    import paper_2503_13086_gb300 as gs
    n = params.shape[1]
    stride = -(-n // 32) * 32
    padded = np.zeros((59, stride), np.float32)
    padded[:, :n] = params
    f = gs.Field(scene_extent=7.0, tiling=(16, 16, 256))
    f.set_gaussians(padded, n)
    gpu = [f.render(cams[v]).cpu().numpy() for v in views]
    f.close()
    torch.cuda.synchronize()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "field.npy")
        np.save(path, padded)
        with mp.get_context("spawn").Pool(len(views)) as pool:
            ref = pool.map(_oracle_render_worker, [(path, n, cams[v]) for v in views], chunksize=1)
    out = []
    for g_img, o_img in zip(gpu, ref):
        mse = float(np.mean((g_img.astype(np.float64) - o_img.astype(np.float64)) ** 2))
        out.append(10.0 * np.log10(1.0 / max(mse, 1e-30)))
    return out


_STREAM_INPUTS = {}


def cached_stream_inputs(n):
    """The full-length stream's inputs, made once per process (the load-balance segment reuses them)."""
    key = n
    if key not in _STREAM_INPUTS:
        _STREAM_INPUTS.clear()
        _STREAM_INPUTS[key] = stream_inputs(n, seed=0, n_gt=4_000_000)
    return _STREAM_INPUTS[key]


def segment_load(args):
    """The load-balancing term (Eq. 9-10) in a streaming session: the paper's weights 0.47 L1 +
    0.12 D-SSIM + 0.41 L_load, the load weight a tenth and a hundredth of it, and none (0.47 / 0.12 / 0),
    all pruning the Gaussians whose opacity fell below 0.005 after every arrival (3DGS's opacity
    pruning), over the first args.load_arrivals arrivals of the stream: Gaussian count, step time,
    latency, PSNR."""
    import gc
    import paper_2503_13086_gb300 as gs
    cams, targets, pts = cached_stream_inputs(args.arrivals)
    k = min(args.load_arrivals, len(cams))
    cams, targets, pts = cams[:k], targets[:k], pts[:k]
    gs.autotune_clear()
    run_stream(cams[:5], targets[:5], pts[:5], batch=1, graph=1, asyn=16, T_I=18, thresh=0.005)
    res = {}
    for name, w in (("paper_weights", (0.47, 0.12, 0.41)), ("load_0.041", (0.47, 0.12, 0.041)),
                    ("load_0.0041", (0.47, 0.12, 0.0041)), ("without_load", (0.47, 0.12, 0.0))):
        res[name] = run_stream(cams, targets, pts, batch=1, graph=1, asyn=16, thresh=0.005, weights=w,
                               prune_opacity=0.005)
        res[name]["weights_l1_ssim_load"] = list(w)
        gc.collect()
    res["workload"] = (f"the first {k} arrivals of the stream, per-view graph path, T_I = 200, opacity pruning "
                       f"below 0.005 after every arrival")
    return res


def segment_stream(args):
    """The streaming session at full length (150 arrivals at 1297 x 840 on a random walk with 60-80 %
    overlap, 5k-20k sparse points each, new points kept down to 0.005 from the field so it grows to
    about 1.5-1.9M Gaussians, T_I = 200 over the new image + 8 neighbours): new-image integration
    latency of the plain per-view eager path, the per-view path replayed from graphs, and the batched
    path (3 views per step, large-batch rates); PSNR against the targets, and of the GPU's renders of
    the final field against the oracle's renders of the same field."""
    import gc
    import paper_2503_13086_gb300 as gs
    cams, targets, pts = cached_stream_inputs(args.arrivals)
    gs.autotune_clear()
    warm = min(args.arrivals, 10)
    for b in (1, 3):
        run_stream(cams[:warm], targets[:warm], pts[:warm], batch=b, graph=1, asyn=16, T_I=18, scaling=1,
                   thresh=0.005)
    res = {}
    final = None
    for name, b, graph, asyn, scaling in (("plain_per_view", 1, 0, 1, 0), ("graph_async_per_view", 1, 1, 16, 0),
                                          ("batched3_graph_scaled", 3, 1, 16, 1)):
        r = run_stream(cams, targets, pts, batch=b, graph=graph, asyn=asyn, scaling=scaling, thresh=0.005,
                       kernel_times=(name == "graph_async_per_view"), keep_field=(name == "graph_async_per_view"))
        if "field" in r:
            final = r.pop("field")
        res[name] = r
        gc.collect()
    views = [int(x) for x in np.linspace(0, len(cams) - 1, 4).round()]
    res["oracle_render_psnr_db"] = {
        "views": views, "psnr_db": oracle_psnr_of_field(final, cams, views),
        "note": "the per-view graph path's final field rendered by the GPU and by the oracle (fp32, one host "
                "process per view) from 4 of the trajectory's cameras"}
    res["workload"] = (f"{args.arrivals} arrivals, 1297x840, random walk 60-80% overlap, 5k-20k sparse points each, "
                       f"new-point threshold 0.005, T_I = 200 over the new image + 8 neighbours, 4M-Gaussian hidden "
                       f"scene")
    res["autotune"] = f"tiling autotuned per class, cache filled by untimed sessions over the first {warm} arrivals"
    return res


def segment_batched(args):
    """The batched local & semi-global step: 500k Gaussians, 9 views at mixed sizes, one graph."""
    return batched_step(steps=max(3, min(args.steps, 20)), warmup=3)


def segment_serve(args):
    """Multi-session serving: 4 scenes at 1920x1080 / 1280x720, each growing to about 3M Gaussians."""
    return serve(args)


def batched_step(steps, warmup):
    """Batched local & semi-global step: 500k Gaussians, 9 views at mixed sizes (960 x 540 to
    1600 x 1060), autotuned tiling, one graph replay per step; device time from CUDA events."""
    import torch
    import paper_2503_13086_gb300 as gs
    torch.cuda.set_device(0)
    n = 500_000
    p = gi.ring_scene(n, seed=5, stride=n)
    cams = gi.batched_views(9, seed=2)
    stream = torch.cuda.Stream()
    field = gs.Field(stream=stream, scene_extent=7.0, use_graph=1, tiling=None)  # autotuned
    field.set_gaussians(p)
    ids = [field.add_image(c, gi.uniform_target(c["width"], c["height"], k)) for k, c in enumerate(cams)]
    tune = field.autotune(ids, reps=3)
    for _ in range(warmup):
        field.optimize_step(ids)
    field.snapshot()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot, pairs = 0.0, 0
    for _ in range(steps):
        field.restore()
        torch.cuda.synchronize()
        ev0.record(stream)
        field.optimize_step(ids)
        ev1.record(stream)
        torch.cuda.synchronize()
        tot += ev0.elapsed_time(ev1)
        pairs += field.stats()["last_pairs"]
    tiling = field.stats()["last_tiling"]
    # per-kernel times from the same steps run again with an event around every kernel
    field.set_timing(True)
    for _ in range(steps):
        field.restore()
        field.optimize_step(ids)
    torch.cuda.synchronize()
    kms, ksteps = field.kernel_times()
    field.close()
    return {"workload": "batched: 500k Gaussians, 9 views at mixed sizes, one graph", "steps": steps,
            "ms_per_step": tot / steps, "pairs_per_step": pairs // steps, "pairs_per_s": pairs / (tot * 1e-3),
            "kernel_ms_per_step": {nm: round(x / max(1, ksteps), 4) for nm, x in zip(KERNELS, kms)},
            "sizes": [(c["width"], c["height"]) for c in cams],
            "tiling": f"{tiling[0]}x{tiling[1]}/{tiling[2]}",
            "autotune_ms": {f"{c[0]}x{c[1]}/{c[2]}": round(t, 4) for c, t in tune["candidates"]}}


def run_batched(args):
    print(json.dumps(batched_step(args.steps, args.warmup)))


def run_stream_long(args):
    print(json.dumps(segment_stream(args)))


def serve(args):
    """Multi-session serving: 4 scenes at 1920x1080 / 1280x720 arriving at 1-3 Hz (seeded Poisson),
    each growing by up to args.serve_points new Gaussians per arrival; sessions are admitted and
    deferred by the HBM budget."""
    import torch
    import paper_2503_13086_gb300 as gs  # noqa: F401
    from paper_2503_13086_gb300.serving import Scene, Server, summarize
    torch.cuda.set_device(0)
    scenes = []
    for s in range(4):
        Wv, Hv = (1920, 1080) if s % 2 == 0 else (1280, 720)
        cams, targets, pts = stream_inputs(args.serve_arrivals, seed=10 + s, n_gt=args.serve_gt, Wv=Wv, Hv=Hv,
                                           pts_range=(args.serve_points // 2, args.serve_points + 1))
        rng = np.random.default_rng(s)
        t, reqs = 0.0, []
        for c, tg, (xyz, rgb, tr) in zip(cams, targets, pts):
            reqs.append((t, dict(cam=c, target=tg, pts_xyz=xyz, pts_rgb=rgb, tracks=tr)))
            t += rng.exponential(1.0 / rng.uniform(1.0, 3.0))
        scenes.append(Scene(s, reqs, dict(T_I=200, N_m=9, batch_views=args.serve_batch, batch_scaling=1,
                                          use_graph=1, scene_extent=7.0, seed=s,
                                          add_dist_thresh=args.serve_thresh)))
    torch.cuda.synchronize()
    srv = Server(hbm_budget_bytes=int(args.serve_budget_gb * (1 << 30)),
                 session_budget_bytes=int(args.serve_session_gb * (1 << 30)), max_active=4)
    out = srv.run(scenes)
    summ = summarize(out, srv.wall_s, srv.log)
    summ.update(peak_device_bytes=srv.peak_device_bytes, wall_s=srv.wall_s,
                deferred=sum(1 for _, e, _ in srv.log if e == "defer"),
                throttled=sum(1 for _, e, _ in srv.log if e == "throttle"),
                admission="by measured bytes in use + 2 x the largest growth per request (estimate before the first)",
                n_gaussians={sid: r["stats"]["n_gaussians"] for sid, r in out.items()},
                bytes_in_use={sid: r["stats"]["bytes_in_use"] for sid, r in out.items()},
                config={"arrivals_per_scene": args.serve_arrivals, "points_per_arrival": [args.serve_points // 2,
                                                                                     args.serve_points],
                        "gt_gaussians": args.serve_gt, "batch_views": args.serve_batch, "batch_scaling": 1,
                        "new_point_threshold": args.serve_thresh,
                        "hbm_budget_gb": args.serve_budget_gb, "session_estimate_gb": args.serve_session_gb})
    return {"workload": "serving: 4 scenes, 1920x1080 and 1280x720, 1-3 Hz arrivals", **summ}


def run_serve(args):
    print(json.dumps(serve(args)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1, help="GPUs (one rank each under torchrun; independent sessions)")
    ap.add_argument("--steps", type=int, default=200, help="timed steps")
    ap.add_argument("--warmup", type=int, default=10, help="untimed warm-up steps (at least 3)")
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"],
                    help="gs: the CUDA library; reference: the CPU oracle on the same workload")
    ap.add_argument("--workload", default="scene", choices=["scene", "batched", "serve", "stream"],
                    help="scene: the headline step (+ streaming latency); batched: 9 views per step; "
                         "serve: sessions under an HBM budget; stream: a full-length arrival stream")
    ap.add_argument("--arrivals", type=int, default=150, help="arriving images of the streaming run")
    ap.add_argument("--serve-arrivals", type=int, default=28, help="arriving images per scene of the serving run")
    ap.add_argument("--segments", default="stream,load,batched,serve",
                    help="scene workload: the measurements after the headline (comma list of stream, load, batched, "
                         "serve; 'none' for the headline alone)")
    ap.add_argument("--load-arrivals", type=int, default=30,
                    help="load: arrivals of the load-balancing comparison (the stream's first ones)")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0,
                    help="serve: the HBM the sessions may hold together (below 4 sessions' peak, so deferral and "
                         "throttling are exercised)")
    ap.add_argument("--serve-session-gb", type=float, default=16.0,
                    help="serve: a new session's estimate, used for admission until it has measured its own use")
    ap.add_argument("--serve-points", type=int, default=150_000, help="serve: most sparse points per arrival (at least half as many)")
    ap.add_argument("--serve-gt", type=int, default=4_000_000, help="serve: Gaussians of each hidden scene")
    ap.add_argument("--serve-batch", type=int, default=3, help="serve: views per optimisation step")
    ap.add_argument("--serve-thresh", type=float, default=0.005, help="serve: new-point distance threshold")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timings")
    ap.add_argument("--no-autotune-report", action="store_true",
                    help="skip the timed run of the autotuned session (profiling runs)")
    ap.add_argument("--tiling", default="16x16x256",
                    help="scene workload headline tiling: WxHxB (tile width, height, blend batch) or auto")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "stream":
        run_stream_long(args)
    else:
        run_gs(args)


if __name__ == "__main__":
    main()
