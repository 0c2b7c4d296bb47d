#!/usr/bin/env python
"""Benchmark of the VoGE renderer hot path on GB300.

One step = one analysis-by-synthesis fitting iteration over 8 views of
512x512 with N = 50,000 anisotropic Gaussians, K = 20, eta = 0.01, RGB:
  voge_render_fwd (project, bin, coarse K-nearest selection, fine
  transmittance/weights/blend) -> voge_mse_grad against the target images ->
  voge_render_bwd (adjoint, gradients of means, inverse covariances, colours
  and the 8 camera poses) -> voge_adam_step on all Gaussian parameters.
Every kernel in the step is this library's.  Metric: Mpix/s (pixels of all
views rendered forward + backward per second, all ranks).

Prints one JSON line.  Beyond the contract's keys it carries: Gaussian-ray
evaluations per second (coarse-pass traces counted on the device), the
forward and forward + backward of every workload shape (64^2 dense frame,
256^2 feature scene, the 8-view step's scene, 1024^2 / 500k scene) fused and
split, with pair rates against the measured pair ceilings; the serving load
sweep; the sampler, pose-fitting and converter rows.  --impl reference times
the FP64 CPU oracle on a bounded pixel sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s fwd+bwd (50k Gaussians, 512², K=20) vs plain; serving p50/p99 ms"
UNIT = "Mpix/s"
WORKLOAD = dict(views=8, side=512, N=50_000, K=20, eta=0.01, C=3, tau=1.0)


def workload_config(world=1):
    """The `config` of both arms: the workload, not the sample an arm times."""
    return {"workload": "fit_8x512: 8 views 512x512, N=50,000 anisotropic Gaussians, K=20, eta=0.01, RGB; "
                        "step = forward + MSE + backward + Adam",
            **WORKLOAD, "pixels_per_step": WORKLOAD["views"] * WORKLOAD["side"] ** 2,
            "parallelism": f"replicas x{world}",
            "l2": "each step writes 0.34 GB of weights/index lists (> 126 MB L2)"}
# Algorithmic FP32 work of the fine pass (Eq. 7-8) per (k, j) pair of a pixel's
# kept list, counting an FMA as 2 FLOP:
#   forward  24 = depth difference of two-float l (3) + scale (1) + A&S 7.1.28
#             erf: degree-6 polynomial (12) + 4 squarings (4) + reciprocal (1)
#             + signed accumulation (3)
#   backward 28 = adjoint pair: difference and scale (4), A&S 7.1.26 erf with
#             e^{-u^2} (15), accumulation of dm, du, dl_k, dl_j, dr (9); the
#             timed step hands the forward's weights to the backward
#             (voge_render_bwd_w), so the forward pair is not recomputed
#             (it would add 24)
# plus, per kept entry, 80 FLOP for the chain to camera space (backward only)
# and, in the forward, 30 FLOP for each Gaussian-ray trace of Eq. 6 (offsets
# 4, b and its numerator 11, qb 5, the threshold test 1, l 5, sigma and e^{q}
# 4): every coarse-pass trace (counted on the device, voge_render_stats) and
# the fine pass's set-up trace of each kept entry.
FLOP_PER_PAIR = {"fwd": 24, "bwd": 28}
FLOP_PER_ENTRY_BWD = 80
FLOP_PER_TRACE = 30
# GB300: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2070 MHz max SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="voge", choices=["voge", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=4.0, help="measured seconds of each serving run")
    ap.add_argument("--no-configs", action="store_true", help="skip the forward / fwd+bwd rows of the other workloads")
    ap.add_argument("--split-forward", action="store_true",
                    help="the step's forward as two kernels (selection, then the fine pass): for profiling the fine pass")
    ap.add_argument("--no-sampler", action="store_true")
    ap.add_argument("--no-posefit", action="store_true")
    ap.add_argument("--no-converters", action="store_true")
    ap.add_argument("--no-alu-ceilings", action="store_true", help="skip the measured ALU ceilings")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples; VOGE_CLOCKS_DIR keeps them somewhere lasting
        d = os.environ.get("VOGE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"voge_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle ---
def oracle_sample(sc, cams, n_pix, rng, nthreads):
    """Oracle forward (brute force over all N) + analytic backward on n_pix sampled pixels."""
    import oracle

    allp = oracle.all_pixels(cams)
    pix = np.ascontiguousarray(allp[np.sort(rng.choice(allp.shape[0], n_pix, replace=False))])
    m, p, a = (sc[k].astype(np.float64) for k in ("means", "inv_cov", "attr"))
    t0 = time.perf_counter()
    fwd = oracle.render(cams, m, p, a, K=WORKLOAD["K"], tau=WORKLOAD["tau"], eta=WORKLOAD["eta"], pix=pix,
                        nthreads=nthreads)
    g = rng.standard_normal(fwd["image"].shape)
    oracle.render_bwd(cams, m, p, a, WORKLOAD["tau"], pix, fwd["idx"], g, nthreads=nthreads)
    return time.perf_counter() - t0


def oracle_configs(nthreads, seed=0):
    """The oracle's forward + backward on the two smaller workloads: the whole
    64x64 dense frame (128 Gaussians, every candidate kept, no threshold) and
    8192 random pixels of the 256x256 feature scene (4000 Gaussians, C = 128)."""
    import oracle
    from paper_2205_15401_gb300 import scenes

    rng = np.random.default_rng(seed)
    out = {}
    for name, sc, n_pix in (("plain_64", scenes.plain_64(seed=0), None),
                            ("posefit_256", scenes.posefit_256(seed=0), 8192)):
        cams = scenes.cameras(sc, oracle.pose_to_RT)
        pix = oracle.all_pixels(cams)
        if n_pix is not None:
            pix = np.ascontiguousarray(pix[np.sort(rng.choice(pix.shape[0], n_pix, replace=False))])
        m, p, a = (sc[k].astype(np.float64) for k in ("means", "inv_cov", "attr"))
        t0 = time.perf_counter()
        fwd = oracle.render(cams, m, p, a, K=sc["K"], tau=sc["tau"], eta=sc["eta"], pix=pix, nthreads=nthreads)
        g = rng.standard_normal(fwd["image"].shape)
        oracle.render_bwd(cams, m, p, a, sc["tau"], pix, fwd["idx"], g, nthreads=nthreads)
        t = time.perf_counter() - t0
        out[name] = {"value": pix.shape[0] / t / 1e6, "unit": UNIT, "pixels": int(pix.shape[0]), "seconds": t}
    return out


def cpu_baseline(sc, cams, target_s, seed=0):
    nthreads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    n0 = 16 * nthreads
    t0 = oracle_sample(sc, cams, n0, rng, nthreads)
    n = int(min(200_000, max(n0, n0 * target_s / max(t0, 1e-3))))
    t = oracle_sample(sc, cams, n, rng, nthreads)
    return {"value": n / t / 1e6, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{n} random pixels of the 8x512x512 views, FP64 forward (all {WORKLOAD['N']} Gaussians "
                      f"tested per pixel) + analytic backward, {t:.1f} s",
            "other_workloads": oracle_configs(nthreads, seed)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2205_15401_gb300 import scenes

    oracle.build()
    sc = scenes.fit_8x512(seed=args.seed)
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    nthreads = os.cpu_count() or 1
    rng = np.random.default_rng(args.seed)
    # size each step so that warmup + steps take about two minutes
    n0 = 8 * nthreads
    t0 = oracle_sample(sc, cams, n0, rng, nthreads)
    total = max(1, args.steps + args.warmup)
    n = int(max(n0, min(100_000, n0 * (120.0 / total) / max(t0, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample(sc, cams, n, rng, nthreads)
    t = 0.0
    for _ in range(args.steps):
        t += oracle_sample(sc, cams, n, rng, nthreads)
    value = n * args.steps / t / 1e6
    sample = f"{n} random pixels per step of the 8x512x512 views, FP64 forward + analytic backward"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": workload_config(1),
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- serving ---
def sampler_bench(voge, index, weights, N, dev, reps=10):
    """voge_sample on the step's own lists and weights with synthetic features
    of 3 (texture) and 128 (deep features) channels: device time per call and
    the algorithmic bytes (lists, weights and features read once, the
    per-kernel rows written and normalised) against the measured HBM peak."""
    import torch

    P, L = index.shape
    peak = measured_hbm_gbs()
    out = {"workload": f"lists and weights of the fit_8x512 forward ({P} pixels, L={L}, N={N}); features N(0,1)"}
    for C in (3, 128):
        g = torch.Generator(device=dev).manual_seed(C)
        phi = torch.randn((P, C), device=dev, generator=g)
        alpha = torch.empty((N, C), device=dev)
        wsum = torch.empty((N,), device=dev)
        for _ in range(3):
            voge.voge_sample(index, weights, phi, N, alpha, wsum)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            voge.voge_sample(index, weights, phi, N, alpha, wsum)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = P * L * 8 + P * C * 4 + N * (C + 1) * 4 * 3
        gbs = nbytes / (ms / 1e3) / 1e9
        out[f"C{C}"] = {"ms": ms, "mpix_s": P / (ms / 1e3) / 1e6, "algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                        "hbm_peak_gbs": peak, "frac": gbs / peak if peak else None}
    return out


def posefit_bench(voge, dev, steps=20, warmup=3):
    """Feature-level pose fitting at the scale of Sec. 4.1's render-and-compare
    loop: 144 start poses (12 azimuths x 4 elevations x 3 rolls) of the
    posefit_256 object (N = 4000, 128-channel features, 256 x 256) fitted as
    one batch; device time per fitting step of all starts."""
    import torch

    from paper_2205_15401_gb300 import scenes
    from paper_2205_15401_gb300.posefit import PoseFitter

    sc = scenes.posefit_256(seed=0)
    side, C = 256, sc["attr"].shape[1]
    true = sc["poses"][0]
    m, p, a = (torch.tensor(sc[k], device=dev) for k in ("means", "inv_cov", "attr"))
    R, T = voge.voge_pose_to_RT(true)
    cam = {"R": R, "T": T, "F": float(side), "Ox": side / 2, "Oy": side / 2, "H": side, "W": side}
    target = voge.Renderer([cam], m.shape[0], C, K=20, tau=1.0, thresh=1e-3, device=dev).forward(m, p, a)[0].clone()
    starts = np.array([[az, el, true[2], ro] for az in np.linspace(-np.pi, np.pi, 12, endpoint=False)
                       for el in (-0.2, 0.1, 0.4, 0.7) for ro in (-0.1, 0.0, 0.1)])
    fitter = PoseFitter(m, p, a, target, side, side, float(side), starts, lr=0.02, device=dev)
    for _ in range(warmup):
        fitter.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(steps):
        fitter.step()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1) / steps
    return {"workload": "posefit_256: N=4000, C=128 features, 256x256, K=20; 144 start poses fitted as one batch "
                        "(forward + MSE + backward to the cameras + pose chain + Adam per step)",
            "starts": len(starts), "ms_per_step": ms, "start_steps_per_s": len(starts) / (ms / 1e3),
            "mpix_s": len(starts) * side * side / (ms / 1e3) / 1e6, "wall_ms_per_step": 1e3 * wall / steps}


def converters_bench(voge, dev, reps=5):
    """Mesh converter on a 400 x 800 UV sphere (320k vertices, 640k faces) and
    point-cloud converter on 50k points with m = 8 (App. A.4): device ms per call."""
    import torch

    from paper_2205_15401_gb300 import scenes

    V, F = scenes.uv_sphere(400, 800, 1.0, seed=0, jitter=0.01)
    Vd, Fd = torch.tensor(V, device=dev), torch.tensor(F, device=dev)
    X = torch.tensor(np.random.default_rng(0).uniform(-1, 1, (50_000, 3)).astype(np.float32), device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    return {"mesh": {"vertices": int(V.shape[0]), "faces": int(F.shape[0]), "flatten": 0.3,
                     "ms": timed(lambda: voge.voge_mesh_to_gaussians(Vd, Fd, 0.5, 0.3))},
            "points": {"points": int(X.shape[0]), "m": 8, "ms": timed(lambda: voge.voge_points_to_gaussians(X, 8, 0.5))}}


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def serving_bench(dev, seconds, batching, graphs, mean_gap_s=0.002, seed=0, warmup_s=0.5, max_queue=0):
    """Poisson render-and-compare requests against resident scenes.

    Scene pool: for each attribute width C in {3, 16, 128}, four scenes with N
    drawn from U[1k, 100k] (the 8-view generator's distribution).  Each request
    picks side in {128, 256, 512}, K in {10, 20, 32}, a scene of its C and a
    random camera on the view sphere; it returns the loss and the gradients of
    the means and the camera into pinned host memory.  batching: continuous
    batching (else one request per tick); graphs: ticks replayed as CUDA
    graphs.  max_queue > 0 bounds the pending queue: past saturation the
    server turns requests away (counted as rejected) instead of building an
    unbounded backlog."""
    import threading

    import torch

    from paper_2205_15401_gb300 import scenes
    from paper_2205_15401_gb300 import voge

    rng = np.random.default_rng(seed)
    srv = voge.Server(mem_budget_bytes=48 << 30, max_slots=256, use_graphs=graphs, batching=batching,
                      inflight_ticks=2 if batching else 1, max_queue=max_queue)
    pool = {}
    for C in (3, 16, 128):
        pool[C] = []
        for q in range(4):
            N = int(rng.integers(1000, 100_001))
            sc = scenes.fit_8x512(seed=1000 + 10 * C + q, N=N, B=1, side=16, C=C)
            pool[C].append((srv.add_scene(sc["means"], sc["inv_cov"], sc["attr"]), N))
    targets = {(side, C): torch.rand((side * side, C)).pin_memory() for side in (128, 256, 512) for C in (3, 16, 128)}
    out_pool = [{"grad_means": torch.empty((100_001, 3)).pin_memory(), "grad_cam": torch.empty(12).pin_memory(),
                 "loss": torch.empty(1).pin_memory()} for _ in range(512)]
    stream = scenes.serving_stream(seed=seed, duration_s=warmup_s + seconds, mean_gap_s=mean_gap_s)
    done, lock = [], threading.Lock()
    tickets = []
    cv = threading.Condition()
    refused = [0]

    def consumer():
        k = 0
        while True:
            with cv:
                while k >= len(tickets):
                    cv.wait()
                item = tickets[k]
            if item is None:
                return
            t, px, arrive = item
            rc, tm = srv.wait(t, -1)
            with lock:
                done.append((arrive, tm, px, rc))
            k += 1

    th = threading.Thread(target=consumer)
    th.start()
    t0 = time.perf_counter()
    for q, req in enumerate(stream):
        delay = req["t"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        sid, N = pool[req["C"]][int(rng.integers(0, 4))]
        side = req["side"]
        pose = [rng.uniform(-np.pi, np.pi), rng.uniform(-1.0, 1.0), 4.0, 0.0]
        R, T = voge.voge_pose_to_RT(pose)
        cam = {"R": R, "T": T, "F": float(side), "Ox": side / 2, "Oy": side / 2, "H": side, "W": side}
        rc, t = srv.submit(cam, targets[(side, req["C"])], req["K"], thresh=0.01, scene=sid,
                           outputs=out_pool[q % len(out_pool)])
        if rc == 0:
            with cv:
                tickets.append((t, side * side, req["t"]))
                cv.notify()
        elif req["t"] >= warmup_s:
            refused[0] += 1
    with cv:
        tickets.append(None)
        cv.notify()
    th.join()
    stats = srv.stats()
    srv.close()
    meas = [(tm, px) for arrive, tm, px, rc in done if rc == 0 and arrive >= warmup_s]
    offered = sum(1 for req in stream if req["t"] >= warmup_s)
    if not meas:
        return {"requests": 0, "offered": offered, "rejected": refused[0]}
    lat = np.array([tm["done_us"] - tm["submit_us"] for tm, _ in meas]) / 1e3
    t_first = min(tm["submit_us"] for tm, _ in meas)
    t_last = max(tm["done_us"] for tm, _ in meas)
    span = (t_last - t_first) / 1e6
    return {"requests": len(meas), "offered": offered, "rejected": refused[0],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "mpix_s": sum(px for _, px in meas) / span / 1e6,
            "requests_per_s": len(meas) / span, "ticks": stats["ticks"],
            "requests_per_tick": stats["requests_in_ticks"] / max(stats["ticks"], 1),
            "graphs": stats["graphs_captured"]}


def serving_suite(dev, seconds, seed=0):
    """The serving workload (mean gap 2 ms) and a load sweep to past
    saturation, each load with three arms: continuous batching with CUDA-graph
    ticks; one request per tick with graph ticks (separates graph replay from
    batching); one request per tick with plain launches (the per-request
    comparator).  Past saturation the pending queue is bounded (256), so the
    arms deliver what they can and turn the rest away."""
    arms = (("batched", True, True), ("per_request_graphs", False, True), ("per_request_plain", False, False))
    out = {"workload": "Poisson arrivals, 0.5 s warm-up then measured; N U[1k,100k] (resident scenes), side "
                       "{128,256,512}, C {3,16,128}, K {10,20,32}; latency = submit to outputs in host memory",
           "measured_s": seconds}
    for gap_ms in (2.0, 1.0, 0.5, 0.25):
        row = {}
        for name, batching, graphs in arms:
            row[name] = serving_bench(dev, seconds, batching, graphs, mean_gap_s=gap_ms / 1e3, seed=seed,
                                      max_queue=256)
        out[f"gap_{gap_ms:g}ms"] = row
    # the configured workload's line: mean gap 2 ms
    out["batched"] = out["gap_2ms"]["batched"]
    out["plain"] = out["gap_2ms"]["per_request_plain"]
    return out


def _traced(voge, fn, reps):
    """Run fn reps times with the library's kernel tracing on: (CUDA-event ms
    per call, {kernel: ms per call})."""
    import torch

    voge.voge_trace_reset()
    voge.voge_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    voge.voge_trace_enable(False)
    tr = voge.voge_trace_read()
    return e0.elapsed_time(e1) / reps, {k: t / reps for k, (n, t) in tr.items() if n > 0}


def _sum_ms(kms, prefixes):
    return sum(t for k, t in kms.items() if k.startswith(prefixes))


def workload_rows(voge, dev, alu, reps=20):
    """Forward and forward + backward of every workload shape, each timed
    alone: Mpix/s, Gaussian-ray evaluations per second, and each tile
    kernel's pair rate against the measured pair ceilings and its FLOP rate
    against the measured FMA rate.  The forward is also timed split (the
    selection kernel, then the fine kernel over its lists: the fine pass
    measured on its own, Eq. 7-8).  The backward takes the forward's weights
    and a fixed N(0,1) image gradient.  Gaussian-ray evaluations: the coarse
    pass's traces (counted on the device) plus one set-up trace per kept entry
    in the forward, two per kept entry in the backward (set-up and chain)."""
    import torch

    from paper_2205_15401_gb300 import scenes

    fma = alu["fma_tflops"] if alu else None
    out = {}
    for name, sc in (("plain_64", scenes.plain_64(seed=0)), ("posefit_256", scenes.posefit_256(seed=0)),
                     ("fit_8x512", scenes.fit_8x512(seed=0)), ("large_1024", scenes.large_1024(seed=0))):
        cams = scenes.cameras(sc, voge.voge_pose_to_RT)
        N, C = sc["means"].shape[0], sc["attr"].shape[1]
        m, p, a = (torch.tensor(sc[k], device=dev) for k in ("means", "inv_cov", "attr"))
        row = {"N": N, "C": C, "K": sc["K"], "eta": sc["eta"], "views": len(cams),
               "side": int(cams[0]["H"])}
        for form, flags in (("fused", 0), ("split", voge.VOGE_FLAG_SPLIT_FORWARD)):
            r = voge.Renderer(cams, N, C, K=sc["K"], tau=sc["tau"], thresh=sc["eta"], flags=flags, device=dev)
            img, w, idx = r.alloc_outputs()
            g_img = torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
            gm, gp, ga = torch.zeros_like(m), torch.zeros_like(p), torch.zeros_like(a)
            gc = torch.zeros((len(cams), 12), device=dev)

            def fwd():
                r.forward(m, p, a, out=(img, w, idx))

            def fwd_bwd():
                r.forward(m, p, a, out=(img, w, idx))
                r.backward(m, p, a, idx, g_img, gm, gp, ga, gc, weights=w)

            for _ in range(3):
                fwd_bwd()
            fwd()
            st = voge.voge_render_stats(r.workspace)
            ms_f, k_f = _traced(voge, fwd, reps)
            ms_fb, k_fb = _traced(voge, fwd_bwd, reps)
            P, T, E, pairs = r.pixels, st["traces"], st["entries"], st["pairs"]
            f = {"ms_fwd": ms_f, "ms_fwd_bwd": ms_fb, "mpix_s_fwd": P / ms_f / 1e3,
                 "mpix_s_fwd_bwd": P / ms_fb / 1e3, "kernels_fwd": k_f,
                 "gaussian_ray_evals_per_s": {"fwd": (T + E) / (ms_f / 1e3), "fwd_bwd": (T + 3 * E) / (ms_fb / 1e3)}}
            if form == "fused":
                row.update({"pixels": P, "coarse_traces": T, "entries": E, "pairs": pairs})
            ms_pairs_f = _sum_ms(k_f, ("k_render", "k_fine"))
            if ms_pairs_f > 0:
                f["fwd_pair_kernel_gpairs"] = pairs / ms_pairs_f / 1e6
                if alu:
                    f["fwd_pair_frac"] = f["fwd_pair_kernel_gpairs"] / alu["fwd_gpairs"]
            if form == "fused" and fma:
                ms_r = _sum_ms(k_f, ("k_render",))
                if ms_r > 0:
                    tf = (pairs * FLOP_PER_PAIR["fwd"] + (T + E) * FLOP_PER_TRACE) / ms_r / 1e9
                    f["render_tflops"] = tf
                    f["render_frac_of_measured_fma"] = tf / fma
            if form == "split":
                ms_fine = _sum_ms(k_f, ("k_fine",))
                ms_sel = _sum_ms(k_f, ("k_select",))
                f["select_ms"], f["fine_ms"] = ms_sel, ms_fine
                if ms_fine > 0:
                    f["fine_gpairs"] = pairs / ms_fine / 1e6
                    f["fine_tflops"] = (pairs * FLOP_PER_PAIR["fwd"] + E * FLOP_PER_TRACE) / ms_fine / 1e9
                    if alu:
                        f["fine_frac_of_pair_ceiling"] = f["fine_gpairs"] / alu["fwd_gpairs"]
                    if fma:
                        f["fine_frac_of_measured_fma"] = f["fine_tflops"] / fma
            ms_b = _sum_ms(k_fb, ("k_backward",))
            if form == "fused" and ms_b > 0:
                f["bwd_kernel_ms"] = ms_b
                f["bwd_gpairs"] = pairs / ms_b / 1e6
                tf = (pairs * FLOP_PER_PAIR["bwd"] + E * FLOP_PER_ENTRY_BWD) / ms_b / 1e9
                f["bwd_tflops"] = tf
                if alu:
                    f["bwd_pair_frac"] = f["bwd_gpairs"] / alu["bwd_gpairs"]
                if fma:
                    f["bwd_frac_of_measured_fma"] = tf / fma
            row[form] = f
            del r, img, w, idx, g_img
        out[name] = row
        torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------- GPU path ---
def reduce_over_ranks(ms, pixels, world, device):
    """Whole-job timing: the slowest rank's time and the pixels of all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(pixels)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


# The sources that define the step's kernels and their launches: the committed
# DRAM traffic stays valid while these are unchanged.
KERNEL_SOURCES = ("voge_api.cu", "voge_backward.cu", "voge_device.cuh", "voge_forward.cu", "voge_project.cu",
                  "voge_trace.cu", "voge_trace.cuh")


# The kernels of the forward pass (projection, binning, tile sort, render) and
# of the backward pass (adjoint, gradient finalisation, pose chain) by name.
FWD_KERNELS = ("k_project", "k_tile_totals", "k_scan_tiles", "k_scatter", "k_sort_tiles", "k_render", "k_select",
               "k_fine")
BWD_KERNELS = ("k_backward", "k_grad_finalize", "k_pose_grad")


def pass_throughput(trace, pixels_per_step, steps):
    """Mpix/s of the forward and of the backward pass alone, from the traced
    device time of their kernels per step (the step also runs MSE and Adam)."""
    out = {}
    for name, prefixes in (("fwd", FWD_KERNELS), ("bwd", BWD_KERNELS)):
        ms = sum(t for k, (n, t) in trace.items() if k.startswith(prefixes)) / max(steps, 1)
        if ms > 0:
            out[name] = {"mpix_s": pixels_per_step / (ms / 1e3) / 1e6, "ms_per_step": ms}
    return out or None


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2205_15401_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, src_hash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this exact source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == src_hash:
            try:
                return float(parts[2])
            except ValueError:
                return None
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2205_15401_gb300 import build as vbuild
    from paper_2205_15401_gb300 import scenes
    from paper_2205_15401_gb300 import voge

    vbuild.build()
    voge.lib()

    W = WORKLOAD
    sc = scenes.fit_8x512(seed=args.seed + rank, N=W["N"], B=W["views"], side=W["side"], C=W["C"], K=W["K"])
    cams = scenes.cameras(sc, voge.voge_pose_to_RT)
    N, C = W["N"], W["C"]
    r = voge.Renderer(cams, N, C, K=W["K"], tau=W["tau"], thresh=W["eta"],
                      flags=voge.VOGE_FLAG_SPLIT_FORWARD if args.split_forward else 0, device=dev)
    P = r.pixels

    # flat parameter / gradient / Adam buffers: [means 3N | inv_cov 6N | attr CN]
    n_par = N * (3 + 6 + C)
    host_par = np.concatenate([sc["means"].reshape(-1), sc["inv_cov"].reshape(-1), sc["attr"].reshape(-1)])
    par = torch.tensor(host_par, device=dev)
    grad = torch.zeros(n_par, device=dev)
    m_adam, v_adam = torch.zeros(n_par, device=dev), torch.zeros(n_par, device=dev)

    def views(buf):
        return buf[: 3 * N].view(N, 3), buf[3 * N: 9 * N].view(N, 6), buf[9 * N:].view(N, C)

    means, inv_cov, attr = views(par)
    g_means, g_inv_cov, g_attr = views(grad)
    g_cam = torch.zeros((W["views"], 12), device=dev)
    loss = torch.zeros(1, device=dev)
    image, weights, index = r.alloc_outputs()
    g_image = torch.empty_like(image)

    # target: render of the perturbed parameters (outside the timed region)
    tm = torch.tensor(sc["target_means"], device=dev)
    ta = torch.tensor(sc["target_attr"], device=dev)
    target = r.forward(tm, inv_cov.clone(), ta)[0].clone()

    step_no = [0]

    def step():
        r.forward(means, inv_cov, attr, out=(image, weights, index))
        loss.zero_()
        voge.voge_mse_grad(image, target, g_image, loss)
        r.backward(means, inv_cov, attr, index, g_image, g_means, g_inv_cov, g_attr, g_cam, reuse_projection=True,
                   weights=weights)
        step_no[0] += 1
        voge.voge_adam_step(par, grad, m_adam, v_adam, lr=1e-4, step=step_no[0])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    voge.voge_trace_reset()
    voge.voge_trace_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    voge.voge_trace_enable(False)
    trace = voge.voge_trace_read()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max, pix_all = reduce_over_ranks(ms, P * args.steps, world, dev)
    value = pix_all / (ms_max / 1e3) / 1e6
    launches = sum(n for n, _ in trace.values())
    passes = pass_throughput(trace, P, args.steps)

    # ------------------------------------------------ measured ALU ceilings
    # Register-only loops of the FMA, ex2 and both pair terms on this GPU: the
    # measured peak of the roofline, and the speed-of-light of the pair loops.
    alu = None if args.no_alu_ceilings else voge.voge_measure_alu_peaks()
    torch.cuda.synchronize()

    # ------------------------------------------------ what one step's forward did
    r.forward(means, inv_cov, attr, out=(image, weights, index))
    st = voge.voge_render_stats(r.workspace)
    pairs, entries, traces = float(st["pairs"]), float(st["entries"]), float(st["traces"])
    step_s = ms_max / args.steps / 1e3
    ray_evals = {"coarse_traces_per_step": traces, "entries_per_step": entries, "pairs_per_step": pairs,
                 "fwd_bwd_per_s": (traces + 3 * entries) / step_s,
                 "what": "Gaussian-ray evaluations (Eq. 6): the coarse pass's traces (counted on the device) + one "
                         "set-up trace per kept entry (forward) + two per kept entry (backward set-up and chain)"}
    if passes and "fwd" in passes:
        ray_evals["fwd_per_s"] = (traces + entries) / (passes["fwd"]["ms_per_step"] / 1e3)

    # ------------------------------------------------ roofline of the top kernel
    top = max(trace.items(), key=lambda kv: kv[1][1]) if trace else (None, (0, 0.0))
    top_name, (top_n, top_ms) = top
    roofline = None
    if top_name and top_n > 0:
        avg_s = top_ms / top_n / 1e3
        if top_name.startswith("k_backward"):
            flop = pairs * FLOP_PER_PAIR["bwd"] + entries * FLOP_PER_ENTRY_BWD
        elif top_name.startswith("k_render"):
            flop = pairs * FLOP_PER_PAIR["fwd"] + (traces + entries) * FLOP_PER_TRACE
        else:
            flop = None
        if flop is not None:
            ach = flop / avg_s / 1e12
            measured = alu is not None and alu["fma_tflops"] > 0
            peak = alu["fma_tflops"] if measured else FP32_PEAK_TFLOPS
            roofline = {"bound": "alu", "kernel": top_name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "traffic": profiled_traffic(top_name, kernel_source_hash()),
                        "peak_source": "measured: FP32 FMA register loop on every SM, this run (of measured)"
                        if measured else "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz",
                        "peak_derived": FP32_PEAK_TFLOPS, "avg_launch_ms": top_ms / top_n,
                        "flop_per_launch": flop, "pairs_per_launch": pairs}
    kernels = {k: {"launches": n, "ms_per_launch": t / max(n, 1), "share": t / max(sum(x for _, x in trace.values()),
                                                                                  1e-30)}
               for k, (n, t) in trace.items()}
    pair_frac = {}
    for side, prefix, key in (("fwd", "k_render", "fwd_gpairs"), ("bwd", "k_backward", "bwd_gpairs")):
        ent = [(k, n, t) for k, (n, t) in trace.items() if k.startswith(prefix) and n > 0]
        if alu and ent and alu[key] > 0:
            k, n, t = max(ent, key=lambda e: e[2])
            got = pairs / (t / n / 1e3) / 1e9
            pair_frac[side] = {"kernel": k, "achieved_gpairs": got, "ceiling_gpairs": alu[key], "frac": got / alu[key]}
    alu_ceilings = None if alu is None else {
        "fma_tflops": alu["fma_tflops"], "ex2_tops": alu["ex2_tops"], "fwd_gpairs": alu["fwd_gpairs"],
        "bwd_gpairs": alu["bwd_gpairs"], "pairs": pair_frac,
        "how": "voge_measure_alu_peaks: register-only loops on every SM, CUDA events"}

    # ------------------------------------------------ e2e through host buffers
    # The same step as the timed one (forward, MSE, backward, Adam) through the
    # public API, with the parameters and targets copied in from pinned host
    # memory and the loss and updated parameters copied back, every step, as
    # a pipelined training loop runs it: the inputs of step i + 1 are copied
    # on a second stream, into the other of two buffer sets, while step i
    # runs (a data loader's prefetch), and the host reads step i's loss while
    # step i + 1 runs.  The timed region ends when the last step's results
    # are in host memory.
    e2e = None
    if not args.no_e2e:
        h_par = torch.tensor(host_par).pin_memory()
        h_target = target.cpu().pin_memory()
        h_outs = [torch.empty(n_par).pin_memory(), torch.empty(n_par).pin_memory()]
        h_losses = [torch.empty(1).pin_memory(), torch.empty(1).pin_memory()]
        pars = [torch.empty_like(par), torch.empty_like(par)]
        targets = [torch.empty_like(target), torch.empty_like(target)]
        cstream = torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_out = [torch.cuda.Event(), torch.cuda.Event()]
        main = torch.cuda.current_stream()
        # device time of the copies themselves (events on their own streams)
        copy_ev = {"in": [], "out": []}

        def make_step(pb, tb):
            mb, pvb, ab = views(pb)

            def st():
                r.forward(mb, pvb, ab, out=(image, weights, index))
                loss.zero_()
                voge.voge_mse_grad(image, tb, g_image, loss)
                r.backward(mb, pvb, ab, index, g_image, g_means, g_inv_cov, g_attr, g_cam, reuse_projection=True,
                           weights=weights)
                step_no[0] += 1
                voge.voge_adam_step(pb, grad, m_adam, v_adam, lr=1e-4, step=step_no[0])
            return st

        steps_e2e = [make_step(pars[0], targets[0]), make_step(pars[1], targets[1])]

        def copy_in(b, after_out):
            # buffer set b was last used by the step two back: its results
            # must be out first
            with torch.cuda.stream(cstream):
                if after_out:
                    cstream.wait_event(ev_out[b])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(cstream)
                pars[b].copy_(h_par, non_blocking=True)
                targets[b].copy_(h_target, non_blocking=True)
                e1.record(cstream)
                copy_ev["in"].append((e0, e1))
                ev_in[b].record(cstream)

        def e2e_run(k):
            copy_in(0, False)
            losses = []
            for i in range(k):
                b = i & 1
                if i + 1 < k:
                    copy_in(b ^ 1, i >= 1)
                main.wait_event(ev_in[b])
                steps_e2e[b]()
                o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                o0.record(main)
                h_outs[b].copy_(pars[b], non_blocking=True)
                h_losses[b].copy_(loss, non_blocking=True)
                o1.record(main)
                copy_ev["out"].append((o0, o1))
                ev_out[b].record(main)
                if i >= 1:  # the previous step's loss, read while this one runs
                    ev_out[b ^ 1].synchronize()
                    losses.append(float(h_losses[b ^ 1][0]))
            ev_out[(k - 1) & 1].synchronize()
            losses.append(float(h_losses[(k - 1) & 1][0]))
            return losses

        e2e_run(args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        copy_ev["in"].clear()
        copy_ev["out"].clear()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        t_e2e, _ = reduce_over_ranks(time.perf_counter() - t0, 0, world, dev)
        torch.cuda.synchronize()
        h2d_ms = sum(a.elapsed_time(b) for a, b in copy_ev["in"]) / max(len(copy_ev["in"]), 1)
        d2h_ms = sum(a.elapsed_time(b) for a, b in copy_ev["out"]) / max(len(copy_ev["out"]), 1)
        e2e = {"value": pix_all / t_e2e / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(4 * (n_par + target.numel())),
               "d2h_bytes_per_step": int(4 * (n_par + 1)),
               "ms_per_step": 1e3 * t_e2e / args.steps,
               "h2d_ms_per_step": h2d_ms, "d2h_ms_per_step": d2h_ms,
               "what": "forward + MSE + backward + Adam as the timed step; every step's parameters and targets "
                       "copied in from pinned host memory (the next step's on a second stream during the "
                       "current step) and its loss and updated parameters copied out, the host reading each "
                       "step's loss while the next step runs; the timed region ends with the last step's "
                       "results in host memory"}

    # ------------------------------------------------ plain comparator
    plain = None
    if not args.no_plain:
        rp = voge.Renderer(cams, N, C, K=W["K"], tau=W["tau"], thresh=W["eta"], flags=voge.VOGE_FLAG_PLAIN,
                           device=dev)

        def plain_step():
            rp.forward(means, inv_cov, attr, out=(image, weights, index))
            loss.zero_()
            voge.voge_mse_grad(image, target, g_image, loss)
            rp.backward(means, inv_cov, attr, index, g_image, g_means, g_inv_cov, g_attr, g_cam,
                        reuse_projection=True, weights=weights)
            grad.zero_()

        plain_step()
        torch.cuda.synchronize()
        k_plain = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k_plain):
            plain_step()
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / k_plain
        plain = {"value": P / (pms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": pms,
                 "what": "same step, every pixel tests every Gaussian (no tile binning)"}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_suite(dev, args.serving_seconds, seed=args.seed)

    workloads = None
    if rank == 0 and not args.no_configs:
        workloads = workload_rows(voge, dev, alu)

    # ------------------------------------------------ neural sampler (Sec. 3.4 Eq. 10)
    sampler = None
    if not args.no_sampler:
        sampler = sampler_bench(voge, index[:, : r.L].contiguous(), weights[:, : r.L].contiguous(), N, dev)

    converters = None
    if not args.no_converters:
        converters = converters_bench(voge, dev)

    posefit = None
    if not args.no_posefit:
        posefit = posefit_bench(voge, dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        cpu = cpu_baseline(sc, scenes.cameras(sc, oracle.pose_to_RT), args.cpu_seconds)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": workload_config(world),
               "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "plain": plain,
               "gaussian_ray_evals": ray_evals, "workloads": workloads,
               "serving": serving, "sampler": sampler, "posefit": posefit, "converters": converters,
               "clocks": clk, "kernels": kernels, "passes": passes, "alu_ceilings": alu_ceilings, "loss": float(loss.item())}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
