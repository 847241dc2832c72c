"""Benchmark: element-point influence evaluations per second on the THGEM unit cell.

Workload (the configuration the headline metric is quoted on): hexagonal THGEM cell,
pitch 1 mm, 9,996 flat rectangles and triangles, 5 x 5 periodic images, potential and
field at 1,000,000 points uniform in the cell volume, mixed precision (FP32 far-field
Gauss rules, FP64 near-field closed forms), charge densities from a mixed solve with
FP64 refinement.  One step = one evaluation of all points (the whole hot path of the
evaluation: every element, every image, every point).  Synthetic, seeded inputs.

The timed step is the mixed evaluation as it meets 1e-6 relative error per point (FP32
pass, then a two-float re-evaluation of the points whose estimated error exceeds 1e-6 of
their own value).  Reported next to it: the single FP32 pass alone with its per-point
error, the plain FP64 path's rate (on a point sample), both mixed forms' errors against
the FP64 path (normwise and per point), the stage times, the roofline of the dominant
kernel, the end-to-end rate through the host-buffer C-ABI call, and the FP64 CPU oracle
timed on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
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

N_POINTS = 1_000_000
HEADLINE_METRIC = "element-point influence evals/s (mixed FP32/FP64, <=1e-6 rel err per point vs FP64 path)"
FP64_SAMPLE = 19_456
CHECK_SAMPLE = 512
ROOFLINE_SAMPLE = 8192
SC_CARRIERS = 1_000_000  # points whose refinement decision is taken again to count the refined pairs
ORACLE_SAMPLE = 2_048
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--fp64-points", type=int, default=FP64_SAMPLE,
                    help="sample size of the FP64-path comparison (accuracy and FP64 rate)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=40)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-space-charge", action="store_true")
    ap.add_argument("--workload", default="thgem_eval",
                    choices=["thgem_eval", "double_thgem_solve", "space_charge", "lu", "am", "fastvol"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(n_points):
    from paper_2606_24154_gb300 import inputs as I
    g = I.thgem()
    pts = I.cell_points(g, n_points, I.rng(1, 0))
    return g, pts


def oracle_rate(g, pts, n):
    """FP64 CPU oracle on a bounded sample of the same workload (evals/s, threads)."""
    from oracle import oracle as O
    sigma = I_sigma(g)
    sample = pts[:n]
    t = time.perf_counter()
    O.eval_points(g, sigma, sample)
    dt = time.perf_counter() - t
    return n * g.n * g.n_images / dt, O.num_threads(), dt


def I_sigma(g):
    """Seeded structured charge density for the CPU sample (the oracle's cost does not
    depend on its values)."""
    from paper_2606_24154_gb300 import inputs as I
    return I.rng(1, 5).normal(size=g.n) * 1e-6


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g, pts = workload(max(ORACLE_SAMPLE, 256))
    n = min(ORACLE_SAMPLE, pts.shape[0]) // 4  # per step: a quarter of the sample
    from oracle import oracle as O
    sigma = I_sigma(g)
    for w in range(args.warmup):
        O.eval_points(g, sigma, pts[:max(8, n // 8)])
    times = []
    for s in range(args.steps):
        sl = pts[(s * n) % (pts.shape[0] - n):][:n]
        t = time.perf_counter()
        O.eval_points(g, sigma, sl)
        times.append(time.perf_counter() - t)
    per = statistics.mean(times)
    val = n * g.n * g.n_images / per
    line = {
        "impl": "reference", "metric": HEADLINE_METRIC, "value": val, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"thgem_cell N={g.n} images={g.n_images} points={N_POINTS} mixed eval",
                   "elements": g.n, "images": g.n_images, "points_per_gpu": N_POINTS,
                   "reference_sample": f"{n} of the points per step, FP64 oracle on the host cores"},
        "cpu_baseline": {"value": val, "unit": "evals/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{n} of {N_POINTS} points per step, all {g.n} elements x {g.n_images} images"},
        "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_run(N, ctxs, geoms, n_req, scale, precision, seed, rate_hz=2000.0, max_wall_s=90.0):
    """Replay a seeded Poisson trace (rate_hz requests/s, sizes log-uniform in [1e2, 1e6]
    times `scale`, geometry uniform over the resident contexts) through the server;
    returns p50/p99 latency (submit -> outputs in host memory) and points/s.  No request is
    submitted after max_wall_s (the submitted ones are drained and reported)."""
    from paper_2606_24154_gb300 import inputs as I
    t_arr, sizes, geo = I.serving_trace(n_req, I.rng(4, seed), rate_hz=rate_hz, n_geometries=len(ctxs))
    sizes = np.maximum(1, (sizes * scale).astype(np.int64))
    reqs = []
    for k in range(n_req):
        g = geoms[geo[k]]
        pts = np.ascontiguousarray(I.cell_points(g, int(sizes[k]), I.rng(4, 1000 + k)))
        reqs.append((pts, np.empty(pts.shape[0]), np.empty((pts.shape[0], 3))))
    srv = N.nebem_server_create([c.h for c in ctxs])
    ids = [None] * n_req
    done = [False] * n_req
    break_cap = False
    t0 = time.perf_counter()
    i = 0
    first = 0  # oldest request not known to be complete
    while i < n_req or not all(done[:i]):
        now = time.perf_counter() - t0
        if now > 900.0:
            N.nebem_server_destroy(srv)
            raise RuntimeError("serving trace did not complete within 900 s")
        if now > max_wall_s and i < n_req:
            n_req = i  # capped: drain what was submitted
            break_cap = True
        while i < n_req and t_arr[i] <= now:
            ids[i] = N.nebem_server_submit(srv, int(geo[i]), reqs[i][0], reqs[i][1], reqs[i][2], precision)
            i += 1
        # one poll per round drives the server, which completes (and timestamps) every
        # finished request; then the oldest pending requests are checked in order
        while first < i and N.nebem_server_poll(srv, ids[first]):
            done[first] = True
            first += 1
        time.sleep(50e-6)
    for k in range(n_req):  # every request is complete by now; this only records it
        done[k] = done[k] or N.nebem_server_poll(srv, ids[k])
    ids, sizes = ids[:n_req], sizes[:n_req]
    times = np.array([N.nebem_server_request_times(srv, r) for r in ids])
    N.nebem_server_destroy(srv)
    print(f"bench: serving {n_req} requests at {rate_hz:g}/s x{scale:g} precision {precision}: "
          f"{time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
    lat = (times[:, 2] - times[:, 0]) * 1e3
    span = times[:, 2].max() - times[:, 0].min()
    return {"requests": n_req, "rate_hz": rate_hz, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "points_per_s": float(sizes.sum() / span),
            "points": int(sizes.sum()), "makespan_s": float(span), "size_scale": scale,
            "wall_s": time.perf_counter() - t0, "capped": break_cap}


def pointwise(a, ref):
    """largest per-point relative error |a_i - ref_i| / max(|ref_i|, 1e-6 max|ref|); rows of
    a 2-D array are vectors (E)"""
    if a.ndim == 1:
        r, d = ref.abs(), (a - ref).abs()
    else:
        r, d = ref.norm(dim=1), (a - ref).norm(dim=1)
    return float((d / r.clamp(min=1e-6 * float(r.max()))).max())


def timed_steps(step, stream, flush, steps, warmup, sampler=None, barrier=None):
    """W untimed steps, then K steps each bracketed by CUDA events on `stream`, with an L2
    flush (512 MB write) before each; `barrier` (ranks) and a device synchronisation on both
    sides of the timed region.  Returns the per-step ms and the wall time."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    if barrier:
        barrier()
        torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], time.perf_counter() - t0


def space_charge_section(N, g, n_car, steps, dev):
    """Dynamic space charge on the THGEM cell (1e6 point carriers, Gaussian cloud sigma
    0.1 mm in the hole, half ions): the mixed dynamic step, the carrier-carrier sum alone,
    and the FP64 GPU path on a sample of targets with the mixed sums' errors against it
    (per target, at the carriers and at points of the cell away from the net-neutral cloud)."""
    import torch
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import roofline as R
    pos, q = I.carrier_cloud(g, n_car, I.rng(3, 0))
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    N.nebem_space_charge(c.h, pos, q, 1e-6)
    N.nebem_step(c.h, 1, 1e-4, 1e-9, N.NEBEM_MIXED, n_car)  # warm-up
    N.nebem_space_charge(c.h, pos, q, 1e-6)
    torch.cuda.synchronize()
    t = time.perf_counter()
    N.nebem_step(c.h, steps, 1e-4, 1e-9, N.NEBEM_MIXED, n_car)
    s_step = (time.perf_counter() - t) / steps
    # the carrier-carrier sum alone (every carrier, self excluded)
    N.nebem_space_charge(c.h, pos, q, 1e-6)
    N.nebem_space_charge_eval(c.h, pos[:4096], N.NEBEM_MIXED)  # warm-up
    t = time.perf_counter()
    N.nebem_space_charge_eval(c.h, pos, N.NEBEM_MIXED, exclude_self=True)
    t_sum = time.perf_counter() - t
    pairs = n_car * (n_car - 1)
    meas = N.nebem_peak_rates(c.h)
    peak_ops = max(meas["ffma"], meas["ffma2_lanes"])  # measured FP32 lane-op peak
    mphi_all, mE_all = N.nebem_space_charge_eval(c.h, pos, N.NEBEM_MIXED, exclude_self=True)
    # FP64 path on samples: carriers and points of the cell.  Self exclusion needs the whole
    # carrier set as targets, so at the sampled carriers the FP64 sums include each carrier's
    # own term, ke q / s in phi (zero in E), which is taken out again.
    ns = 2048
    tgt = pos[:ns]
    t = time.perf_counter()
    rphi, rE = N.nebem_space_charge_eval(c.h, tgt, N.NEBEM_FP64)
    t64 = time.perf_counter() - t
    ke = 1.0 / (4.0 * np.pi * 8.8541878128e-12)
    rphi = rphi - ke * q[:ns] / 1e-6
    mphi, mE = mphi_all[:ns], mE_all[:ns]
    far = I.cell_points(g, 512, I.rng(3, 2))
    fphi64, fE64 = N.nebem_space_charge_eval(c.h, far, N.NEBEM_FP64)
    fphi, fE = N.nebem_space_charge_eval(c.h, far, N.NEBEM_MIXED)
    c.close()

    def per_target(a, ref):
        a, ref = torch.from_numpy(a), torch.from_numpy(ref)
        return {"pointwise": pointwise(a, ref),
                "normwise": float((a - ref).abs().max() / ref.abs().max()) if a.ndim == 1
                else float((a - ref).norm(dim=1).max() / ref.norm(dim=1).max())}

    return {"workload": f"thgem_cell N={g.n}, {n_car} carriers (Gaussian 0.1 mm, half ions), mu 1e-4 m^2/Vs, "
                        f"dt 1 ns", "steps": steps,
            "mixed_s_per_step": s_step,
            "carrier_pairs_per_s_in_step": (pairs + g.n * n_car) / s_step,
            "carrier_sum": {"s": t_sum, "pairs_per_s": pairs / t_sum,
                            "lane_op_frac": pairs * R.SC_OPS_PER_PAIR / t_sum / peak_ops,
                            "note": "host-timed nebem_space_charge_eval of all carriers at all carriers; "
                                    f"{R.SC_OPS_PER_PAIR} FP32 lane ops per pair; peak measured "
                                    "(nebem_peak_rates)"},
            "fp64_path": {"sample_targets": ns, "pairs_per_s": ns * (n_car - 1) / t64,
                          "speedup_mixed_over_fp64": (pairs / t_sum) / (ns * (n_car - 1) / t64)},
            "accuracy_vs_fp64": {"at_carriers_phi": per_target(mphi, rphi), "at_carriers_E": per_target(mE, rE),
                                 "away_from_cloud_phi": per_target(fphi, fphi64),
                                 "away_from_cloud_E": per_target(fE, fE64),
                                 "pointwise_form": "|d_i| / max(|ref_i|, 1e-6 max|ref|), E as a vector"}}


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import nebem as N

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    N.load()

    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import sharding as S
    g = I.thgem()
    # weak scaling: every rank evaluates its own points (seed stream = rank)
    pts_h = I.cell_points(g, args.points, I.rng(1, S.shard_seed_stream(rank)))
    n_el, n_img = g.n, g.n_images
    ctx = N.Context(device=local).set_geometry(g)
    sigma, info, _ = ctx.solve(N.NEBEM_MIXED)
    # the single FP32 pass (no refinement) on the same charge densities, for comparison
    single = N.Context(device=local, mixed_point_tol=0.0).set_geometry(g)
    single.set_sigma(sigma)

    stream = torch.cuda.Stream(device=dev)
    s_handle = stream.cuda_stream
    npts = pts_h.shape[0]
    pts = torch.from_numpy(pts_h).to(dev)
    phi = torch.empty(npts, dtype=torch.float64, device=dev)
    E = torch.empty((npts, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        N.nebem_eval_device(ctx.h, pts.data_ptr(), npts, phi.data_ptr(), E.data_ptr(), N.NEBEM_MIXED, s_handle)

    sampler = ClockSampler(local)
    torch.cuda.nvtx.range_push("timed")
    step_ms, wall = timed_steps(step, stream, flush, args.steps, args.warmup, sampler,
                                dist.barrier if world > 1 else None)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    stats = N.nebem_eval_stats(ctx.h)  # stage times and refined counts of the last timed step
    ms = statistics.mean(step_ms)
    evals = npts * n_el * n_img
    ms, total_evals = S.reduce_step_time(ms, evals, dev)
    value = total_evals / (ms * 1e-3)

    # ---- the single FP32 pass, same protocol
    phi1 = torch.empty_like(phi)
    E1 = torch.empty_like(E)

    def step1():
        N.nebem_eval_device(single.h, pts.data_ptr(), npts, phi1.data_ptr(), E1.data_ptr(), N.NEBEM_MIXED, s_handle)

    single_ms = statistics.mean(timed_steps(step1, stream, flush, args.steps, args.warmup)[0])
    single_value = evals / (single_ms * 1e-3)

    # ---- accuracy against the FP64 path on a sample, and the FP64 path's rate
    ns = min(args.fp64_points, npts)
    phi64 = torch.empty(ns, dtype=torch.float64, device=dev)
    E64 = torch.empty((ns, 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        N.nebem_eval_device(ctx.h, pts.data_ptr(), ns, phi64.data_ptr(), E64.data_ptr(), N.NEBEM_FP64, s_handle)
        b.record(stream)
    torch.cuda.synchronize()
    fp64_rate = ns * n_el * n_img / (a.elapsed_time(b) * 1e-3)
    accuracy = {"sample_points": ns, "reference": "FP64 GPU path (closed forms for every pair)",
                "pointwise_form": "|d_i| / max(|ref_i|, 1e-6 max|ref|), E as a vector"}
    for name, (p_, e_) in (("refined", (phi, E)), ("single_pass", (phi1, E1))):
        accuracy[name] = {"phi_pointwise": pointwise(p_[:ns], phi64), "E_pointwise": pointwise(e_[:ns], E64),
                          "phi_normwise": float((p_[:ns] - phi64).abs().max() / phi64.abs().max()),
                          "E_normwise": float((e_[:ns] - E64).norm(dim=1).max() / E64.norm(dim=1).max())}
    accuracy["sigma_refinement"] = {"iterations": info.iterations, "correction": info.correction}

    # ---- roofline of the dominant kernel: the first refinement level (two-float, FP32 lanes)
    from paper_2606_24154_gb300 import roofline as R
    peaks, peak_src = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    # peaks of the pipes, measured on this GPU (FP32 lanes: the better of scalar and packed FMA)
    meas = N.nebem_peak_rates(ctx.h)
    peak_ops = max(meas["ffma"], meas["ffma2_lanes"])
    peak_mufu = meas["mufu_rsqrt"]
    peak_fp64 = meas["dfma"]
    sub = pts_h[:min(ROOFLINE_SAMPLE, npts)]
    _, _, err_r, _ = N.nebem_eval_err(ctx.h, sub)
    _, _, err_s, _ = N.nebem_eval_err(single.h, sub)
    refined_sub = sub[(err_r != err_s).any(axis=1)]
    counts_l1 = R.tier_counts(g, refined_sub, sample=CHECK_SAMPLE)
    n_phi, n_E = stats.refined_level1_phi_only, stats.refined_level1_E_only
    ops_l1 = ((stats.refined_level1 - n_phi - n_E) * R.acc1_ops_per_point(counts_l1, n_el)
              + n_phi * R.acc1_ops_per_point(counts_l1, n_el, "phi") + n_E * R.acc1_ops_per_point(counts_l1, n_el, "E"))
    ach_l1 = ops_l1 / (stats.ms_level1 * 1e-3)
    counts = R.tier_counts(g, pts_h, sample=CHECK_SAMPLE)
    ops_fp32 = R.fp32_ops_per_launch(counts, npts / CHECK_SAMPLE)
    ach_fp32 = ops_fp32 / (stats.ms_fp32 * 1e-3)
    # ---- end to end through the host-buffer call (pinned host memory, copies inside)
    pts_pin = torch.from_numpy(pts_h).pin_memory()
    phi_pin = torch.empty(npts, dtype=torch.float64).pin_memory()
    E_pin = torch.empty((npts, 3), dtype=torch.float64).pin_memory()
    e2e_times = []
    import ctypes as C
    L = N.load()
    dp = C.POINTER(C.c_double)
    for k in range(max(2, args.steps // 2) + 1):
        t = time.perf_counter()
        rc = L.nebem_eval(ctx.h, C.cast(pts_pin.data_ptr(), dp), npts, C.cast(phi_pin.data_ptr(), dp),
                          C.cast(E_pin.data_ptr(), dp), N.NEBEM_MIXED)
        if rc != 0:
            raise N.NebemError(rc, "nebem_eval")
        if k > 0:
            e2e_times.append(time.perf_counter() - t)
    e2e_ms, _ = S.reduce_step_time(statistics.mean(e2e_times) * 1e3, evals, dev)
    e2e_val = total_evals / (e2e_ms * 1e-3)

    # ---- solve of the same geometry: mixed (FP32 LU + FP64 refinement) vs plain FP64
    solve = {}
    for name, prec in ((("mixed", N.NEBEM_MIXED), ("fp64", N.NEBEM_FP64)) if world == 1 else ()):
        c2 = N.Context(device=local).set_geometry(g)
        _, inf, _ = c2.solve(prec)
        solve[name] = {"ms_fill": inf.ms_fill, "ms_factor": inf.ms_factor, "ms_solve": inf.ms_solve,
                       "refinement_iterations": inf.iterations}
        # weighting fields of every conductor (Sec. 2.1) with the retained factors: the k
        # right-hand sides through each sweep together, against k single unit-voltage solves
        k = len(g.voltages)
        ro = list(range(k))
        N.nebem_weighting_fields(c2.h, ro, prec, g.n)  # warm-up (work space)
        t = time.perf_counter()
        W, winf, _ = N.nebem_weighting_fields(c2.h, ro, prec, g.n)
        wall_multi = time.perf_counter() - t
        ms_single, t = 0.0, time.perf_counter()
        for r in ro:
            v = np.zeros(k)
            v[r] = 1.0
            N.nebem_set_bc(c2.h, v)
            _, sinf, _ = c2.solve(prec)
            ms_single += sinf.ms_solve
        wall_single = time.perf_counter() - t
        solve[name]["weighting"] = {"readouts": k, "ms_multi_rhs": winf.ms_solve, "ms_k_single_solves": ms_single,
                                    "wall_ms_multi_rhs": wall_multi * 1e3, "wall_ms_k_single_solves": wall_single * 1e3,
                                    "refinement_iterations": winf.iterations, "residual": winf.residual}
        N.nebem_set_bc(c2.h, g.voltages)
        c2.close()

    # ---- serving: configs 0-2 resident (cube, THGEM cell, double THGEM), continuous batching
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        from paper_2606_24154_gb300 import inputs as I
        geoms = [I.cube(), g, I.double_thgem()]
        sctx = [N.Context(device=local).set_geometry(geoms[0]), ctx, N.Context(device=local).set_geometry(geoms[2])]
        t = time.perf_counter()
        sctx[0].solve(N.NEBEM_MIXED)
        _, inf2, _ = sctx[2].solve(N.NEBEM_MIXED)
        setup = time.perf_counter() - t
        print(f"bench: serving setup {setup:.1f} s", file=sys.stderr, flush=True)
        # the same three geometries and densities with the single FP32 pass (no refinement)
        single_s = []
        for k, c_ in enumerate(sctx):
            c1 = N.Context(device=local, mixed_point_tol=0.0).set_geometry(geoms[k])
            c1.set_sigma(c_.sigma())
            single_s.append(c1)
        small = 0.01
        serving = {"trace": "Poisson arrivals, sizes log-uniform 1e2..1e6 (x size_scale), geometry uniform over "
                            "3 resident (cube, THGEM cell, double THGEM)",
                   "full_trace_2000_per_s": serving_run(N, sctx, geoms, args.serving_requests, 1.0, N.NEBEM_MIXED,
                                                        0, 2000.0, 60.0),
                   "note": "the full-size trace at 2000/s is an overload (drain rate); the rate sweeps use the "
                           "trace with sizes x 0.01, below and above each mode's capacity",
                   "sweep_mixed_single_pass": [serving_run(N, single_s, geoms, n, small, N.NEBEM_MIXED, 2 + i, rate,
                                                           30.0)
                                               for i, (rate, n) in enumerate(((50.0, 200), (150.0, 200),
                                                                               (2000.0, 200)))],
                   "sweep_mixed_refined": [serving_run(N, sctx, geoms, n, small, N.NEBEM_MIXED, 2 + i, rate, 40.0)
                                           for i, (rate, n) in enumerate(((4.0, 100), (8.0, 100), (2000.0, 40)))],
                   "sweep_fp64": [serving_run(N, sctx, geoms, 16, small, N.NEBEM_FP64, 2, 0.4, 60.0)],
                   "double_thgem_solve": {"elements": geoms[2].n, "ms_fill": inf2.ms_fill,
                                          "ms_factor_fp32": inf2.ms_factor, "ms_refine": inf2.ms_solve,
                                          "iterations": inf2.iterations, "correction": inf2.correction},
                   "setup_s": setup}
        for c1 in single_s:
            c1.close()
        sctx[0].close()
        sctx[2].close()

    space = None
    if rank == 0 and world == 1 and not args.no_space_charge:
        t = time.perf_counter()
        space = space_charge_section(N, g, SC_CARRIERS, 2, dev)
        space["section_s"] = time.perf_counter() - t
        print(f"bench: space charge {space['section_s']:.1f} s", file=sys.stderr, flush=True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, dt = oracle_rate(g, pts_h, ORACLE_SAMPLE)
        cpu = {"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"{ORACLE_SAMPLE} of {npts} points, all {n_el} elements x {n_img} images "
                         f"({dt:.1f} s FP64 on the host)"}

    if rank == 0:
        line = {
            "metric": HEADLINE_METRIC,
            "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"thgem_cell N={n_el} images={n_img} points={npts} mixed eval, "
                                   f"refined to 1e-6 per point",
                       "elements": n_el, "images": n_img, "points_per_gpu": npts,
                       "l2": "flushed between timed steps (512 MB write)", "parallelism": f"points sharded x{world}"},
            "stages": {"ms_fp32_pass": stats.ms_fp32, "ms_refine_level1": stats.ms_level1,
                       "ms_refine_level2": stats.ms_level2, "points": stats.points,
                       "refined_level1": stats.refined_level1, "refined_level2": stats.refined_level2,
                       "refined_level1_phi_only": stats.refined_level1_phi_only,
                       "refined_level1_E_only": stats.refined_level1_E_only},
            "single_pass": {"value": single_value, "unit": "evals/s", "ms_per_step": single_ms,
                            "note": "the FP32 pass alone (mixed_point_tol = 0): its per-point error is in "
                                    "accuracy.single_pass"},
            "accuracy": accuracy,
            "fp64_path": {"value": fp64_rate, "unit": "evals/s", "sample_points": ns,
                          "speedup_refined_over_fp64": value / world / fp64_rate,
                          "roofline": {"bound": "fp64",
                                       "achieved": fp64_rate * R.FP64_INST_PER_PAIR / 1e12,
                                       "peak": peak_fp64 / 1e12,
                                       "unit": "T FP64 instructions/s",
                                       "frac": fp64_rate * R.FP64_INST_PER_PAIR / peak_fp64,
                                       "note": "278 FP64 instructions per pair (ncu count); peak = measured FP64 "
                                               "FMA rate (nebem_peak_rates)"}},
            "roofline": {"bound": "alu", "kernel": "k_eval_acc_far<1> (first refinement level, two-float)",
                         "achieved": ach_l1 / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": ach_l1 / peak_ops, "traffic": None,
                         "peak_source": "measured on this GPU (nebem_peak_rates: the better of scalar and "
                                        "packed FP32 FMA, lanes counted)",
                         "peak_unit_counts": R.fp32_peak_ops(sm_max) / 1e12,
                         "peaks_measured": {k: v / 1e12 for k, v in meas.items()},
                         "note": "FP32 lane operations counted from the code (roofline.ACC1_*) x the refined "
                                 "points' pair and node counts / the level's event time (flag step and FP64 near "
                                 "pairs included); traffic: no capture of this kernel version",
                         "fp32_pass": {"kernel": "k_eval_far", "achieved": ach_fp32 / 1e12,
                                       "frac": ach_fp32 / peak_ops,
                                       "mufu_frac": counts["nodes"] * (npts / CHECK_SAMPLE) / (stats.ms_fp32 * 1e-3)
                                       / peak_mufu}},
            "tiers": counts,
            "tiers_refined": counts_l1,
            "solve_thgem": solve,
            "serving": serving,
            "space_charge": space,
            "e2e": {"value": e2e_val, "unit": "evals/s", "h2d_bytes_per_step": int(pts_pin.numel() * 8),
                    "d2h_bytes_per_step": int((phi_pin.numel() + E_pin.numel()) * 8)},
            "cpu_baseline": cpu,
            # per step: k_bin_keys, k_bin_scan, k_bin_scatter, k_eval_far, k_eval_near, then
            # k_flag + k_eval_acc_far + near per refinement level
            "gpu_launches": 11 * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    single.close()
    ctx.close()
    return 0


def run_double_thgem_solve(args):
    """Double THGEM (40,368 elements, 25 images): the mixed solve (mixed fill, FP32 LU, FP64
    refinement to 1e-8) against the plain FP64 solve (FP64 fill, FP64 LU); one step = one
    full mixed solve in a fresh context."""
    import torch

    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import nebem as N
    from paper_2606_24154_gb300 import roofline as R
    B.build()
    g = I.double_thgem()
    res = {"mixed": [], "fp64": None}
    sig_m = None
    for step in range(max(1, args.steps)):
        c = N.Context().set_geometry(g)
        t = time.perf_counter()
        sig_m, inf, _ = c.solve(N.NEBEM_MIXED)
        res["mixed"].append({"wall_s": time.perf_counter() - t, "ms_fill": inf.ms_fill, "ms_factor": inf.ms_factor,
                             "ms_refine": inf.ms_solve, "iterations": inf.iterations,
                             "correction": inf.correction})
        c.close()
    c = N.Context().set_geometry(g)
    t = time.perf_counter()
    sig_d, inf, _ = c.solve(N.NEBEM_FP64)
    res["fp64"] = {"wall_s": time.perf_counter() - t, "ms_fill": inf.ms_fill, "ms_factor": inf.ms_factor,
                   "ms_solve": inf.ms_solve}
    # residual |K sigma - b| / sum_j |K_ij sigma_j| of both solutions on sampled rows of the
    # FP64 matrix (b = the conductor voltage on conductor rows, 0 on interface rows)
    rows = np.random.default_rng(5).choice(g.n, 16, replace=False)
    cols = np.arange(g.n)
    bvec = np.where(g.elements["bc"] == I.BC_CONDUCTOR, g.voltages[np.maximum(g.elements["conductor"], 0)], 0.0)
    resid = {"mixed": 0.0, "fp64": 0.0}
    for i in rows:
        Ki = N.nebem_matrix_entries(c.h, np.full(g.n, i), cols)
        for name, sg in (("mixed", sig_m), ("fp64", sig_d)):
            tt = Ki * sg
            resid[name] = max(resid[name], float(abs(tt.sum() - bvec[i]) / np.abs(tt).sum()))
    c.close()
    err = float(np.abs(sig_m - sig_d).max() / np.abs(sig_d).max())
    n = g.n
    oracle = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        rows = np.repeat(np.arange(4), n)
        cols = np.tile(np.arange(n), 4)
        frate, cores = _oracle_rate(lambda: O.fill_entries(g, rows, cols), 4 * n * g.n_images)
        A = np.random.default_rng(0).random((2048, 2048)) + 2048 * np.eye(2048)
        lrate, _ = _oracle_rate(lambda: O.lu_factor(A), (2.0 / 3.0) * 2048 ** 3)
        oracle = {"fill_pairs_per_s": frate, "fill_cores": cores, "lu_flops_per_s_n2048": lrate, "lu_cores": 1,
                  "sample": "4 full rows of the 40k matrix (all images); LU of a 2048 x 2048 matrix (one thread)"}
    best = min(r["ms_factor"] for r in res["mixed"])
    fill_ms = min(r["ms_fill"] for r in res["mixed"])
    cts = R.fill_tier_counts(g)
    fops = R.fill_ops(cts, n)
    peaks, _ = load_peaks()
    fpeak = R.fp32_peak_ops(peaks.get("sm_max_mhz", 2070.0))
    pairs = n * n * g.n_images
    line = {"metric": "double THGEM solve: mixed fill + FP32 LU + FP64 refinement vs FP64 fill + FP64 LU",
            "workload": f"double_thgem N={n} images={g.n_images}",
            "value": min(r["wall_s"] for r in res["mixed"]), "unit": "s (whole mixed solve)",
            "higher_is_better": False, "fp64_solve_s": res["fp64"]["wall_s"],
            "lu_fp32_tflops": (2.0 / 3.0) * n ** 3 / (best * 1e-3) / 1e12, "sigma_rel_err_mixed_vs_fp64": err,
            "row_residual_fp64_matrix": resid,
            "accuracy_note": "residual of each sigma on 16 sampled rows of the FP64 matrix, relative to the row's "
                             "sum of |terms|: the refined mixed sigma solves the system more exactly than the plain "
                             "FP64 LU solve, whose forward error at this size is what sigma_rel_err shows",
            "fp64_lu_tflops": (2.0 / 3.0) * n ** 3 / (res["fp64"]["ms_factor"] * 1e-3) / 1e12, "runs": res,
            "fill_pairs_per_s_mixed": pairs / (fill_ms * 1e-3),
            "fill_pairs_per_s_fp64": pairs / (res["fp64"]["ms_fill"] * 1e-3),
            "fill_roofline": {"bound": "alu", "achieved": fops / (fill_ms * 1e-3) / 1e12, "peak": fpeak / 1e12,
                              "unit": "Tops/s", "frac": fops / (fill_ms * 1e-3) / fpeak,
                              "ops_per_pair": fops / pairs, "tiers": cts,
                              "note": "two-float FP32 operations of the mixed fill (counted per row-column, far "
                                      "pair and Gauss node from the kernel code) / fill time (far + near kernels)"},
            "oracle_fp64": oracle}
    print(json.dumps(line), flush=True)
    return 0


def run_space_charge(args):
    """Dynamic space charge on the THGEM cell: 1e6 point carriers (Gaussian cloud, sigma
    0.1 mm, half ions), per step: known-charge RHS at the collocation points, solve with
    the retained factors, E at every carrier from all elements (images) and all other
    carriers, drift x += sign(q) mu E dt (mu = 1e-4 m^2/Vs, dt = 1 ns)."""
    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import nebem as N
    B.build()
    g = I.thgem()
    n_car = args.points
    pos, q = I.carrier_cloud(g, n_car, I.rng(3, 0))
    out = {}
    for name, prec in (("mixed", N.NEBEM_MIXED),):
        c = N.Context().set_geometry(g)
        c.solve(prec)
        N.nebem_space_charge(c.h, pos, q, 1e-6)
        N.nebem_step(c.h, max(1, args.warmup), 1e-4, 1e-9, prec, n_car)
        N.nebem_space_charge(c.h, pos, q, 1e-6)
        t = time.perf_counter()
        N.nebem_step(c.h, args.steps, 1e-4, 1e-9, prec, n_car)
        dt = (time.perf_counter() - t) / args.steps
        pairs = n_car * (n_car - 1) + g.n * n_car
        out[name] = {"s_per_step": dt, "carrier_pairs_per_s": pairs / dt,
                     "element_evals_per_s": n_car * g.n * g.n_images / dt}
        c.close()
    # the same steps with the carriers reduced to line charges (Alg. 3) before every step
    voxel = [20e-6, 20e-6, 40e-6]
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    N.nebem_space_charge(c.h, pos, q, 1e-6)
    nl = N.nebem_space_charge_lines(c.h, voxel)
    N.nebem_step(c.h, max(1, args.warmup), 1e-4, 1e-9, N.NEBEM_MIXED, n_car)
    N.nebem_space_charge(c.h, pos, q, 1e-6)
    N.nebem_space_charge_lines(c.h, voxel)
    t = time.perf_counter()
    N.nebem_step(c.h, args.steps, 1e-4, 1e-9, N.NEBEM_MIXED, n_car)
    dt = (time.perf_counter() - t) / args.steps
    t = time.perf_counter()
    N.nebem_space_charge_eval(c.h, pos, N.NEBEM_MIXED)
    t_sum = time.perf_counter() - t
    out["mixed_lines"] = {"s_per_step": dt, "voxel_m": voxel, "lines": nl,
                          "line_pairs_per_step": n_car * nl,
                          "line_sum_at_carriers_s_host_api": t_sum,
                          "line_pairs_per_s_host_api": n_car * nl / t_sum,
                          "element_evals_per_s": n_car * g.n * g.n_images / dt}
    c.close()
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        nt = 256
        rate, cores = _oracle_rate(lambda: O.space_charge(pos, q, tgt=pos[:nt], soft=1e-6), nt * n_car)
        lines = O.voxel_lines(pos, q, voxel)
        lrate, _ = _oracle_rate(lambda: O.line_charge(lines, pos[:2048]), 2048 * len(lines))
        out["oracle_fp64"] = {"carrier_pairs_per_s": rate, "line_pairs_per_s": lrate, "cores": cores,
                              "sample": f"{nt} carriers x all {n_car} sources; 2048 carriers x all lines"}
    line = {"metric": "dynamic space-charge step time", "workload": f"thgem_cell N={g.n} carriers={n_car}",
            "value": out["mixed"]["s_per_step"], "unit": "s/step", "higher_is_better": False, "steps": args.steps,
            "detail": out}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_rate(fn, units):
    """The FP64 oracle timed on the host cores for `units` units of work: (units/s, threads)."""
    from oracle import oracle as O
    O.build()
    t = time.perf_counter()
    fn()
    return units / (time.perf_counter() - t), O.num_threads()


def run_fastvol(args):
    """FastVolume (Sec. 3.3) on the THGEM cell: a map on a rectilinear grid graded through
    the foil (node values from the mixed evaluation), then trilinear lookups at --points
    points in the cell; build time, lookup rate and interpolation error in the drift region
    against the direct evaluation."""
    import torch

    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import nebem as N
    B.build()
    g = I.thgem()
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    p = g.pitch
    # nodes kept off element edges and vertices (where the in-plane field diverges) by
    # small offsets, and strictly between the electrode planes
    ax = np.linspace(-0.5 * p, 0.5 * p, 41) + 1.3e-6
    ay = np.linspace(-p / np.sqrt(3), p / np.sqrt(3), 47) + 0.7e-6
    az = np.concatenate([np.linspace(g.z_range[0] + 2e-6, -0.6e-3, 30), np.linspace(-0.59e-3, 0.59e-3, 60) + 1.1e-6,
                         np.linspace(0.6e-3, g.z_range[1] - 2e-6, 30)])
    nodes = len(ax) * len(ay) * len(az)
    torch.cuda.synchronize()
    t = time.perf_counter()
    N.nebem_fastvol_build(c.h, ax, ay, az, N.NEBEM_MIXED)
    t_build = time.perf_counter() - t
    pts = I.cell_points(g, args.points, I.rng(1, 0))
    d_pts = torch.from_numpy(pts).cuda()
    d_phi = torch.empty(args.points, dtype=torch.float64, device="cuda")
    d_E = torch.empty((args.points, 3), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    times = []
    for step in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        N.nebem_fastvol_eval_device(c.h, d_pts.data_ptr(), args.points, d_phi.data_ptr(), d_E.data_ptr(),
                                    st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        if step >= args.warmup:
            times.append(e0.elapsed_time(e1) * 1e-3)
    t_look = min(times)
    # direct evaluation of the same points (mixed) for the error and the speed-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    d_phi2 = torch.empty_like(d_phi)
    d_E2 = torch.empty_like(d_E)
    N.nebem_eval_device(c.h, d_pts.data_ptr(), args.points, d_phi2.data_ptr(), d_E2.data_ptr(), N.NEBEM_MIXED,
                        st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    t_direct = e0.elapsed_time(e1) * 1e-3
    phi, E, phi2, E2 = (x.cpu().numpy() for x in (d_phi, d_E, d_phi2, d_E2))
    drift = (pts[:, 2] > 1.2e-3) & (pts[:, 2] < 3.0e-3)
    relE = np.linalg.norm(E - E2, axis=1) / np.linalg.norm(E2, axis=1)
    c.close()
    line = {"metric": "FastVolume lookups", "workload": f"thgem_cell N={g.n} grid={len(ax)}x{len(ay)}x{len(az)} "
            f"points={args.points}", "value": args.points / t_look, "unit": "points/s", "higher_is_better": True,
            "steps": args.steps, "detail": {
                "nodes": nodes, "build_s": t_build, "lookup_s": t_look, "direct_mixed_eval_s": t_direct,
                "speedup_lookup_vs_direct": t_direct / t_look,
                "drift_region_E_rel_err_median": float(np.median(relE[drift])),
                "drift_region_E_rel_err_p99": float(np.quantile(relE[drift], 0.99)),
                "all_points_E_rel_err_median": float(np.median(relE)),
                "non_finite_lookups": int((~np.isfinite(E)).any(axis=1).sum())}}
    print(json.dumps(line), flush=True)
    return 0


def run_am(args):
    """Adaptive Modelling on the THGEM cell with 11 x 11 periodic copies (solved in mixed
    precision): potential and field at --points points (mixed) for PrimAfter = -1 (every
    copy by elements) and 4, 3, 2, 1, 0; time per map and the largest error against the
    full evaluation, as in the paper's PrimAfter table."""
    import torch

    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import nebem as N
    B.build()
    g = I.thgem()
    g.img_lo, g.img_hi = -5, 5
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    pts = I.cell_points(g, args.points, I.rng(1, 0))
    d_pts = torch.from_numpy(pts).cuda()
    d_phi = torch.empty(args.points, dtype=torch.float64, device="cuda")
    d_E = torch.empty((args.points, 3), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()  # a real stream: a NULL handle would mean the context's own
    rows, ref = [], None
    for pa in (-1, 4, 3, 2, 1, 0):
        N.nebem_set_primitives(c.h, g.primitives, g.prim_of, pa)
        times = []
        for step in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            N.nebem_eval_device(c.h, d_pts.data_ptr(), args.points, d_phi.data_ptr(), d_E.data_ptr(),
                                N.NEBEM_MIXED, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            if step >= args.warmup:
                times.append(e0.elapsed_time(e1) * 1e-3)
        phi, E = d_phi.cpu().numpy(), d_E.cpu().numpy()
        if ref is None:
            ref = (phi.copy(), E.copy())
        rows.append({"prim_after": pa, "s_per_map": min(times),
                     "phi_max_rel_err": float(np.abs(phi - ref[0]).max() / np.abs(ref[0]).max()),
                     "E_max_rel_err": float(np.abs(E - ref[1]).max() / np.abs(ref[1]).max())})
    sig = c.sigma()
    c.close()
    oracle = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        sample = pts[:32]
        r_full, cores = _oracle_rate(lambda: O.eval_points(g, sig, sample), 32)
        r_am, _ = _oracle_rate(lambda: O.eval_am(g, sig, g.primitives, g.prim_of, 1, sample), 32)
        oracle = {"points_per_s_full": r_full, "points_per_s_prim_after_1": r_am, "cores": cores,
                  "sample": "32 of the map's points"}
    full = rows[0]["s_per_map"]
    line = {"metric": "Adaptive Modelling map time", "workload":
            f"thgem_cell N={g.n} primitives={len(g.primitives)} images=121 points={args.points} mixed",
            "value": min(r["s_per_map"] for r in rows if r["prim_after"] == 1), "unit": "s/map (PrimAfter=1)",
            "higher_is_better": False, "steps": args.steps, "speedup_prim_after_1": full / rows[4]["s_per_map"],
            "detail": rows, "oracle_fp64": oracle}
    print(json.dumps(line), flush=True)
    return 0


def run_lu(args):
    """Dense LU of an n x n matrix (n = --points) on the device, FP32 (tcgen05 trailing
    updates) and FP64; one step = one factorisation of a fresh copy.  The matrix is a
    seeded random matrix plus n on the diagonal (well conditioned, pivoting still active)."""
    import torch

    from paper_2606_24154_gb300 import build as B
    from paper_2606_24154_gb300 import nebem as N
    B.build()
    n = args.points
    gen = torch.Generator(device="cuda").manual_seed(20261203)
    A0 = torch.rand((n, n), generator=gen, device="cuda", dtype=torch.float64) - 0.5
    A0 += torch.eye(n, device="cuda", dtype=torch.float64) * 0.1 * n ** 0.5
    piv = torch.empty(n, dtype=torch.int32, device="cuda")
    c = N.Context()
    out = {}
    st = torch.cuda.Stream()
    for name, dt, fn in (("fp32_tc", torch.float32, N.nebem_lu_factor_device_f32),
                         ("fp64", torch.float64, N.nebem_lu_factor_device)):
        A = torch.empty((n, n), dtype=dt, device="cuda")
        times = []
        for step in range(args.warmup + args.steps):
            A.copy_(A0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(c.h, A.data_ptr(), n, piv.data_ptr(), st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            if step >= args.warmup:
                times.append(e0.elapsed_time(e1) * 1e-3)
        t = min(times)
        out[name] = {"s": t, "tflops": (2.0 / 3.0) * n ** 3 / t / 1e12}
        del A
    c.close()
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        A = np.random.default_rng(0).random((2048, 2048)) + 2048 * np.eye(2048)
        lrate, cores = _oracle_rate(lambda: O.lu_factor(A), (2.0 / 3.0) * 2048 ** 3)
        out["oracle_fp64"] = {"flops_per_s": lrate, "cores": 1, "sample": "n = 2048 (the oracle's LU is one thread)"}
    line = {"metric": "dense LU factorisation", "workload": f"random n={n} (+diagonal), column-major",
            "value": out["fp32_tc"]["tflops"], "unit": "TFLOP/s (2/3 n^3)", "higher_is_better": True,
            "steps": args.steps, "detail": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "double_thgem_solve":
        return run_double_thgem_solve(args)
    if args.workload == "space_charge":
        return run_space_charge(args)
    if args.workload == "lu":
        return run_lu(args)
    if args.workload == "am":
        return run_am(args)
    if args.workload == "fastvol":
        return run_fastvol(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
